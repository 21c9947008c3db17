"""Seeded optical properties, heat loads and ray budgets for the synthetic workloads.

Parameter generators only. The five workloads follow the case studies the build is
measured on (sizes in the docstring of ``workload``); emissivities are drawn with
numpy's PCG64 and passed to both the oracle and the library as data.
"""
from __future__ import annotations

import numpy as np

from . import meshes


def optical_sets(n_faces: int, n_sets: int = 1, lo: float = 0.1, hi: float = 0.9, seed: int = 1):
    """eps ~ U[lo, hi] per face and set (set s uses seed + s), rho = 1 - eps (opaque surfaces)."""
    eps = np.stack([np.random.Generator(np.random.PCG64(seed + s)).uniform(lo, hi, n_faces)
                    for s in range(n_sets)])
    return eps.astype(np.float64), (1.0 - eps).astype(np.float64)


def heat_loads(n_faces: int, lo: float = 0.0, hi: float = 50.0, seed: int = 3):
    """Q_i ~ U[lo, hi] W per node."""
    return np.random.Generator(np.random.PCG64(seed)).uniform(lo, hi, n_faces).astype(np.float64)


def uniform_rays(n_faces: int, per_face: int):
    return np.full(n_faces, int(per_face), dtype=np.int64)


def _patch_areas(mesh: meshes.Mesh) -> np.ndarray:
    """Planar face areas from the vertex positions (used only to share out the ray budget)."""
    v = mesh.verts.astype(np.float64)
    t = mesh.tris
    cr = np.cross(v[t[:, 1]] - v[t[:, 0]], v[t[:, 2]] - v[t[:, 0]])
    a = 0.5 * np.linalg.norm(cr, axis=1)
    return np.bincount(mesh.tri_face, weights=a, minlength=mesh.n_faces)


def rays_by_area(mesh: meshes.Mesh, total: int):
    """Ray budget split by face area: floor(R*A_i/sum A), remainder to the largest
    fractional parts, at least one ray per face; the counts sum to ``total``."""
    area = _patch_areas(mesh)
    share = total * area / area.sum()
    n = np.maximum(np.floor(share).astype(np.int64), 1)
    rem = int(total - n.sum())
    if rem > 0:
        order = np.argsort(-(share - np.floor(share)), kind="stable")
        n[order[:rem]] += 1
    return n


def workload(name: str, rays_scale: float = 1.0):
    """The synthetic case-study workloads.

    cube       closed unit cube, 6 faces, 1e5 rays per face, eps = 0.8, rho = 0.2.
    plates     two 1 m plates 0.5 m apart, 16x16 sub-faces each (512 faces, 1,024
               triangles), 1e6 rays per sub-face (5.12e8), eps ~ U[0.1, 0.9] (seed 1).
    small_sat  0.3x0.3x0.6 m body + four hinged panels at 45 deg, 20,736 triangles,
               2,048 faces, 1e8 rays split by area, eps ~ U[0.05, 0.9] (seed 2).
    thermal    the plates mesh with Q ~ U[0, 50] W (seed 3) and a 3 K sink.
    plates_sided  the plates mesh with both sides of every sub-face radiating (Sec. 5.2:
               two-faced nodes, C_i = 2): 1e6 rays per side (1.024e9), rows 2i+X of
               side X; eps ~ U[0.1, 0.9] per side (seed 4), rho = 1 - eps.
    spacecraft ~200k triangles, 10,240 faces, 1e9 rays split by area, 16 eps/rho sets
               eps ~ U[0.05, 0.9] (seeds 10..25).
    ``rays_scale`` multiplies the ray budget (tests use small fractions).
    """
    if name == "cube":
        m = meshes.cube()
        rays = uniform_rays(m.n_faces, max(1, int(1e5 * rays_scale)))
        eps = np.full((1, m.n_faces), 0.8)
        rho = np.full((1, m.n_faces), 0.2)
        return dict(mesh=m, rays=rays, seed=0, eps=eps, rho=rho, open=False)
    if name in ("plates", "thermal"):
        m = meshes.plates(16)
        rays = uniform_rays(m.n_faces, max(1, int(1e6 * rays_scale)))
        eps, rho = optical_sets(m.n_faces, 1, 0.1, 0.9, seed=1)
        d = dict(mesh=m, rays=rays, seed=0, eps=eps, rho=rho, open=True)
        if name == "thermal":
            d.update(Q=heat_loads(m.n_faces, seed=3), T_sink=3.0)
        return d
    if name == "plates_sided":
        m = meshes.plates(16)
        rays = uniform_rays(2 * m.n_faces, max(1, int(1e6 * rays_scale)))
        eps, rho = optical_sets(2 * m.n_faces, 1, 0.1, 0.9, seed=4)
        return dict(mesh=m, rays=rays, seed=0, eps=eps, rho=rho, open=True,
                    faces_per_node=np.full(m.n_faces, 2, np.int32))
    if name == "small_sat":
        m = meshes.small_sat()
        rays = rays_by_area(m, max(m.n_faces, int(1e8 * rays_scale)))
        eps, rho = optical_sets(m.n_faces, 1, 0.05, 0.9, seed=2)
        return dict(mesh=m, rays=rays, seed=0, eps=eps, rho=rho, open=True)
    if name == "spacecraft":
        m = meshes.spacecraft()
        rays = rays_by_area(m, max(m.n_faces, int(1e9 * rays_scale)))
        eps, rho = optical_sets(m.n_faces, 16, 0.05, 0.9, seed=10)
        return dict(mesh=m, rays=rays, seed=0, eps=eps, rho=rho, open=True)
    raise ValueError(f"unknown workload {name!r}")
