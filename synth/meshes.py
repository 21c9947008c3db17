"""Deterministic triangle meshes shaped like the thesis's case studies.

Every mesh is a list of planar parallelogram patches. A patch is split into a
grid of quads (two triangles each, wound so that (b-a) x (c-a) points along the
patch's front normal U x V); its quads are then grouped, in serpentine order,
into contiguous runs that form the faces (the rows of the view-factor matrix).
Faces never straddle patches, so every face is planar.

Geometry only: vertex positions, triangle indices and the triangle -> face map.
"""
from __future__ import annotations

import dataclasses
import hashlib

import numpy as np


@dataclasses.dataclass
class Mesh:
    name: str
    verts: np.ndarray      # float32 [V, 3]
    tris: np.ndarray       # int32   [T, 3]
    tri_face: np.ndarray   # int32   [T]
    n_faces: int
    patch_of_face: np.ndarray  # int32 [N]: the patch each face belongs to
    n_patches: int

    @property
    def n_tris(self) -> int:
        return int(self.tris.shape[0])

    def digest(self) -> str:
        h = hashlib.sha256()
        for a in (self.verts, self.tris, self.tri_face):
            h.update(np.ascontiguousarray(a).tobytes())
        return h.hexdigest()[:16]


def _split_counts(total: int, weights) -> np.ndarray:
    """Largest-remainder split of ``total`` items over ``weights`` (each >= 1)."""
    w = np.asarray(weights, dtype=np.float64)
    share = total * w / w.sum()
    base = np.maximum(np.floor(share).astype(np.int64), 1)
    rem = total - int(base.sum())
    if rem > 0:
        order = np.argsort(-(share - np.floor(share)), kind="stable")
        for k in order[:rem]:
            base[k] += 1
    elif rem < 0:
        order = np.argsort(share - np.floor(share), kind="stable")
        for k in order:
            if rem == 0:
                break
            if base[k] > 1:
                base[k] -= 1
                rem += 1
    return base


def patch_mesh(name, patches, faces_per_patch=None):
    """Build a mesh from patches (P, U, V, nu, nv).

    ``faces_per_patch[p]`` faces are made from patch p's nu*nv quads by cutting its
    serpentine quad sequence into near-equal contiguous runs (None: one face per quad).
    """
    verts, tris, tri_face, patch_of_face = [], [], [], []
    v_base = 0
    face_base = 0
    for p, (P, U, V, nu, nv) in enumerate(patches):
        P = np.asarray(P, np.float64)
        U = np.asarray(U, np.float64)
        V = np.asarray(V, np.float64)
        ii, jj = np.meshgrid(np.arange(nu + 1), np.arange(nv + 1), indexing="ij")
        grid = P + (ii[..., None] / nu) * U + (jj[..., None] / nv) * V
        verts.append(grid.reshape(-1, 3))
        vid = lambda i, j: v_base + i * (nv + 1) + j  # noqa: E731
        order = []
        for j in range(nv):
            row = range(nu) if j % 2 == 0 else range(nu - 1, -1, -1)
            order.extend((i, j) for i in row)
        nq = nu * nv
        nf = nq if faces_per_patch is None else int(faces_per_patch[p])
        if nf < 1 or nf > nq:
            raise ValueError("faces per patch must be in [1, quads]")
        bounds = np.floor(np.arange(nf + 1) * nq / nf).astype(np.int64)
        for f in range(nf):
            for q in range(bounds[f], bounds[f + 1]):
                i, j = order[q]
                a, b, c, d = vid(i, j), vid(i + 1, j), vid(i + 1, j + 1), vid(i, j + 1)
                tris.append((a, b, c))
                tris.append((a, c, d))
                tri_face.extend((face_base + f, face_base + f))
            patch_of_face.append(p)
        face_base += nf
        v_base += (nu + 1) * (nv + 1)
    return Mesh(name=name,
                verts=np.ascontiguousarray(np.concatenate(verts), dtype=np.float32),
                tris=np.ascontiguousarray(np.array(tris, dtype=np.int32)),
                tri_face=np.ascontiguousarray(np.array(tri_face, dtype=np.int32)),
                n_faces=face_base,
                patch_of_face=np.array(patch_of_face, dtype=np.int32),
                n_patches=len(patches))


def cube():
    """Closed unit cube [0,1]^3: 6 inward-facing square faces, 12 triangles."""
    e = np.eye(3)
    patches = [
        ((0, 0, 0), e[1], e[2], 1, 1),  # x = 0, normal +x
        ((1, 0, 0), e[2], e[1], 1, 1),  # x = 1, normal -x
        ((0, 0, 0), e[2], e[0], 1, 1),  # y = 0, normal +y
        ((0, 1, 0), e[0], e[2], 1, 1),  # y = 1, normal -y
        ((0, 0, 0), e[0], e[1], 1, 1),  # z = 0, normal +z
        ((0, 0, 1), e[1], e[0], 1, 1),  # z = 1, normal -z
    ]
    return patch_mesh("cube", patches, [1] * 6)


def plates(n_sub: int = 16, size: float = 1.0, gap: float = 0.5):
    """Two coaxial size x size plates ``gap`` apart, facing each other, open system.

    Bottom plate z=0 (normal +z) then top plate z=gap (normal -z); each split into
    n_sub x n_sub square sub-faces (one face per quad): 2*n_sub^2 faces.
    """
    patches = [
        ((0, 0, 0), (size, 0, 0), (0, size, 0), n_sub, n_sub),
        ((0, 0, gap), (0, size, 0), (size, 0, 0), n_sub, n_sub),
    ]
    return patch_mesh(f"plates{n_sub}", patches, None)


def perpendicular_squares(n_sub: int = 1):
    """Two unit squares sharing the edge x in [0,1], y=z=0, at 90 degrees, open system."""
    patches = [
        ((0, 0, 0), (1, 0, 0), (0, 1, 0), n_sub, n_sub),  # z = 0, normal +z
        ((0, 0, 0), (0, 0, 1), (1, 0, 0), n_sub, n_sub),  # y = 0, normal +y
    ]
    return patch_mesh("perp_squares", patches, [1, 1])


def discs(r1: float = 1.0, r2: float = 2.0, h: float = 1.0, segments: int = 256, back_gap: float = 1e-4):
    """Two coaxial discs (polygons of ``segments`` sides) facing each other, plus their back faces.

    Faces: 0 = disc 1 (z=0, normal +z), 1 = disc 2 (z=h, normal -z), 2 = back of disc 1
    (normal -z, ``back_gap`` below), 3 = back of disc 2 (normal +z, ``back_gap`` above).
    Each face is a triangle fan around the centre; open system.
    """
    ang = 2.0 * np.pi * np.arange(segments) / segments
    verts, tris, tri_face = [], [], []

    def fan(radius, z, up, face):
        base = len(verts)
        verts.append((0.0, 0.0, z))
        for a in ang:
            verts.append((radius * np.cos(a), radius * np.sin(a), z))
        for k in range(segments):
            a, b = base + 1 + k, base + 1 + (k + 1) % segments
            tris.append((base, a, b) if up else (base, b, a))
            tri_face.append(face)

    fan(r1, 0.0, True, 0)
    fan(r2, h, False, 1)
    fan(r1, -back_gap, False, 2)
    fan(r2, h + back_gap, True, 3)
    return Mesh(name="discs", verts=np.array(verts, np.float32), tris=np.array(tris, np.int32),
                tri_face=np.array(tri_face, np.int32), n_faces=4,
                patch_of_face=np.arange(4, dtype=np.int32), n_patches=4)


def two_sided_plates(size: float = 1.0, gap: float = 1.0, back_gap: float = 1e-4):
    """Two coaxial size x size plates ``gap`` apart, each with its outer side as a face.

    Faces (the numbering of the thesis's parallel-plates model, 0-based): 0 = outer side
    of the bottom plate (z = -back_gap, normal -z), 1 = inner side of the bottom plate
    (z = 0, normal +z), 2 = inner side of the top plate (z = gap, normal -z), 3 = outer
    side of the top plate (z = gap + back_gap, normal +z). Two triangles each; open system.
    """
    patches = [
        ((0, 0, -back_gap), (0, size, 0), (size, 0, 0), 1, 1),
        ((0, 0, 0), (size, 0, 0), (0, size, 0), 1, 1),
        ((0, 0, gap), (0, size, 0), (size, 0, 0), 1, 1),
        ((0, 0, gap + back_gap), (size, 0, 0), (0, size, 0), 1, 1),
    ]
    return patch_mesh("two_sided_plates", patches, [1] * 4)


def _grouped(name, patches, n_faces):
    quads = [nu * nv for (_, _, _, nu, nv) in patches]
    return patch_mesh(name, patches, _split_counts(n_faces, quads))


def small_sat(quad: float = 0.0125, n_faces: int = 2048):
    """Small-satellite-shaped mesh: 0.3x0.3x0.6 m body and four 0.3x0.6 m panels.

    Body x,y in [-0.15, 0.15], z in [0, 0.6], outward faces. Each panel is hinged on
    one top edge of the body and opened 45 degrees outward; its front side faces the
    body. 1.25 cm quads give 10,368 quads (20,736 triangles), grouped into
    ``n_faces`` planar faces (faces per patch proportional to its quads).
    """
    a, h, L = 0.15, 0.6, 0.6
    n3, n6 = int(round(0.3 / quad)), int(round(0.6 / quad))
    c = s = np.sqrt(0.5)
    patches = [
        ((-a, -a, 0), (0, 2 * a, 0), (2 * a, 0, 0), n3, n3),        # bottom, -z
        ((-a, -a, h), (2 * a, 0, 0), (0, 2 * a, 0), n3, n3),        # top, +z
        ((a, -a, 0), (0, 2 * a, 0), (0, 0, h), n3, n6),             # +x
        ((-a, -a, 0), (0, 0, h), (0, 2 * a, 0), n3, n6),            # -x
        ((-a, a, 0), (0, 0, h), (2 * a, 0, 0), n6, n3),             # +y
        ((-a, -a, 0), (2 * a, 0, 0), (0, 0, h), n3, n6),            # -y
    ]
    # panels: hinge along a top edge, panel direction (outward*sin45, -cos45);
    # the front normal U x V points back toward the body
    patches += [
        ((a, -a, h), (0, 2 * a, 0), (s * L, 0, -c * L), n3, n6),     # +x panel
        ((-a, -a, h), (-s * L, 0, -c * L), (0, 2 * a, 0), n6, n3),   # -x panel
        ((-a, a, h), (0, s * L, -c * L), (2 * a, 0, 0), n6, n3),     # +y panel
        ((-a, -a, h), (2 * a, 0, 0), (0, -s * L, -c * L), n3, n6),   # -y panel
    ]
    return _grouped("small_sat", patches, n_faces)


def spacecraft(n_faces: int = 10240, quad: float = 0.013, boom_sides: int = 32, seed: int = 7):
    """Procedural spacecraft: body box, 6 solar panels, 2 radiators and a cylindrical boom.

    Body 1.0 x 1.0 x 1.5 m (x,y in [-0.5,0.5], z in [0,1.5]); two wings of three
    1.0 x 1.0 m panels along +-y, tilted by a seeded angle about y; two 1.0 x 0.8 m
    radiators standing off the +-x faces; a boom (``boom_sides``-gon prism, radius
    0.05 m, 2 m long) hanging from the bottom face. About 200k triangles grouped
    into ``n_faces`` planar faces.
    """
    rng = np.random.default_rng(seed)
    q = quad
    n = lambda length: max(1, int(round(length / q)))  # noqa: E731
    patches = []
    bx, bz = 0.5, 1.5
    patches += [
        ((-bx, -bx, 0), (0, 2 * bx, 0), (2 * bx, 0, 0), n(1.0), n(1.0)),      # bottom -z
        ((-bx, -bx, bz), (2 * bx, 0, 0), (0, 2 * bx, 0), n(1.0), n(1.0)),     # top +z
        ((bx, -bx, 0), (0, 2 * bx, 0), (0, 0, bz), n(1.0), n(1.5)),           # +x
        ((-bx, -bx, 0), (0, 0, bz), (0, 2 * bx, 0), n(1.5), n(1.0)),          # -x
        ((-bx, bx, 0), (0, 0, bz), (2 * bx, 0, 0), n(1.5), n(1.0)),           # +y
        ((-bx, -bx, 0), (2 * bx, 0, 0), (0, 0, bz), n(1.0), n(1.5)),          # -y
    ]
    # wings: panels k = 0..2 along +y and -y, tilted about the y axis, front facing -z side
    for sign in (+1, -1):
        for k in range(3):
            tilt = np.deg2rad(10.0 + 20.0 * rng.random())
            y0 = sign * (bx + 0.1 + 1.05 * k)
            U = np.array([np.cos(tilt), 0.0, np.sin(tilt)])
            P = np.array([-0.5 * np.cos(tilt), y0, 0.75 - 0.5 * np.sin(tilt)])
            V = np.array([0.0, sign * 1.0, 0.0])
            if sign > 0:
                patches.append((P, V, U, n(1.0), n(1.0)))
            else:
                patches.append((P, U, V, n(1.0), n(1.0)))
    # radiators: 1.0 (y) x 0.8 (x) plates standing 0.2 m off the +-x faces, facing the body
    for sign in (+1, -1):
        x0 = sign * (bx + 0.2)
        P = np.array([x0, -0.5, 0.35])
        if sign > 0:
            patches.append((P, (0, 0, 0.8), (0, 1.0, 0), n(0.8), n(1.0)))  # normal -x
        else:
            patches.append((P, (0, 1.0, 0), (0, 0, 0.8), n(1.0), n(0.8)))  # normal +x
    # boom: prism of boom_sides facets, radius r, from z=0 down to z=-2, outward facets
    r, Lb = 0.05, 2.0
    for k in range(boom_sides):
        a0 = 2 * np.pi * k / boom_sides
        a1 = 2 * np.pi * (k + 1) / boom_sides
        p0 = np.array([r * np.cos(a0), r * np.sin(a0), -Lb])
        p1 = np.array([r * np.cos(a1), r * np.sin(a1), -Lb])
        patches.append((p0, p1 - p0, (0, 0, Lb), 1, n(Lb) * 2))
    return _grouped("spacecraft", patches, n_faces)
