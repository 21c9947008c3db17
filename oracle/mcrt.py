"""MCRT oracle: ctypes front end of ``mcrt.c`` (Sec. 3.5.1, Eq. 3.15).

TEST INFRASTRUCTURE ONLY (see the package docstring). ``build()`` compiles
``mcrt.c`` with gcc into ``oracle/_build/liboracle_mcrt.so``.
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "mcrt.c")
_OUT_DIR = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_OUT_DIR, "liboracle_mcrt.so")
_lib = None


def build(force: bool = False) -> str:
    """Compile the C oracle (no FMA contraction, no fast-math)."""
    os.makedirs(_OUT_DIR, exist_ok=True)
    if force or not os.path.exists(_LIB_PATH) or os.path.getmtime(_LIB_PATH) < os.path.getmtime(_SRC):
        tmp = _LIB_PATH + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-ffp-contract=off", "-fno-fast-math", "-fopenmp",
                               "-fPIC", "-shared", "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _load():
    global _lib
    if _lib is None:
        lib = ctypes.CDLL(build())
        P = ctypes.c_void_p
        i64, i32, u64 = ctypes.c_int64, ctypes.c_int32, ctypes.c_uint64
        lib.oracle_philox4x32_10.argtypes = [P, P, P]
        lib.oracle_philox4x32_10.restype = None
        lib.oracle_face_geometry.argtypes = [P, i64, P, i64, P, i32, P, P, P, P]
        lib.oracle_sample_rays.argtypes = [P, i64, P, i64, P, i32, i32, u64, u64, i64, P, P, P, P]
        lib.oracle_closest_hits.argtypes = [P, i64, P, i64, P, i32, P, P, P, i64, P, P]
        lib.oracle_trace_counts.argtypes = [P, i64, P, i64, P, i32, P, u64, u64, ctypes.c_int,
                                            ctypes.c_int, P, i32, P]
        lib.oracle_trace_reflect.argtypes = [P, i64, P, i64, P, i32, P, P, P, i32, u64, u64, ctypes.c_int,
                                             ctypes.c_int, P, i32, P, P]
        lib.oracle_sample_rays_side.argtypes = [P, i64, P, i64, P, i32, i32, i32, u64, u64, i64, P, P, P]
        lib.oracle_trace_sided.argtypes = [P, i64, P, i64, P, i32, P, u64, u64, ctypes.c_int, ctypes.c_int, P,
                                           i32, P]
        lib.oracle_max_threads.argtypes = []
        lib.oracle_unit_circle.argtypes = [ctypes.c_uint32, i64, P, P]
        for fn in ("oracle_face_geometry", "oracle_sample_rays", "oracle_closest_hits",
                   "oracle_trace_counts", "oracle_trace_reflect", "oracle_sample_rays_side",
                   "oracle_trace_sided", "oracle_max_threads", "oracle_unit_circle"):
            getattr(lib, fn).restype = ctypes.c_int
        _lib = lib
    return _lib


def _ptr(a):
    return a.ctypes.data_as(ctypes.c_void_p) if a is not None else None


def _mesh_arrays(verts, tris, tri_face):
    v = np.ascontiguousarray(verts, dtype=np.float32)
    t = np.ascontiguousarray(tris, dtype=np.int32)
    f = np.ascontiguousarray(tri_face, dtype=np.int32)
    return v, t, f


def _check(st, what):
    if st != 0:
        raise ValueError(f"oracle {what} failed with status {st}")


def philox4x32_10(counter, key):
    """One Philox4x32-10 block (Salmon et al. 2011) -> 4 uint32."""
    lib = _load()
    c = np.ascontiguousarray(counter, dtype=np.uint32)
    k = np.ascontiguousarray(key, dtype=np.uint32)
    out = np.zeros(4, dtype=np.uint32)
    lib.oracle_philox4x32_10(_ptr(c), _ptr(k), _ptr(out))
    return out


def unit_circle(t0, n):
    """cos and sin (float32) of 2 pi t 2^-24, t = t0 .. t0+n-1, as the ray sampling forms them."""
    lib = _load()
    c = np.zeros(n, np.float32)
    s = np.zeros(n, np.float32)
    _check(lib.oracle_unit_circle(ctypes.c_uint32(t0), ctypes.c_int64(n), _ptr(c), _ptr(s)), "unit_circle")
    return c, s


def face_geometry(verts, tris, tri_face, n_faces):
    """Face areas (fp64), frames (t, b, n as float32[N,3,3]), triangle CDF thresholds, origin lift."""
    lib = _load()
    v, t, f = _mesh_arrays(verts, tris, tri_face)
    area = np.zeros(n_faces, dtype=np.float64)
    frame = np.zeros((n_faces, 3, 3), dtype=np.float32)
    thr = np.zeros(len(t), dtype=np.uint32)
    tmin = np.zeros(1, dtype=np.float32)
    _check(lib.oracle_face_geometry(_ptr(v), len(v), _ptr(t), len(t), _ptr(f), n_faces,
                                    _ptr(area), _ptr(frame), _ptr(thr), _ptr(tmin)), "face_geometry")
    return area, frame, thr, float(tmin[0])


def face_areas(verts, tris, tri_face, n_faces):
    return face_geometry(verts, tris, tri_face, n_faces)[0]


def sample_rays(verts, tris, tri_face, n_faces, face, seed, ray0, n):
    """Origins, directions, source triangles and extra direction draws (always 0: the
    direction comes from the ray's one draw) of rays [ray0, ray0+n) of ``face``."""
    lib = _load()
    v, t, f = _mesh_arrays(verts, tris, tri_face)
    o = np.zeros((n, 3), np.float32)
    d = np.zeros((n, 3), np.float32)
    tri = np.zeros(n, np.int32)
    att = np.zeros(n, np.int32)
    _check(lib.oracle_sample_rays(_ptr(v), len(v), _ptr(t), len(t), _ptr(f), n_faces, face, seed,
                                  ray0, n, _ptr(o), _ptr(d), _ptr(tri), _ptr(att)), "sample_rays")
    return o, d, tri, att


def closest_hits(verts, tris, tri_face, n_faces, origins, dirs, src_tri=None):
    """Brute-force closest hit (triangle index or -1, t) for arbitrary rays."""
    lib = _load()
    v, t, f = _mesh_arrays(verts, tris, tri_face)
    o = np.ascontiguousarray(origins, np.float32)
    d = np.ascontiguousarray(dirs, np.float32)
    s = None if src_tri is None else np.ascontiguousarray(src_tri, np.int32)
    n = len(o)
    hit = np.zeros(n, np.int32)
    tt = np.zeros(n, np.float32)
    _check(lib.oracle_closest_hits(_ptr(v), len(v), _ptr(t), len(t), _ptr(f), n_faces, _ptr(o),
                                   _ptr(d), _ptr(s), n, _ptr(hit), _ptr(tt)), "closest_hits")
    return hit, tt


def trace_counts(verts, tris, tri_face, n_faces, rays_per_face, seed, ray_offset=0,
                 use_bvh=True, threads=0, faces=None):
    """Hit counts N_ij, int64[N, N+1] (column N = environment), Eq. 3.15 numerators.

    ``faces`` restricts the work to a subset of source rows (the other rows stay 0);
    rows are independent because every ray is addressed by (seed, ray, face).
    """
    lib = _load()
    v, t, f = _mesh_arrays(verts, tris, tri_face)
    rays = np.ascontiguousarray(rays_per_face, dtype=np.int64)
    if rays.shape != (n_faces,):
        raise ValueError("rays_per_face must have one entry per face")
    counts = np.zeros((n_faces, n_faces + 1), dtype=np.int64)
    sub = None if faces is None else np.ascontiguousarray(faces, dtype=np.int32)
    _check(lib.oracle_trace_counts(_ptr(v), len(v), _ptr(t), len(t), _ptr(f), n_faces, _ptr(rays),
                                   seed, ray_offset, int(bool(use_bvh)), int(threads), _ptr(sub),
                                   0 if sub is None else len(sub), _ptr(counts)), "trace_counts")
    return counts


def trace_reflect(verts, tris, tri_face, n_faces, rays_per_face, eps, rho, seed, ray_offset=0, max_bounces=4096,
                  use_bvh=True, threads=0, faces=None):
    """Direct Monte Carlo of Gebhart factors with diffuse reflections (Eq. 4.5 as a random
    walk): counts int64[N, N+1] of rays of face i absorbed on face j (column N: escaped)
    and stats {rays, hits, lost, overflow}. B_ij is estimated by counts_ij / N_i."""
    lib = _load()
    v, t, f = _mesh_arrays(verts, tris, tri_face)
    rays = np.ascontiguousarray(rays_per_face, dtype=np.int64)
    e = np.ascontiguousarray(eps, dtype=np.float64)
    r = np.ascontiguousarray(rho, dtype=np.float64)
    if rays.shape != (n_faces,) or e.shape != (n_faces,) or r.shape != (n_faces,):
        raise ValueError("rays_per_face, eps and rho must have one entry per face")
    counts = np.zeros((n_faces, n_faces + 1), dtype=np.int64)
    stats = np.zeros(4, dtype=np.int64)
    sub = None if faces is None else np.ascontiguousarray(faces, dtype=np.int32)
    _check(lib.oracle_trace_reflect(_ptr(v), len(v), _ptr(t), len(t), _ptr(f), n_faces, _ptr(rays), _ptr(e),
                                    _ptr(r), int(max_bounces), seed, ray_offset, int(bool(use_bvh)), int(threads),
                                    _ptr(sub), 0 if sub is None else len(sub), _ptr(counts), _ptr(stats)),
           "trace_reflect")
    return counts, {"rays": int(stats[0]), "hits": int(stats[1]), "lost": int(stats[2]),
                    "overflow": int(stats[3])}


def sample_rays_side(verts, tris, tri_face, n_faces, face, side, seed, ray0, n):
    """Origins, directions and source triangles of rays [ray0, ray0+n) of side ``side``
    (0 = A, along the face normal; 1 = B) of ``face``."""
    lib = _load()
    v, t, f = _mesh_arrays(verts, tris, tri_face)
    o = np.zeros((n, 3), np.float32)
    d = np.zeros((n, 3), np.float32)
    tri = np.zeros(n, np.int32)
    _check(lib.oracle_sample_rays_side(_ptr(v), len(v), _ptr(t), len(t), _ptr(f), n_faces, face, side, seed,
                                       ray0, n, _ptr(o), _ptr(d), _ptr(tri)), "sample_rays_side")
    return o, d, tri


def trace_sided(verts, tris, tri_face, n_faces, rays_per_side, seed, ray_offset=0, use_bvh=True, threads=0,
                rows=None):
    """Side-resolved hit counts int64[2N, 2N+1] (Sec. 5.2.4-5.2.5): row 2f+X counts the rays
    emitted from side X of face f, column 2g+Y the rays whose closest hit lies on side Y
    of face g, column 2N the environment. ``rays_per_side[2f+X]`` rays leave side X of f;
    ``rows`` restricts the work to a subset of rows."""
    lib = _load()
    v, t, f = _mesh_arrays(verts, tris, tri_face)
    rays = np.ascontiguousarray(rays_per_side, dtype=np.int64)
    if rays.shape != (2 * n_faces,):
        raise ValueError("rays_per_side must have two entries per face")
    counts = np.zeros((2 * n_faces, 2 * n_faces + 1), dtype=np.int64)
    sub = None if rows is None else np.ascontiguousarray(rows, dtype=np.int32)
    _check(lib.oracle_trace_sided(_ptr(v), len(v), _ptr(t), len(t), _ptr(f), n_faces, _ptr(rays), seed,
                                  ray_offset, int(bool(use_bvh)), int(threads), _ptr(sub),
                                  0 if sub is None else len(sub), _ptr(counts)), "trace_sided")
    return counts


def max_threads() -> int:
    return int(_load().oracle_max_threads())


def view_factors(counts, rays_per_face):
    """F_ij = N_ij / N_i (Eq. 3.15), fp64."""
    c = np.asarray(counts, dtype=np.float64)
    n = np.asarray(rays_per_face, dtype=np.float64)
    return c / n[:, None]
