"""Python front end of libradgeb: the C calls of include/radgeb.h with torch tensors.

Argument marshalling only: every step runs in the library's CUDA kernels. Device
buffers are torch tensors on the context's device (torch is used for memory and
streams); host-side arguments are numpy arrays or Python numbers. Every call is
enqueued on ``stream`` (default: torch's current stream).
"""
from __future__ import annotations

import ctypes

import numpy as np
import torch

from . import _native
from ._native import RadgebError


def _stream(stream):
    if stream is None:
        stream = torch.cuda.current_stream()
    return ctypes.c_void_p(stream.cuda_stream)


def _dptr(t: torch.Tensor, dtype, name, numel=None, device=None):
    if not isinstance(t, torch.Tensor) or not t.is_cuda:
        raise TypeError(f"{name} must be a CUDA tensor")
    if t.dtype != dtype:
        raise TypeError(f"{name} must be {dtype}, got {t.dtype}")
    if not t.is_contiguous():
        raise ValueError(f"{name} must be contiguous")
    if numel is not None and t.numel() != numel:
        raise ValueError(f"{name} must have {numel} elements, got {t.numel()}")
    if device is not None and t.device.index != device:
        raise ValueError(f"{name} is on cuda:{t.device.index}, the context on cuda:{device}")
    return ctypes.c_void_p(t.data_ptr())


def _hptr(a: np.ndarray):
    return a.ctypes.data_as(ctypes.c_void_p)


def _ws(ws, device=None):
    """(pointer, bytes) of an optional caller-owned workspace (a CUDA tensor), or (NULL, 0)."""
    if ws is None:
        return ctypes.c_void_p(None), ctypes.c_size_t(0)
    if not isinstance(ws, torch.Tensor) or not ws.is_cuda or not ws.is_contiguous():
        raise TypeError("ws must be a contiguous CUDA tensor")
    if device is not None and ws.device.index != device:
        raise ValueError(f"ws is on cuda:{ws.device.index}, the context on cuda:{device}")
    return ctypes.c_void_p(ws.data_ptr()), ctypes.c_size_t(ws.numel() * ws.element_size())


class Context:
    """A library context bound to one CUDA device (rg_create / rg_destroy)."""

    def __init__(self, device: int = 0):
        self.lib = _native.load()
        self.device = int(device)
        h = ctypes.c_void_p()
        st = self.lib.rg_create(ctypes.byref(h), self.device)
        if st != 0:
            raise RadgebError(st, f"rg_create(device={device}) failed")
        self.handle = h

    def check(self, st: int, what: str):
        if st != 0:
            msg = self.lib.rg_last_error(self.handle)
            raise RadgebError(st, f"{what}: {msg.decode() if msg else ''}")

    def close(self):
        if getattr(self, "handle", None):
            self.lib.rg_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()


class Mesh:
    """A mesh uploaded with its BVH: built on the host (rg_mesh_create) or, with
    ``gpu_bvh``, on the device (rg_mesh_create_gpu_bvh; the same tree)."""

    def __init__(self, ctx: Context, verts, tris, tri_face, n_faces: int, use_bvh: int = -1,
                 gpu_bvh: bool = False):
        self.ctx = ctx
        v = np.ascontiguousarray(verts, np.float32)
        t = np.ascontiguousarray(tris, np.int32)
        f = np.ascontiguousarray(tri_face, np.int32)
        h = ctypes.c_void_p()
        if not gpu_bvh:
            ctx.check(ctx.lib.rg_mesh_create(ctx.handle, _hptr(v), len(v), _hptr(t), len(t), _hptr(f), int(n_faces),
                                             int(use_bvh), ctypes.byref(h)), "rg_mesh_create")
        else:
            ctx.check(ctx.lib.rg_mesh_create_gpu_bvh(ctx.handle, _hptr(v), len(v), _hptr(t), len(t), _hptr(f),
                                                     int(n_faces), int(use_bvh), ctypes.byref(h)),
                      "rg_mesh_create_gpu_bvh")
        self.handle = h
        self.n_faces = int(n_faces)
        self.n_tris = len(t)

    @classmethod
    def from_synth(cls, ctx, m, use_bvh=-1, gpu_bvh=False):
        return cls(ctx, m.verts, m.tris, m.tri_face, m.n_faces, use_bvh, gpu_bvh)

    def bvh(self):
        """(nodes float32 [bvh_nodes, 16] in the traversal layout, triangle of every
        traversal-order record int32 [n_tris]) (rg_mesh_get_bvh)."""
        n = self.info()["bvh_nodes"]
        nodes = np.zeros((n, 16), np.float32)
        rec = np.zeros(self.n_tris, np.int32)
        self.ctx.check(self.ctx.lib.rg_mesh_get_bvh(self.handle, _hptr(nodes) if n else None, _hptr(rec)),
                       "rg_mesh_get_bvh")
        return nodes, rec

    def info(self) -> dict:
        mi = _native.MeshInfo()
        self.ctx.check(self.ctx.lib.rg_mesh_get_info(self.handle, ctypes.byref(mi)), "rg_mesh_get_info")
        return {k: getattr(mi, k) for k, _ in mi._fields_}

    def face_areas(self) -> np.ndarray:
        out = np.zeros(self.n_faces, np.float64)
        self.ctx.check(self.ctx.lib.rg_face_areas(self.handle, _hptr(out)), "rg_face_areas")
        return out

    def close(self):
        if getattr(self, "handle", None):
            self.ctx.lib.rg_mesh_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def trace(ctx: Context, mesh: Mesh, rays_per_face, seed: int, ray_offset: int = 0, fma_free: bool = True,
          counts: torch.Tensor | None = None, stream=None) -> torch.Tensor:
    """MCRT hit counts N_ij, int64 [N, N+1] on the device (rg_trace); accumulates into ``counts``."""
    N = mesh.n_faces
    rays = np.ascontiguousarray(rays_per_face, np.int64)
    if rays.shape != (N,):
        raise ValueError("rays_per_face must have one entry per face")
    if counts is None:
        counts = torch.zeros((N, N + 1), dtype=torch.int64, device=f"cuda:{ctx.device}")
    ctx.check(ctx.lib.rg_trace(ctx.handle, mesh.handle, _hptr(rays), int(seed) & (2 ** 64 - 1), int(ray_offset),
                               int(bool(fma_free)), _dptr(counts, torch.int64, "counts", N * (N + 1), ctx.device),
                               _stream(stream)), "rg_trace")
    return counts


def trace_stats(ctx: Context, mesh: Mesh, rays_per_face, seed: int, ray_offset: int = 0, fma_free: bool = True,
                counts: torch.Tensor | None = None, stream=None):
    """rg_trace_stats: (counts, {"rays", "box_tests", "tri_tests"})."""
    N = mesh.n_faces
    rays = np.ascontiguousarray(rays_per_face, np.int64)
    if counts is None:
        counts = torch.zeros((N, N + 1), dtype=torch.int64, device=f"cuda:{ctx.device}")
    st = np.zeros(3, np.uint64)
    ctx.check(ctx.lib.rg_trace_stats(ctx.handle, mesh.handle, _hptr(rays), int(seed) & (2 ** 64 - 1),
                                     int(ray_offset), int(bool(fma_free)),
                                     _dptr(counts, torch.int64, "counts", N * (N + 1), ctx.device), _hptr(st),
                                     _stream(stream)), "rg_trace_stats")
    return counts, {"rays": int(st[0]), "box_tests": int(st[1]), "tri_tests": int(st[2])}


def trace_sided(ctx: Context, mesh: Mesh, rays_per_side, seed: int, ray_offset: int = 0, fma_free: bool = True,
                counts: torch.Tensor | None = None, stream=None) -> torch.Tensor:
    """Side-resolved MCRT hit counts, int64 [2N, 2N+1] on the device (rg_trace_sided): row
    2f+X = side X of face f (0 = A, the side its normal points to; 1 = B), column 2g+Y,
    column 2N = environment; accumulates into ``counts``."""
    N = mesh.n_faces
    rays = np.ascontiguousarray(rays_per_side, np.int64)
    if rays.shape != (2 * N,):
        raise ValueError("rays_per_side must have two entries per face")
    if counts is None:
        counts = torch.zeros((2 * N, 2 * N + 1), dtype=torch.int64, device=f"cuda:{ctx.device}")
    ctx.check(ctx.lib.rg_trace_sided(ctx.handle, mesh.handle, _hptr(rays), int(seed) & (2 ** 64 - 1),
                                     int(ray_offset), int(bool(fma_free)),
                                     _dptr(counts, torch.int64, "counts", 2 * N * (2 * N + 1), ctx.device),
                                     _stream(stream)), "rg_trace_sided")
    return counts


def trace_reflect(ctx: Context, mesh: Mesh, rays_per_face, eps, rho, seed: int, max_bounces: int = 4096,
                  ray_offset: int = 0, fma_free: bool = True, counts: torch.Tensor | None = None, stream=None):
    """REFs directly from MCRT with diffuse reflections (rg_trace_reflect): (counts int64
    [N, N+1] of rays absorbed per face, {"rays", "hits", "lost", "overflow"}).
    ``eps`` and ``rho`` are per-face host arrays."""
    N = mesh.n_faces
    rays = np.ascontiguousarray(rays_per_face, np.int64)
    e = np.ascontiguousarray(eps, np.float64)
    r = np.ascontiguousarray(rho, np.float64)
    if rays.shape != (N,) or e.shape != (N,) or r.shape != (N,):
        raise ValueError("rays_per_face, eps and rho must have one entry per face")
    if counts is None:
        counts = torch.zeros((N, N + 1), dtype=torch.int64, device=f"cuda:{ctx.device}")
    st = np.zeros(4, np.uint64)
    ctx.check(ctx.lib.rg_trace_reflect(ctx.handle, mesh.handle, _hptr(rays), _hptr(e), _hptr(r), int(max_bounces),
                                       int(seed) & (2 ** 64 - 1), int(ray_offset), int(bool(fma_free)),
                                       _dptr(counts, torch.int64, "counts", N * (N + 1), ctx.device), _hptr(st),
                                       _stream(stream)), "rg_trace_reflect")
    return counts, {"rays": int(st[0]), "hits": int(st[1]), "lost": int(st[2]), "overflow": int(st[3])}


def launch_count(ctx: Context) -> int:
    """Kernels the context has launched so far (rg_launch_count)."""
    n = ctypes.c_int64(0)
    ctx.check(ctx.lib.rg_launch_count(ctx.handle, ctypes.byref(n)), "rg_launch_count")
    return n.value


KERNEL_CLASSES = {"trace": 0, "residual_gemm": 1, "gemm": 2, "enforce": 3, "factor": 4}


def workspace_bytes(ctx: Context) -> int:
    """Device workspace the context holds (rg_workspace_bytes)."""
    n = ctypes.c_size_t(0)
    ctx.check(ctx.lib.rg_workspace_bytes(ctx.handle, ctypes.byref(n)), "rg_workspace_bytes")
    return n.value


def solver_workspace(kind: str, n: int, rank: int = 0) -> int:
    """Bytes of caller-owned workspace a dense-solve call of n faces needs (rg_solver_workspace);
    kind one of gebhart, gebhart_adjoint, gebhart_adjoint_factored, temperatures,
    temperatures_sets, enforce_lsq."""
    out = ctypes.c_size_t(0)
    st = _native.load().rg_solver_workspace(_native.WS_KIND[kind], int(n), int(rank), ctypes.byref(out))
    if st != 0:
        raise RadgebError(st, f"rg_solver_workspace({kind}, {n}, {rank})")
    return out.value


def gebhart_workspace(n: int, n_sets: int = 1, precision="bf16", keep_factors: bool = False) -> int:
    """Bytes of caller-owned workspace rg_gebhart needs, or with keep_factors the bytes of the
    factor store it fills for the adjoints (rg_gebhart_workspace)."""
    out = ctypes.c_size_t(0)
    st = _native.load().rg_gebhart_workspace(int(n), int(n_sets), _prec(precision), int(bool(keep_factors)),
                                             ctypes.byref(out))
    if st != 0:
        raise RadgebError(st, f"rg_gebhart_workspace({n}, {n_sets})")
    return out.value


def gebhart_factor_store(n: int, n_sets: int, precision="bf16", device=0) -> torch.Tensor:
    """A device buffer (uint8) for the factors rg_gebhart keeps for the REF adjoints."""
    nbytes = gebhart_workspace(n, n_sets, precision, keep_factors=True)
    return torch.empty(nbytes, dtype=torch.uint8, device=torch.device("cuda", int(device)))


def kernel_timer(ctx: Context, enable: bool):
    """Start (clearing earlier records) or stop the context's kernel timer (rg_kernel_timer)."""
    ctx.check(ctx.lib.rg_kernel_timer(ctx.handle, int(bool(enable))), "rg_kernel_timer")


def kernel_timer_read(ctx: Context, kind: str) -> dict:
    """Launches, summed CUDA-event duration (ms), executed tensor-core flops and algorithmic
    flops of the timed launches of one kernel class since the timer was started
    (rg_kernel_timer_read)."""
    n = ctypes.c_int64(0)
    ms = ctypes.c_double(0.0)
    fl = ctypes.c_double(0.0)
    alg = ctypes.c_double(0.0)
    ctx.check(ctx.lib.rg_kernel_timer_read(ctx.handle, KERNEL_CLASSES[kind], ctypes.byref(n), ctypes.byref(ms),
                                           ctypes.byref(fl), ctypes.byref(alg)), "rg_kernel_timer_read")
    return {"launches": n.value, "ms": ms.value, "flops": fl.value, "alg_flops": alg.value}


def counts_to_F(ctx: Context, counts: torch.Tensor, rays: torch.Tensor, F: torch.Tensor | None = None,
                stream=None) -> torch.Tensor:
    """F_ij = N_ij / N_i (rg_counts_to_F)."""
    n = counts.shape[0]
    if F is None:
        F = torch.empty((n, n + 1), dtype=torch.float64, device=counts.device)
    ctx.check(ctx.lib.rg_counts_to_F(ctx.handle, n, _dptr(counts, torch.int64, "counts", n * (n + 1), ctx.device),
                                     _dptr(rays, torch.int64, "rays", n, ctx.device),
                                     _dptr(F, torch.float64, "F", n * (n + 1), ctx.device), _stream(stream)),
              "rg_counts_to_F")
    return F


def enforce_iterative(ctx: Context, F: torch.Tensor, omega: torch.Tensor, tol: float = 1e-12, maxit: int = 10000,
                      stream=None) -> int:
    """In-place iterative closure + reciprocity enforcer (rg_enforce_iterative); returns iterations."""
    n = F.shape[0]
    it = ctypes.c_int32(0)
    ctx.check(ctx.lib.rg_enforce_iterative(ctx.handle, n, _dptr(omega, torch.float64, "omega", n, ctx.device),
                                           _dptr(F, torch.float64, "F", n * (n + 1), ctx.device), float(tol),
                                           int(maxit), ctypes.byref(it), _stream(stream)), "rg_enforce_iterative")
    return it.value


def kappa(ctx: Context, rays: torch.Tensor, omega: torch.Tensor, mode="fractional_variance", F=None,
          param: float | None = None, K: torch.Tensor | None = None, stream=None) -> torch.Tensor:
    """Reciprocity weights kappa [N, N] (rg_kappa): "triangulation" (param = exponent,
    default 0.4) or "fractional_variance" (needs the MCRT F; param = z, default 1.96)."""
    n = omega.numel()
    m = _native.KAPPA[mode] if isinstance(mode, str) else int(mode)
    if param is None:
        param = 0.4 if m == _native.KAPPA["triangulation"] else 1.96
    if K is None:
        K = torch.empty((n, n), dtype=torch.float64, device=omega.device)
    Fp = ctypes.c_void_p(None) if F is None else _dptr(F, torch.float64, "F", n * (n + 1), ctx.device)
    ctx.check(ctx.lib.rg_kappa(ctx.handle, n, m, Fp, _dptr(rays, torch.int64, "rays", n, ctx.device),
                               _dptr(omega, torch.float64, "omega", n, ctx.device), float(param),
                               _dptr(K, torch.float64, "kappa", n * n, ctx.device), _stream(stream)), "rg_kappa")
    return K


def enforce_iterative_kappa(ctx: Context, F: torch.Tensor, omega: torch.Tensor, K: torch.Tensor, tol: float = 1e-12,
                            maxit: int = 10000, stream=None) -> int:
    """In-place iterative enforcer with per-pair reciprocity weights (rg_enforce_iterative_kappa)."""
    n = F.shape[0]
    it = ctypes.c_int32(0)
    ctx.check(ctx.lib.rg_enforce_iterative_kappa(ctx.handle, n, _dptr(omega, torch.float64, "omega", n, ctx.device),
                                                 _dptr(K, torch.float64, "kappa", n * n, ctx.device),
                                                 _dptr(F, torch.float64, "F", n * (n + 1), ctx.device), float(tol),
                                                 int(maxit), ctypes.byref(it), _stream(stream)),
              "rg_enforce_iterative_kappa")
    return it.value


def enforce_lsq(ctx: Context, F: torch.Tensor, omega: torch.Tensor, nnr: bool = True, spva: bool = True,
                max_passes: int = 1000, stream=None, ws=None) -> int:
    """In-place least-squares optimum with NNR / SPVA (rg_enforce_lsq); returns projections."""
    n = F.shape[0]
    p = ctypes.c_int32(0)
    ctx.check(ctx.lib.rg_enforce_lsq(ctx.handle, n, _dptr(omega, torch.float64, "omega", n, ctx.device),
                                     _dptr(F, torch.float64, "F", n * (n + 1), ctx.device), int(bool(nnr)),
                                     int(bool(spva)), int(max_passes), ctypes.byref(p), *_ws(ws, ctx.device), _stream(stream)),
              "rg_enforce_lsq")
    return p.value


def aggregate(ctx: Context, F_sub: torch.Tensor, sub_area: torch.Tensor, sub_group: torch.Tensor, n_group: int,
              stream=None):
    """Group view factors (rg_aggregate) -> (F_group [G, G+1], group areas [G])."""
    n = F_sub.shape[0]
    Fg = torch.empty((n_group, n_group + 1), dtype=torch.float64, device=F_sub.device)
    Sg = torch.empty(n_group, dtype=torch.float64, device=F_sub.device)
    ctx.check(ctx.lib.rg_aggregate(ctx.handle, n, _dptr(F_sub, torch.float64, "F_sub", n * (n + 1), ctx.device),
                                   _dptr(sub_area, torch.float64, "sub_area", n, ctx.device),
                                   _dptr(sub_group, torch.int32, "sub_group", n, ctx.device), int(n_group),
                                   _dptr(Fg, torch.float64, "F_group"), _dptr(Sg, torch.float64, "group_area"),
                                   _stream(stream)), "rg_aggregate")
    return Fg, Sg


def aggregate_sided(ctx: Context, F2: torch.Tensor, sub_area: torch.Tensor, sub_group: torch.Tensor, n_group: int,
                    stream=None):
    """Side-resolved group view factors F^{X->Y}_nm and F^{X,inf}_n (Eq. 5.6-5.7, the first two
    lines of Eq. 5.28) from side-resolved sub-surface factors F2 [2n, 2n+1] (the layout of
    trace_sided) -> (F2_group [2G, 2G+1], group areas [G]).

    rg_aggregate with the sides as sub-surfaces: side X of sub-surface i (area S_i) joins
    side X of its group, so that sum_i S_i = S_n and the weights are S_i / S_n per side."""
    n = F2.shape[0] // 2
    g = sub_group.to(device=F2.device, dtype=torch.int32)
    sides = torch.stack([2 * g, 2 * g + 1], dim=1).reshape(-1).contiguous()
    area2 = sub_area.to(device=F2.device, dtype=torch.float64).repeat_interleave(2).contiguous()
    Fg, Sg = aggregate(ctx, F2, area2, sides, 2 * n_group, stream)
    return Fg, Sg[0::2].contiguous()


def node_view_factors(ctx: Context, F2: torch.Tensor, faces_per_node: torch.Tensor, fractions: bool = True,
                      stream=None):
    """Node view factors F [n, n+1] (Eq. 5.17) and, if asked, the view fractions f [2n, 2n+1]
    (Eq. 5.27 / 5.29) from side-resolved factors F2 [2n, 2n+1] (rg_node_view_factors)."""
    n = F2.shape[0] // 2
    Fn = torch.empty((n, n + 1), dtype=torch.float64, device=F2.device)
    fr = torch.empty_like(F2) if fractions else None
    ctx.check(ctx.lib.rg_node_view_factors(ctx.handle, n, _dptr(F2, torch.float64, "F2", 2 * n * (2 * n + 1),
                                                                 ctx.device),
                                           _dptr(faces_per_node, torch.int32, "faces_per_node", n, ctx.device),
                                           _dptr(Fn, torch.float64, "F_node"),
                                           None if fr is None else _dptr(fr, torch.float64, "frac"),
                                           _stream(stream)), "rg_node_view_factors")
    return Fn, fr


def node_couplings(ctx: Context, B2: torch.Tensor, eps2: torch.Tensor, face_area: torch.Tensor,
                   faces_per_node: torch.Tensor, stream=None):
    """Node couplings of two-faced nodes (App. C, rg_node_couplings) from side-resolved REFs
    B2 [2n, 2n+1]: (GR [n, n+1] (Eq. C.3, without sigma), node REFs B [n, n+1], node
    emissivities eps_ij [n, n+1] (Eq. C.4))."""
    n = B2.shape[0] // 2
    GR = torch.empty((n, n + 1), dtype=torch.float64, device=B2.device)
    Bn = torch.empty_like(GR)
    en = torch.empty_like(GR)
    ctx.check(ctx.lib.rg_node_couplings(ctx.handle, n, _dptr(B2, torch.float64, "B2", 2 * n * (2 * n + 1), ctx.device),
                                        _dptr(eps2, torch.float64, "eps2", 2 * n, ctx.device),
                                        _dptr(face_area, torch.float64, "face_area", n, ctx.device),
                                        _dptr(faces_per_node, torch.int32, "faces_per_node", n, ctx.device),
                                        _dptr(GR, torch.float64, "GR"), _dptr(Bn, torch.float64, "B_node"),
                                        _dptr(en, torch.float64, "eps_node"), _stream(stream)), "rg_node_couplings")
    return GR, Bn, en


def _prec(p):
    return _native.PREC[p] if isinstance(p, str) else int(p)


def gebhart(ctx: Context, F: torch.Tensor, eps: torch.Tensor, rho: torch.Tensor, precision="bf16",
            tol: float = 1e-12, max_sweeps: int = 12, B: torch.Tensor | None = None, stream=None, ws=None,
            factors=None, areas=None):
    """REFs of every (eps, rho) set (rg_gebhart) -> (B [S, N, N+1], sweeps, relative residual).
    factors: a store from gebhart_factor_store, filled for the adjoints (or None); areas: the
    face areas of a reciprocal F (the symmetric factorisation), or None."""
    n = F.shape[0]
    eps2 = eps.reshape(-1, n)
    S = eps2.shape[0]
    if B is None:
        B = torch.empty((S, n, n + 1), dtype=torch.float64, device=F.device)
    sw = ctypes.c_int32(0)
    res = ctypes.c_double(0.0)
    ctx.check(ctx.lib.rg_gebhart(ctx.handle, n, _dptr(F, torch.float64, "F", n * (n + 1), ctx.device), S,
                                 _dptr(eps2, torch.float64, "eps", S * n, ctx.device),
                                 _dptr(rho, torch.float64, "rho", S * n, ctx.device),
                                 ctypes.c_void_p(None) if areas is None else _dptr(areas, torch.float64, "areas", n,
                                                                                   ctx.device),
                                 _prec(precision), float(tol),
                                 int(max_sweeps), _dptr(B, torch.float64, "B", S * n * (n + 1), ctx.device),
                                 ctypes.byref(sw), ctypes.byref(res), *_ws(factors, ctx.device),
                                 *_ws(ws, ctx.device), _stream(stream)), "rg_gebhart")
    return B, sw.value, res.value


def gebhart_adjoint(ctx: Context, F, eps, rho, B, dB, precision="bf16", tol: float = 1e-12, max_sweeps: int = 12,
                    stream=None, ws=None, factors=None):
    """(dL/deps, dL/drho) [S, N] from dB = dL/dB (rg_gebhart_adjoint); factors: the store a
    gebhart call filled (or None: K^T is factorised afresh)."""
    n = F.shape[0]
    S = eps.numel() // n
    deps = torch.empty((S, n), dtype=torch.float64, device=F.device)
    drho = torch.empty((S, n), dtype=torch.float64, device=F.device)
    ctx.check(ctx.lib.rg_gebhart_adjoint(ctx.handle, n, _dptr(F, torch.float64, "F", n * (n + 1), ctx.device), S,
                                         _dptr(eps, torch.float64, "eps", S * n, ctx.device),
                                         _dptr(rho, torch.float64, "rho", S * n, ctx.device),
                                         _dptr(B, torch.float64, "B", S * n * (n + 1), ctx.device),
                                         _dptr(dB, torch.float64, "dB", S * n * (n + 1), ctx.device),
                                         _prec(precision), float(tol), int(max_sweeps),
                                         _dptr(deps, torch.float64, "deps"), _dptr(drho, torch.float64, "drho"),
                                         *_ws(factors, ctx.device), *_ws(ws, ctx.device), _stream(stream)),
              "rg_gebhart_adjoint")
    return deps, drho


def temperatures(ctx: Context, B, eps, area, Q, T_sink: float, sigma: float = 5.67e-8, precision="bf16",
                 tol: float = 1e-13, stream=None, ws=None, T=None) -> torch.Tensor:
    """Steady node temperatures (rg_temperatures); T (optional) receives them."""
    n = B.shape[-2]
    if T is None:
        T = torch.empty(n, dtype=torch.float64, device=B.device)
    ctx.check(ctx.lib.rg_temperatures(ctx.handle, n, _dptr(B, torch.float64, "B", n * (n + 1), ctx.device),
                                      _dptr(eps, torch.float64, "eps", n, ctx.device),
                                      _dptr(area, torch.float64, "area", n, ctx.device),
                                      _dptr(Q, torch.float64, "Q", n, ctx.device), float(T_sink), float(sigma),
                                      _prec(precision), float(tol), _dptr(T, torch.float64, "T", n, ctx.device), *_ws(ws, ctx.device), _stream(stream)),
              "rg_temperatures")
    return T


def temperatures_adjoint(ctx: Context, B, eps, area, T_sink: float, T, dT, sigma: float = 5.67e-8,
                         precision="bf16", tol: float = 1e-13, stream=None, ws=None, dB=None, deps=None):
    """(dL/dB [N, N+1], direct dL/deps [N]) from dT = dL/dT (rg_temperatures_adjoint);
    dB and deps (optional) receive them."""
    n = B.shape[-2]
    if dB is None:
        dB = torch.empty((n, n + 1), dtype=torch.float64, device=B.device)
    if deps is None:
        deps = torch.empty(n, dtype=torch.float64, device=B.device)
    ctx.check(ctx.lib.rg_temperatures_adjoint(ctx.handle, n, _dptr(B, torch.float64, "B", n * (n + 1), ctx.device),
                                              _dptr(eps, torch.float64, "eps", n, ctx.device),
                                              _dptr(area, torch.float64, "area", n, ctx.device), float(T_sink),
                                              float(sigma), _dptr(T, torch.float64, "T", n, ctx.device),
                                              _dptr(dT, torch.float64, "dT", n, ctx.device), _prec(precision),
                                              float(tol), _dptr(dB, torch.float64, "dB", n * (n + 1), ctx.device),
                                              _dptr(deps, torch.float64, "deps", n, ctx.device), *_ws(ws, ctx.device), _stream(stream)),
              "rg_temperatures_adjoint")
    return dB, deps


def temperatures_sets(ctx: Context, F, B, eps, rho, area, Q, T_sink: float, sigma: float = 5.67e-8,
                      precision="bf16", tol: float = 1e-13, stream=None, ws=None, T=None) -> torch.Tensor:
    """Steady temperatures of every (eps, rho) set [S, N] (rg_temperatures_sets; F and rho
    precondition the refinement)."""
    n = F.shape[0]
    S = B.numel() // (n * (n + 1))
    if T is None:
        T = torch.empty((S, n), dtype=torch.float64, device=B.device)
    ctx.check(ctx.lib.rg_temperatures_sets(ctx.handle, n, _dptr(F, torch.float64, "F", n * (n + 1), ctx.device), S,
                                           _dptr(B, torch.float64, "B", S * n * (n + 1), ctx.device),
                                           _dptr(eps, torch.float64, "eps", S * n, ctx.device),
                                           _dptr(rho, torch.float64, "rho", S * n, ctx.device),
                                           _dptr(area, torch.float64, "area", n, ctx.device),
                                           _dptr(Q, torch.float64, "Q", S * n, ctx.device), float(T_sink),
                                           float(sigma), _prec(precision), float(tol),
                                           _dptr(T, torch.float64, "T", S * n, ctx.device), *_ws(ws, ctx.device), _stream(stream)),
              "rg_temperatures_sets")
    return T


def temperatures_adjoint_sets(ctx: Context, F, B, eps, rho, area, T_sink: float, T, dT, sigma: float = 5.67e-8,
                              precision="bf16", tol: float = 1e-13, stream=None, ws=None, dB=None, deps=None,
                              factored: bool = False, dB_a=None, dB_b=None):
    """Direct dL/deps [S, N] and dL/dB of every set (rg_temperatures_adjoint_sets): dL/dB in
    full [S, N, N+1], or with factored=True as (a [S, 2, N], b [S, 2, N+1]) with
    dL/dB = sum_r a_r b_r^T. Returns (dB or (a, b), deps)."""
    n = F.shape[0]
    S = B.numel() // (n * (n + 1))
    dev = B.device
    nul = ctypes.c_void_p(None)
    if factored:
        dB_a = torch.empty((S, 2, n), dtype=torch.float64, device=dev) if dB_a is None else dB_a
        dB_b = torch.empty((S, 2, n + 1), dtype=torch.float64, device=dev) if dB_b is None else dB_b
    elif dB is None:
        dB = torch.empty((S, n, n + 1), dtype=torch.float64, device=dev)
    if deps is None:
        deps = torch.empty((S, n), dtype=torch.float64, device=dev)
    ctx.check(ctx.lib.rg_temperatures_adjoint_sets(
        ctx.handle, n, _dptr(F, torch.float64, "F", n * (n + 1), ctx.device), S,
        _dptr(B, torch.float64, "B", S * n * (n + 1), ctx.device), _dptr(eps, torch.float64, "eps", S * n, ctx.device),
        _dptr(rho, torch.float64, "rho", S * n, ctx.device), _dptr(area, torch.float64, "area", n, ctx.device),
        float(T_sink), float(sigma), _dptr(T, torch.float64, "T", S * n, ctx.device),
        _dptr(dT, torch.float64, "dT", S * n, ctx.device), _prec(precision), float(tol),
        nul if factored else _dptr(dB, torch.float64, "dB", S * n * (n + 1), ctx.device),
        _dptr(dB_a, torch.float64, "dB_a", S * 2 * n, ctx.device) if factored else nul,
        _dptr(dB_b, torch.float64, "dB_b", S * 2 * (n + 1), ctx.device) if factored else nul,
        _dptr(deps, torch.float64, "deps", S * n, ctx.device), *_ws(ws, ctx.device), _stream(stream)), "rg_temperatures_adjoint_sets")
    return ((dB_a, dB_b) if factored else dB), deps


def gebhart_adjoint_factored(ctx: Context, F, eps, rho, B, a, b, precision="bf16", tol: float = 1e-12,
                             max_sweeps: int = 12, stream=None, ws=None, deps=None, drho=None, factors=None):
    """(dL/deps, dL/drho) [S, N] for dL/dB = sum_r a_r b_r^T, a [S, r, N], b [S, r, N+1]
    (rg_gebhart_adjoint_factored); factors as in gebhart_adjoint."""
    n = F.shape[0]
    S = eps.numel() // n
    rank = a.shape[-2]
    if deps is None:
        deps = torch.empty((S, n), dtype=torch.float64, device=F.device)
    if drho is None:
        drho = torch.empty((S, n), dtype=torch.float64, device=F.device)
    ctx.check(ctx.lib.rg_gebhart_adjoint_factored(
        ctx.handle, n, _dptr(F, torch.float64, "F", n * (n + 1), ctx.device), S,
        _dptr(eps, torch.float64, "eps", S * n, ctx.device), _dptr(rho, torch.float64, "rho", S * n, ctx.device),
        _dptr(B, torch.float64, "B", S * n * (n + 1), ctx.device), int(rank),
        _dptr(a, torch.float64, "a", S * rank * n, ctx.device),
        _dptr(b, torch.float64, "b", S * rank * (n + 1), ctx.device), _prec(precision), float(tol), int(max_sweeps),
        _dptr(deps, torch.float64, "deps", S * n, ctx.device), _dptr(drho, torch.float64, "drho", S * n, ctx.device),
        *_ws(factors, ctx.device), *_ws(ws, ctx.device), _stream(stream)), "rg_gebhart_adjoint_factored")
    return deps, drho


def debug_wait_timeout(ctx: Context, kind: str, limit_s: float = 0.01, stream=None):
    """Run one bounded device wait against a flag nothing sets (rg_debug_*_timeout);
    raises RadgebError(RG_ERR_CUDA) when the wait runs out, as it should."""
    fn = {"mbarrier": ctx.lib.rg_debug_mbarrier_timeout, "grid": ctx.lib.rg_debug_barrier_timeout}[kind]
    ctx.check(fn(ctx.handle, float(limit_s), _stream(stream)), f"rg_debug_{kind}_timeout")


def tc_gemm(ctx: Context, A: torch.Tensor, B: torch.Tensor, C: torch.Tensor | None = None, alpha: float = 1.0,
            beta: float = 0.0, stream=None) -> torch.Tensor:
    """C = alpha A B^T + beta C on tcgen05 (rg_tc_gemm); A [M, K], B [N, K] bf16 or fp16, C fp32."""
    M, K = A.shape
    N = B.shape[0]
    if B.dtype != A.dtype or A.dtype not in (torch.bfloat16, torch.float16):
        raise TypeError("A and B must both be bf16 or both fp16")
    if C is None:
        C = torch.zeros((M, N), dtype=torch.float32, device=A.device)
    ctx.check(ctx.lib.rg_tc_gemm(ctx.handle, M, N, K, _dptr(A, A.dtype, "A"), A.stride(0), _dptr(B, B.dtype, "B"),
                                 B.stride(0), int(A.dtype == torch.float16), _dptr(C, torch.float32, "C"),
                                 C.stride(0), float(alpha), float(beta), _stream(stream)), "rg_tc_gemm")
    return C


def exact_split(ctx: Context, P: torch.Tensor, dr: torch.Tensor | None = None, trans: bool = False, stream=None):
    """The fixed-point split of P' = P diag(dr) the exact refinement uses (rg_exact_split):
    (slices int16 [n, 5, np], row exponents int32 [n])."""
    n = P.shape[0]
    np_ = (n + 127) // 128 * 128
    sl = torch.empty((n, 5, np_), dtype=torch.int16, device=P.device)
    ex = torch.empty(n, dtype=torch.int32, device=P.device)
    nul = ctypes.c_void_p(None)
    ctx.check(ctx.lib.rg_exact_split(ctx.handle, n, _dptr(P, torch.float64, "P", None, ctx.device), P.stride(0),
                                     int(bool(trans)), nul if dr is None else _dptr(dr, torch.float64, "dr", n),
                                     _dptr(sl, torch.int16, "slices"), _dptr(ex, torch.int32, "rowexp"),
                                     _stream(stream)), "rg_exact_split")
    return sl, ex


def tc_gemm_exact(ctx: Context, A: torch.Tensor, B: torch.Tensor, levels: int, stream=None) -> torch.Tensor:
    """S_a = A_a B^T for integer bf16 operands, a < levels (rg_tc_gemm_exact): int32 [levels, M, N].
    A: [M, >= 5 np], B: [N, np]."""
    M = A.shape[0]
    N, np_ = B.shape
    S = torch.empty((levels, M, N), dtype=torch.int32, device=A.device)
    ctx.check(ctx.lib.rg_tc_gemm_exact(ctx.handle, M, N, np_, int(levels), _dptr(A, torch.bfloat16, "A"), A.stride(0),
                                       _dptr(B, torch.bfloat16, "B"), _dptr(S, torch.int32, "S"), _stream(stream)),
              "rg_tc_gemm_exact")
    return S
