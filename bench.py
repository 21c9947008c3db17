#!/usr/bin/env python
"""Benchmark of the radiative hot path on one GB300 (or N independent replicas).

One step is the whole path on the spacecraft workload, the large model: a procedural
spacecraft (1 x 1 x 1.5 m body, two wings of three tilted 1 m panels, two radiators, a
32-facet boom), 204,512 triangles grouped into N = 10,240 faces, 1e9 rays split by area:
  MCRT counts -> F -> iterative closure/reciprocity enforcer (fp64) -> REFs of 16
  (eps, rho) sets (eps ~ U[0.05, 0.9], rho = 1 - eps; fp16 tensor-core inverse + a
  refinement whose residual is tracked exactly) -> steady temperatures of every set
  (Q ~ U[0, 50] W, 3 K sink) -> their adjoint -> the adjoint of the REFs (dL/deps,
  dL/drho of L = sum of all T; the balance's cotangent dL/dB is rank 2, so K^T is solved
  for two right-hand sides per set).
value = rays traced per second of whole steps (all ranks' rays / the slowest rank).

The plates (N = 512, with the least-squares enforcer and sub-face aggregation) and the
small satellite (N = 2,048) run as extra stages outside the timed steps, as do the
two-faced plates and the plain FP64 GPU path the solves are compared with.

--impl reference times the CPU oracle (the tests' reference implementation) on the host
cores on a bounded sample of the same step and reports the same metric; the bench
line's cpu_baseline is the same measurement.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "MCRT rays/s; Gebhart+adjoint solve ms vs plain FP64 GPU path at 1e-6 error"
HEADLINE = "spacecraft"
WORKLOADS = {
    "spacecraft": ("spacecraft: body + 6 tilted panels + 2 radiators + boom, 204,512 triangles grouped into "
                   "N=10,240 faces, 1e9 rays split by area per step; iterative fp64 enforcement; REFs of 16 eps/rho "
                   "sets (fp16 tensor-core inverse + refinement with an exactly tracked residual); steady "
                   "temperatures of every set (Q ~ U[0,50] W, 3 K sink) and their adjoints; REF adjoints of every "
                   "set (dL/deps, dL/drho of L = sum T, the balance's rank-2 cotangent)"),
    "plates": ("plates: 2 x (16 x 16) sub-faces, N=512, 1,024 triangles, 1e6 rays/sub-face (5.12e8 per step); "
               "iterative + least-squares (NNR+SPVA) enforcement; sub-face->plate aggregation; REFs (N=512, fp16 "
               "tensor-core inverse + fp64-accurate refinement); steady temperatures + adjoints"),
    "small_sat": ("small satellite: box body + 4 hinged panels, 20,736 triangles grouped into N=2,048 faces, 1e8 "
                  "rays split by area; iterative enforcement; REFs (fp16 inverse + refinement); steady "
                  "temperatures + adjoints"),
}
SIGMA = 5.67e-8
T_SINK = 3.0
# Refinement tolerance of the dense solves (relative residual). The refinement tracks its
# residual exactly, so the tolerance sets the accuracy: on the spacecraft, 1e-10 takes five
# sweeps and leaves B 1e-10 from the fp64 solution (row-normwise), the temperatures 5e-9 and
# the gradients 2e-8; 1e-8 stops a sweep earlier but lets the gradients drift to 3e-6.
SOLVE_TOL = 1e-10
# 16-bit type of the tensor-core factorisations: fp16 keeps three more mantissa bits than
# bf16, so its approximate inverses need fewer refinement sweeps (N = 512: 2.95 against
# 3.42 ms for the four solves); the matrices here are bounded by 1, far from fp16's range
SOLVE_PRECISION = "fp16"
# Algorithmic operations of the ray definition: per ray one Philox4x32-10 block (78
# integer operations: 10 rounds of two 32 x 32 -> 64-bit products and four xors, and the
# key schedule), the triangle choice, the point and the polar direction (52 float
# operations, the sine / cosine polynomials included) and the tally: 193 in all; per box
# and triangle test the survey's counts (slab test: 12 float + 6 min/max; Moller-Trumbore:
# 44 float + 1 reciprocal).
OPS_PER_RAY = 193
OPS_PER_BOX = 18
OPS_PER_TRI = 45
# Iterations of the fp64 enforcer on the spacecraft view factors at tol 1e-12 (the count
# the bench line reports as "iterative_iters"); the CPU sample times two oracle
# iterations and scales them by this count.
ENFORCE_ITERS = {"spacecraft": 91}


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--no-e2e", action="store_true", help=argparse.SUPPRESS)
    ap.add_argument("--no-extras", action="store_true",
                    help="only the headline step, its roofline and e2e (no extra stages, FP64 path or CPU sample)")
    ap.add_argument("--trace-once", type=float, default=None, metavar="SCALE",
                    help="instead of the bench line, run one trace launch of --mesh at SCALE x its ray budget "
                         "(the small case the ncu captures use) and print the ray count")
    ap.add_argument("--mesh", default="plates", choices=["plates", "small_sat", "spacecraft"],
                    help="mesh of --trace-once")
    ap.add_argument("--sided", action="store_true",
                    help="with --trace-once: the side-resolved trace of the two-faced plates instead")
    ap.add_argument("--enforce-once", type=int, nargs=2, default=None, metavar=("N", "ITERS"),
                    help="instead of the bench line, run the iterative enforcer once on a seeded N x (N+1) "
                         "matrix for ITERS iterations (the small case its ncu captures use)")
    ap.add_argument("--solve-once", type=int, default=None, metavar="SETS",
                    help="instead of the bench line, run the spacecraft solves (REFs, temperatures, both adjoints) "
                         "for SETS eps/rho sets once on a 1e7-ray F (the case the solver's ncu captures use)")
    ap.add_argument("--solve-n", type=int, default=None, metavar="N",
                    help="with --solve-once: a seeded random N-face system (F_ij ~ U[0, 1.5/N] off the diagonal, "
                         "the rest of each row to the environment, areas U[0.5, 2]) instead of the spacecraft")
    ap.add_argument("--solve-band", type=int, default=0, metavar="W",
                    help="with --solve-n: F non-zero only within W of the diagonal (row sums kept), so that most "
                         "256 x 64 blocks of the exact product's slices are zero, as on the spacecraft")
    ap.add_argument("--reflect", action="store_true",
                    help="instead of the bench line, print one JSON line with the reflection walk's rates "
                         "(REFs by MCRT) on the plates and the cube")
    ap.add_argument("--bvh-build", action="store_true",
                    help="instead of the bench line, print one JSON line comparing the host and device BVH "
                         "builders (build time, tree, trace rate) on the small-satellite and spacecraft meshes")
    ap.add_argument("--solve-scaling", action="store_true",
                    help="instead of the bench line, print one JSON line with tensor-core GEMM rates and REF "
                         "solve + adjoint times against the FP64 GPU path at N = 512, 2,048 and 10,240")
    return ap.parse_args()


# ------------------------------------------------------------------ clocks
class ClockSampler:
    """nvidia-smi samples (200 ms) of the SM clock and throttle reasons during a region."""

    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,clocks_event_reasons.hw_slowdown,"
              "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
              "clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.rows = []
        self.proc = None

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                                          "-i", str(self.index), "-lms", "200"], stdout=subprocess.PIPE,
                                         stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except OSError:
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            parts = [p.strip() for p in line.split(",")]
            if len(parts) == 8:
                self.rows.append(parts)

    def __exit__(self, *a):
        if self.proc:
            time.sleep(0.25)
            self.proc.terminate()
            try:
                self.proc.wait(timeout=2)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self):
        if not self.rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"]}
        sm = [float(r[0]) for r in self.rows if r[0].replace(".", "").isdigit()]
        mx = [float(r[1]) for r in self.rows if r[1].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[k] for r in self.rows for k in range(4) if r[4 + k].lower() == "active"})
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(self.rows)}


# ------------------------------------------------------------------ our implementation
STAGES = ("mcrt", "enforce", "refs", "thermal", "adjoint")


def load_workload(name, rays_scale=1.0):
    """The synthetic workload with its heat loads (Q ~ U[0, 50] W, seed 3) for the balance."""
    import synth
    w = synth.workload("thermal" if name == "plates" else name, rays_scale=rays_scale)
    if "Q" not in w:
        w["Q"] = synth.heat_loads(w["mesh"].n_faces, seed=3)
    return w


class Pipeline:
    """The hot path on one workload: MCRT -> F -> enforcement (with the least-squares
    optimum and the sub-face aggregation when `lsq`) -> REFs of every (eps, rho) set ->
    temperatures and their adjoint per set -> REF adjoint of all sets."""

    def __init__(self, ctx, w, device, lsq=False, gpu_bvh=False):
        import torch
        from paper_2511_04277_gb300 import api
        self.api, self.torch, self.ctx, self.w, self.lsq = api, torch, ctx, w, lsq
        m = w["mesh"]
        self.N = N = m.n_faces
        self.S = S = w["eps"].shape[0]
        d = dict(device=device)
        self.device = device
        self.mesh = api.Mesh.from_synth(ctx, m, gpu_bvh=gpu_bvh)
        self.rays_h = np.ascontiguousarray(w["rays"], np.int64)
        self.rays = torch.as_tensor(self.rays_h, **d)
        self.areas = torch.as_tensor(self.mesh.face_areas(), **d)
        self.groups = torch.as_tensor(m.patch_of_face.astype(np.int32), **d)
        self.eps = torch.as_tensor(w["eps"], **d)
        self.rho = torch.as_tensor(w["rho"], **d)
        self.Q = torch.as_tensor(w["Q"], **d)
        self.ones = torch.ones(N, dtype=torch.float64, **d)
        f64 = dict(dtype=torch.float64, **d)
        self.counts = torch.zeros((N, N + 1), dtype=torch.int64, **d)
        self.F = torch.empty((N, N + 1), **f64)
        self.F_it = torch.empty_like(self.F)
        self.F_ls = torch.empty_like(self.F) if lsq else None
        self.B = torch.empty((S, N, N + 1), **f64)
        # the REF solve keeps each set's 16-bit inverse here; the REF adjoint reads it
        self.factors = api.gebhart_factor_store(N, S, SOLVE_PRECISION, device=torch.device(device).index or 0)
        self.dB_a = torch.empty((S, 2, N), **f64)      # dL/dB of the balance, factored: sum_r a_r b_r^T
        self.dB_b = torch.empty((S, 2, N + 1), **f64)
        self.T = torch.empty((S, N), **f64)
        self.deps_T = torch.empty((S, N), **f64)
        self.Qs = self.Q.expand(S, N).contiguous()
        self.dT = torch.ones((S, N), **f64)
        self.rays_per_step = int(self.rays_h.sum())

    def load_inputs(self, host, gpu_bvh=True):
        """Replace the mesh and the per-step inputs from host buffers (the e2e path): the
        mesh and its BVH are built again from the host arrays, rays / eps / rho / Q copied in
        from pinned memory, the face areas recomputed."""
        self.mesh.close()
        m = self.w["mesh"]
        self.mesh = self.api.Mesh(self.ctx, m.verts, m.tris, m.tri_face, self.N, gpu_bvh=gpu_bvh)
        for k in ("rays", "eps", "rho", "Q"):
            getattr(self, k).copy_(host[k], non_blocking=True)
        self.Qs.copy_(self.Q.expand(self.S, self.N))
        self.areas.copy_(self.torch.as_tensor(self.mesh.face_areas()), non_blocking=True)

    def mcrt(self):
        api = self.api
        self.counts.zero_()
        api.trace(self.ctx, self.mesh, self.rays_h, self.w["seed"], fma_free=True, counts=self.counts)
        api.counts_to_F(self.ctx, self.counts, self.rays, self.F)

    def enforce(self):
        api = self.api
        self.F_it.copy_(self.F)
        self.iters = api.enforce_iterative(self.ctx, self.F_it, self.areas, tol=1e-12)
        if self.lsq:
            self.F_ls.copy_(self.F)
            self.passes = api.enforce_lsq(self.ctx, self.F_ls, self.areas, nnr=True, spva=True)
            self.Fg, self.Sg = api.aggregate(self.ctx, self.F_it, self.areas, self.groups, 2)

    def refs(self):
        _, self.sweeps, self.resid = self.api.gebhart(self.ctx, self.F_it, self.eps, self.rho, SOLVE_PRECISION,
                                                      tol=SOLVE_TOL, B=self.B, factors=self.factors,
                                                      areas=self.areas)

    def thermal(self):
        """Steady temperatures of every set and their adjoint (dL/dB, direct dL/deps of
        L = sum T), all sets in one call each (one shared balance preconditioner)."""
        api, p = self.api, SOLVE_PRECISION
        api.temperatures_sets(self.ctx, self.F_it, self.B, self.eps, self.rho, self.areas, self.Qs, T_SINK, SIGMA,
                              precision=p, tol=SOLVE_TOL, T=self.T)
        api.temperatures_adjoint_sets(self.ctx, self.F_it, self.B, self.eps, self.rho, self.areas, T_SINK, self.T,
                                      self.dT, SIGMA, precision=p, tol=SOLVE_TOL, deps=self.deps_T, factored=True,
                                      dB_a=self.dB_a, dB_b=self.dB_b)

    def adjoint(self):
        """The REF adjoint of every set for the balance's cotangent dL/dB = sum_r a_r b_r^T
        (rank 2): K^T solved for the two left factors of each set, with the inverses the
        REF solve kept (no second factorisation)."""
        self.deps_B, self.drho = self.api.gebhart_adjoint_factored(self.ctx, self.F_it, self.eps, self.rho, self.B,
                                                                   self.dB_a, self.dB_b, precision=SOLVE_PRECISION,
                                                                   tol=SOLVE_TOL, factors=self.factors)

    def step(self, marks=None, stream=None):
        """One pass of the path; with `marks` (one CUDA event per stage) each stage's end is
        recorded on `stream`."""
        for k, name in enumerate(STAGES):
            getattr(self, name)()
            if marks is not None:
                marks[k].record(stream)


def profiled_traffic(summary, source, units):
    """DRAM bytes per launch from a committed ncu summary (profiles/<summary>): the lines
    'source_sha256: <hash of csrc/<source> when captured>' and 'dram_bytes_per_unit: <x>'.
    None when the summary is missing or the kernel source has changed since the capture."""
    import hashlib
    import re
    path = os.path.join(ROOT, "profiles", summary)
    src = os.path.join(ROOT, "paper_2511_04277_gb300", "csrc", source)
    if not os.path.exists(path):
        return None
    text = open(path).read()
    m_sha = re.search(r"source_sha256:\s*`?([0-9a-f]{64})", text)
    m_per = re.search(r"dram_bytes_per_unit:\s*([0-9.eE+-]+)", text)
    sha = hashlib.sha256(open(src, "rb").read()).hexdigest()
    if not m_sha or not m_per or m_sha.group(1) != sha:
        return None
    return float(m_per.group(1)) * units


def lu_equivalent_flops(N, S, sweeps_refs, with_thermal=True):
    """Algorithmic flops of the solve stage, counted as an LU-based solver would do them:
    per set, the REFs (2/3 N^3 + 2 N^2 (N+1), plus 2 N^2 (N+1) per refinement sweep), the REF
    adjoint (2/3 N^3 + 2 N^2 (N+1) for the transposed solve + 2 N^2 (N+1) for Lambda B^T) and
    the balance and its adjoint (2/3 N^3 + 2 N^2 each)."""
    refs = 2.0 / 3.0 * N ** 3 + 2.0 * N * N * (N + 1) * (1 + sweeps_refs)
    adj = 2.0 / 3.0 * N ** 3 + 4.0 * N * N * (N + 1)
    th = 2.0 * (2.0 / 3.0 * N ** 3 + 2.0 * N * N) if with_thermal else 0.0
    return S * (refs + adj + th)


def trace_roofline(api, torch, ctx, pipe, trace_ms, peaks, device, summary=None):
    """ALU roofline of the trace kernel: the ray definition's algorithmic operations per
    launch (per ray, per box test, per triangle test; tests counted by rg_trace_stats on the
    same rays) over the kernel's mean launch time."""
    counts_tmp = torch.zeros_like(pipe.counts)
    _, st = api.trace_stats(ctx, pipe.mesh, pipe.rays_h, pipe.w["seed"], counts=counts_tmp)
    del counts_tmp
    ops = st["rays"] * OPS_PER_RAY + st["box_tests"] * OPS_PER_BOX + st["tri_tests"] * OPS_PER_TRI
    sm_count = torch.cuda.get_device_properties(device).multi_processor_count
    max_mhz = float(peaks.get("sm_max_mhz", 2070.0))
    peak = sm_count * 128 * max_mhz * 1e6 / 1e12
    achieved = ops / (trace_ms * 1e-3) / 1e12
    out = {"kernel": "trace_kernel<fma_free, BVH>", "bound": "alu", "achieved": round(achieved, 3),
           "peak": round(peak, 3), "unit": "Tops/s", "frac": round(achieved / peak, 4), "traffic": None,
           "ops_per_ray": round(ops / st["rays"], 1), "ops_basis": f"{OPS_PER_RAY}/ray + {OPS_PER_BOX}/box test + "
                                                                  f"{OPS_PER_TRI}/triangle test",
           "box_tests_per_ray": round(st["box_tests"] / st["rays"], 3),
           "tri_tests_per_ray": round(st["tri_tests"] / st["rays"], 3), "trace_ms": round(trace_ms, 3),
           "rays_per_s": st["rays"] / (trace_ms * 1e-3),
           "peak_basis": f"{sm_count} SMs x 128 lanes x {max_mhz:.0f} MHz (sm_max_mhz, MEASURED_PEAKS.json)"}
    if summary:
        out["traffic"] = profiled_traffic(summary, "trace.cu", st["rays"])
    return out


def fp64_solve(torch, F, eps, rho, A, Q):
    """Plain FP64 GPU path for one (eps, rho) set: torch.linalg.solve (cuSOLVER) for the
    REFs and the balance, FP64 autograd for dL/deps, dL/drho of L = sum T."""
    N = F.shape[0]
    e = eps.detach().clone().requires_grad_(True)
    r = rho.detach().clone().requires_grad_(True)
    with torch.enable_grad():
        FN = F[:, :N]
        K = torch.eye(N, dtype=F.dtype, device=F.device) - FN * r[None, :]
        E = torch.cat([FN * e[None, :], F[:, N:]], dim=1)
        B = torch.linalg.solve(K, E)
        g = SIGMA * e * A
        t = B.sum(dim=1)
        M = torch.diag(g * t) - g[:, None] * B[:, :N]
        u = torch.linalg.solve(M, Q + g * B[:, N] * T_SINK ** 4)
        T = u ** 0.25
        T.sum().backward()
    return B.detach(), T.detach(), e.grad, r.grad


def load_peaks():
    """MEASURED_PEAKS.json (the machine's measured HBM copy and bf16 GEMM rates), or {}."""
    try:
        return json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except OSError:
        return {}


def l2_flusher(torch, device):
    buf = torch.empty(256 << 20, dtype=torch.uint8, device=device)

    def flush():
        buf.fill_(1)
    return flush


def time_region(torch, fn, stream):
    s, e = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    s.record(stream)
    fn()
    e.record(stream)
    e.synchronize()
    return s.elapsed_time(e)


def max_over_ranks(torch, dist, value, world, device):
    """The largest of every rank's value (all_reduce MAX); the value itself on one rank."""
    if world <= 1:
        return float(value)
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_throughput(units_per_rank, world, ms):
    """Whole-job units per second: every rank's units over the slowest rank's time."""
    return units_per_rank * world / (ms * 1e-3)


def rownorm(x, y):
    """max_i max_j |x_ij - y_ij| / max_j |y_ij| (the row-normwise relative error)."""
    return float(((x - y).abs().amax(dim=-1) / y.abs().amax(dim=-1).clamp_min(1e-300)).max())


def enforce_bytes(n, iters, pair_frac=1.0):
    """Algorithmic HBM bytes of `iters` equal-weight enforcer iterations: the first reads and
    writes the whole N x (N+1) matrix (16 B per entry); every later one, on the symmetric
    matrix, the tiles on and above the diagonal that hold a non-zero (pair_frac of them: the
    zero ones stay zero and are skipped) and the environment column (16 B per stored entry)."""
    if iters <= 0:
        return 0.0
    return 16.0 * n * (n + 1) + 16.0 * (iters - 1) * (pair_frac * n * (n + 1) / 2.0 + n)


def nonzero_pair_fraction(F):
    """Fraction of the enforcer's tile pairs (I, J), I <= J, whose tiles (I, J) or (J, I) of
    the N x N block hold a non-zero (32-wide tiles up to N = 2,048, 64-wide above, as the
    enforcer takes them)."""
    import torch
    n = F.shape[0]
    t = 32 if n <= 2048 else 64
    nt = (n + t - 1) // t
    Z = torch.zeros((nt * t, nt * t), dtype=torch.bool, device=F.device)
    Z[:n, :n] = F[:, :n] != 0
    blk = Z.view(nt, t, nt, t).any(dim=3).any(dim=1)
    blk = blk | blk.T
    return float(torch.triu(blk).sum()) / (nt * (nt + 1) / 2)


def kernel_rooflines(api, ctx, pipe, steps, step_ms, peaks, trace_roof):
    """Per kernel class over the timed steps (the library's kernel timer: CUDA events on the
    launching stream around every launch): share of the step, mean launch time and the
    roofline of its bound."""
    hbm = float(peaks.get("hbm_gbs", 6800.0))
    tc = float(peaks.get("bf16_tflops_sustained", peaks.get("bf16_tflops", 1900.0)))
    out = {}
    for kind in ("trace", "residual_gemm", "gemm", "enforce"):
        r = api.kernel_timer_read(ctx, kind)
        if not r["launches"]:
            continue
        per_launch = r["ms"] / r["launches"]
        row = {"launches_per_step": r["launches"] / steps, "ms_per_step": round(r["ms"] / steps, 3),
               "share_of_step": round(r["ms"] / steps / step_ms, 4), "ms_per_launch": round(per_launch, 4)}
        if kind == "trace":
            ops = trace_roof["achieved"] * 1e12 * trace_roof["trace_ms"] * 1e-3
            ach = ops / (per_launch * 1e-3) / 1e12
            row.update({"kernel": trace_roof["kernel"], "bound": "alu", "achieved": round(ach, 3),
                        "peak": trace_roof["peak"], "unit": "Tops/s", "frac": round(ach / trace_roof["peak"], 4),
                        "traffic": trace_roof["traffic"], "peak_basis": trace_roof["peak_basis"]})
        elif kind in ("residual_gemm", "gemm"):
            alg = r["alg_flops"] / r["ms"] / 1e9
            exe = r["flops"] / r["ms"] / 1e9
            if kind == "residual_gemm":
                # DRAM bytes per executed flop from the committed full-size capture of the
                # spacecraft's exact products, times the executed flops of a mean launch
                traffic = profiled_traffic("exact_gemm_spacecraft.md", "tc_gemm.cuh", r["flops"] / r["launches"])
            else:
                # DRAM bytes per executed flop from the committed full-size capture
                traffic = profiled_traffic("gemm_pair_n4096.md", "tc_gemm.cuh", r["flops"] / r["launches"])
            row.update({"kernel": "tc::gemm_exact_pair_kernel (tcgen05, exact integer level products, zero "
                                  "blocks skipped)"
                        if kind == "residual_gemm" else "tc::gemm_kernel (tcgen05: Newton-Schulz steps, corrections)",
                        "bound": "tensor", "achieved": round(exe, 2), "peak": tc, "unit": "TFLOP/s",
                        "frac": round(exe / tc, 4), "traffic": None if traffic is None else round(traffic),
                        "executed_tflops": round(exe, 2), "executed_frac": round(exe / tc, 4),
                        "peak_basis": "bf16_tflops_sustained of MEASURED_PEAKS.json (kernel timed inside a long "
                                      "step); fp16 has the bf16 rate"})
            if kind == "residual_gemm":
                row["one_slice_dense_tflops"] = round(alg, 2)
                row["note"] = ("achieved = the tensor flops the launches execute: 2 x 256 x 256 x 64 per 256 x 64 "
                               "block of a level's slice holding a non-zero digit (the all-zero blocks are skipped); "
                               "one_slice_dense_tflops counts the dense one-slice product P' D each launch stands "
                               "for (2 n m n per sweep), for comparison")
            else:
                row["note"] = "achieved = executed tensor flops (2 M N K)"
        else:
            it = getattr(pipe, "iters", 0)
            frac = nonzero_pair_fraction(pipe.F_it)
            gb = enforce_bytes(pipe.N, it, frac) / (per_launch * 1e-3) / 1e9
            # DRAM bytes per algorithmic byte from the committed capture at N = 6,144
            traffic = profiled_traffic("enforce_persistent_n6144.md", "enforce.cu", enforce_bytes(pipe.N, it, frac))
            row.update({"kernel": "enforce_persistent", "bound": "hbm", "achieved": round(gb, 1), "peak": hbm,
                        "unit": "GB/s", "frac": round(gb / hbm, 4),
                        "traffic": None if traffic is None else round(traffic),
                        "nonzero_tile_pairs": round(frac, 4),
                        "note": f"{it} iterations per launch: the first reads and writes every entry (16 B), the "
                                "symmetric ones after it the tiles on and above the diagonal that hold a non-zero "
                                "(16 B per stored entry, one fp64 multiplication each, fixed-point row sums)"})
        out[kind] = row
    r = api.kernel_timer_read(ctx, "factor")
    if r["launches"]:
        out["factor"] = {"regions_per_step": r["launches"] / steps, "ms_per_step": round(r["ms"] / steps, 3),
                         "share_of_step": round(r["ms"] / steps / step_ms, 4),
                         "ms_per_factorisation": round(r["ms"] / r["launches"], 4),
                         "note": "Newton-Schulz inverses, start iterate to last step (their GEMMs are also in gemm)"}
    return out


def run_ours(args):
    import torch
    import torch.distributed as dist
    from paper_2511_04277_gb300 import api

    rank = int(os.environ.get("RANK", 0))
    world = int(os.environ.get("WORLD_SIZE", 1))
    local = int(os.environ.get("LOCAL_RANK", 0))
    if world > 1:
        dist.init_process_group("nccl", device_id=torch.device(f"cuda:{local}"))
    torch.cuda.set_device(local)
    device = torch.device(f"cuda:{local}")
    stream = torch.cuda.current_stream()
    ctx = api.Context(local)
    w = load_workload(HEADLINE)
    pipe = Pipeline(ctx, w, device)
    flush = l2_flusher(torch, device)
    rays_per_step = pipe.rays_per_step

    def barrier():
        if world > 1:
            dist.barrier()
        torch.cuda.synchronize()

    for _ in range(max(args.warmup, 0)):
        pipe.step()
    barrier()
    launches0 = api.launch_count(ctx)
    marks_all, starts = [], []
    api.kernel_timer(ctx, True)
    with ClockSampler(local) as clk:
        barrier()
        t0 = time.perf_counter()
        for _ in range(args.steps):
            flush()
            st_ev = torch.cuda.Event(enable_timing=True)
            marks = [torch.cuda.Event(enable_timing=True) for _ in STAGES]
            st_ev.record(stream)
            pipe.step(marks, stream)
            starts.append(st_ev)
            marks_all.append(marks)
        barrier()
        wall = time.perf_counter() - t0
    api.kernel_timer(ctx, False)
    launches = api.launch_count(ctx) - launches0
    step_ms = [s.elapsed_time(m[-1]) for s, m in zip(starts, marks_all)]
    stage_ms = {}
    for k, name in enumerate(STAGES):
        vals = [(s if k == 0 else m[k - 1]).elapsed_time(m[k]) for s, m in zip(starts, marks_all)]
        stage_ms[name] = round(statistics.mean(vals), 3)
    ms = max_over_ranks(torch, dist, statistics.mean(step_ms), world, device)

    out = None
    if rank == 0:
        peaks = load_peaks()
        trace_roof = trace_roofline(api, torch, ctx, pipe, stage_ms["mcrt"], peaks, device,
                                    summary="trace_kernel_spacecraft.md")
        kroof = kernel_rooflines(api, ctx, pipe, args.steps, statistics.mean(step_ms), peaks, trace_roof)
        dominant = max(kroof, key=lambda k: kroof[k]["ms_per_step"]) if kroof else None
        roofline = dict(kroof[dominant]) if dominant else trace_roof
        if dominant:
            roofline["class"] = dominant
        solve_ms = stage_ms["refs"] + stage_ms["thermal"] + stage_ms["adjoint"]
        solve = {"n": pipe.N, "sets": pipe.S, "ours_ms": round(solve_ms, 2),
                 "refs_ms": stage_ms["refs"], "thermal_ms": stage_ms["thermal"], "adjoint_ms": stage_ms["adjoint"],
                 "sweeps": pipe.sweeps, "residual": pipe.resid,
                 "precision": f"{SOLVE_PRECISION} tensor cores + fp64-accurate refinement, tol {SOLVE_TOL:g}",
                 "fp64_path": "torch.linalg.solve float64 + FP64 autograd, one set timed x 16"}
        lu = lu_equivalent_flops(pipe.N, pipe.S, pipe.sweeps)
        tc_peak = float(peaks.get("bf16_tflops_sustained", 1735.6))
        stage_roof = {
            "solve": {"kernel": "tcgen05 GEMMs + helpers (REFs, balances, both adjoints)", "bound": "tensor",
                      "achieved": round(lu / (solve_ms * 1e-3) / 1e12, 2), "peak": tc_peak, "unit": "TFLOP/s",
                      "frac": round(lu / (solve_ms * 1e-3) / 1e12 / tc_peak, 4),
                      "flops_basis": "LU-equivalent: per set 2/3 N^3 + 2 N^2 (N+1) (1 + sweeps) REFs, 2/3 N^3 + "
                                     "4 N^2 (N+1) REF adjoint, 2 (2/3 N^3 + 2 N^2) balance + adjoint"},
            "trace": trace_roof}
        if "enforce" in kroof:
            stage_roof["enforce_iterative"] = kroof["enforce"]
        out = {
            "metric": METRIC, "value": job_throughput(rays_per_step, world, ms), "unit": "rays/s", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(ms, 3), "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None,
            "dtype": f"f32 rays, i64 tallies, f64 enforcement, {SOLVE_PRECISION} tensor-core inverse + f64 refinement",
            "data": "synthetic",
            "config": {"workload": WORKLOADS[HEADLINE], "faces": pipe.N, "triangles": int(w["mesh"].n_tris),
                       "sets": pipe.S, "rays_per_step": rays_per_step, "parallelism": f"replicas x{world}",
                       "l2": "256 MiB buffer written before every timed step (and every step's data, >13 GB, "
                             "exceeds L2); per-step CUDA events exclude the flush",
                       "wall_s_timed_region": round(wall, 3)},
            "stage_ms": stage_ms, "mcrt_rays_per_s": rays_per_step / (stage_ms["mcrt"] * 1e-3),
            "enforce": {"iterative_iters": pipe.iters},
            "solve": solve, "roofline": roofline, "kernel_rooflines": kroof, "stage_rooflines": stage_roof,
            "clocks": clk.summary(), "gpu_launches": int(launches),
        }
        if not args.no_extras:
            out["solve"].update(fp64_comparison(torch, pipe))
            if out["solve"].get("fp64_ms"):
                out["solve"]["speedup"] = round(out["solve"]["fp64_ms"] / solve_ms, 2)
            out["extra_stages"] = extra_stages(api, torch, ctx, flush, stream, device, peaks)
        if not args.no_e2e:
            out["e2e"] = run_e2e(args, api, torch, pipe, stream)
        if not args.no_extras:
            out["cpu_baseline"] = cpu_baseline(w)
    if world > 1:
        dist.barrier()
        dist.destroy_process_group()
    ctx.close()
    return out


def fp64_comparison(torch, pipe):
    """The plain FP64 GPU path on set 0 (timed once, scaled to the sets of the step) and the
    errors of our set-0 outputs against it."""
    try:
        # cuSOLVER's handle and workspace outside the timing: one small well-posed solve
        g = torch.Generator(device=pipe.F_it.device).manual_seed(0)
        Kw = torch.eye(64, dtype=torch.float64, device=pipe.F_it.device) + 0.01 * torch.rand(
            (64, 64), dtype=torch.float64, device=pipe.F_it.device, generator=g)
        torch.linalg.solve(Kw, torch.ones((64, 2), dtype=torch.float64, device=pipe.F_it.device))
        torch.cuda.synchronize()
        box = [None]
        ms = time_region(torch, lambda: box.__setitem__(0, fp64_solve(torch, pipe.F_it, pipe.eps[0], pipe.rho[0],
                                                                      pipe.areas, pipe.Q)),
                         torch.cuda.current_stream())
        B64, T64, de64, dr64 = box[0]
        grad = pipe.deps_B[0] + pipe.deps_T[0]
        out = {"fp64_ms": round(ms * pipe.S, 1), "fp64_ms_one_set": round(ms, 1),
               "err_B_rownorm": rownorm(pipe.B[0], B64),
               "err_T": float((pipe.T[0] - T64).abs().max() / T64.abs().max()),
               "err_deps": float((grad - de64).abs().max() / de64.abs().max()),
               "err_drho": float((pipe.drho[0] - dr64).abs().max() / dr64.abs().max()),
               "closure_B": float((pipe.B.sum(dim=-1) - 1.0).abs().max()),
               "closure_B_fp64": float((B64.sum(dim=-1) - 1.0).abs().max()),
               "errors_basis": "set 0 against the FP64 path; closure_B = max over all sets and rows of "
                               "|sum_j B_ij - 1| (Eq. 4.3)"}
        del B64, T64, de64, dr64
        torch.cuda.empty_cache()
        return out
    except RuntimeError as exc:  # e.g. torch's cuSOLVER wrapper failing to load in this process
        return {"fp64_ms": None, "fp64_unavailable": str(exc).splitlines()[0][:200]}


def extra_stages(api, torch, ctx, flush, stream, device, peaks):
    """The plates and small-satellite workloads (whole steps, median of three after a
    warm-up, with their trace rooflines), the plates solve against the FP64 path, the
    plates stage rooflines and the two-faced plates."""
    import synth
    out = {}
    for name in ("plates", "small_sat"):
        w = load_workload(name)
        p = Pipeline(ctx, w, device, lsq=(name == "plates"))
        p.step()
        torch.cuda.synchronize()
        vals, tr = [], []
        for _ in range(3):
            flush()
            st_ev = torch.cuda.Event(enable_timing=True)
            marks = [torch.cuda.Event(enable_timing=True) for _ in STAGES]
            st_ev.record(stream)
            p.step(marks, stream)
            marks[-1].synchronize()
            vals.append(st_ev.elapsed_time(marks[-1]))
            tr.append(st_ev.elapsed_time(marks[0]))
        ms = statistics.median(vals)
        row = {"workload": WORKLOADS[name], "faces": p.N, "rays_per_step": p.rays_per_step,
               "ms_per_step": round(ms, 3), "rays_per_s": p.rays_per_step / (ms * 1e-3),
               "mcrt_ms": round(statistics.median(tr), 3), "iterative_iters": p.iters, "sweeps": p.sweeps,
               "trace_roofline": trace_roofline(api, torch, ctx, p, statistics.median(tr), peaks, device,
                                                summary=f"trace_kernel_{name}.md")}
        if name == "plates":
            row["passes_lsq"] = p.passes
            row["stage_rooflines"] = stage_rooflines(api, torch, ctx, p, flush, stream, peaks)
            cmp_ = fp64_comparison(torch, p)
            solve_ms = []
            for _ in range(3):
                flush()
                solve_ms.append(time_region(torch, lambda: (p.refs(), p.thermal(), p.adjoint()), stream))
            cmp_["ours_ms"] = round(statistics.median(solve_ms), 4)
            if cmp_.get("fp64_ms"):
                cmp_["speedup"] = round(cmp_["fp64_ms"] / cmp_["ours_ms"], 2)
            row["solve"] = cmp_
        out[name] = row
        p.mesh.close()
        del p
        torch.cuda.empty_cache()
    out["sided"] = sided_stage(api, torch, ctx, flush, stream, synth, peaks)
    return out


def stage_rooflines(api, torch, ctx, pipe, flush, stream, peaks):
    """Achieved fractions of the iterative enforcer (HBM bound: 16 B per entry in the first
    iteration, 16 B per stored entry of the upper triangle in the later ones), the REF solve
    (tensor bound; LU-equivalent flops, 2/3 N^3 + 2 N^2 (N+1), plus
    2 N^2 (N+1) per refinement sweep) and the least-squares enforcer on a small workload."""
    N = pipe.N
    F = torch.empty_like(pipe.F)
    t_enf, iters = [], 0
    for _ in range(3):
        F.copy_(pipe.F)
        flush()
        box = [0]
        t_enf.append(time_region(torch, lambda: box.__setitem__(0, api.enforce_iterative(ctx, F, pipe.areas,
                                                                                          tol=1e-12)), stream))
        iters = box[0]
    ms_e = statistics.median(t_enf)
    pf = nonzero_pair_fraction(F)
    gbs = enforce_bytes(N, iters, pf) / (ms_e * 1e-3) / 1e9
    hbm = float(peaks.get("hbm_gbs", 6800.0))
    t_ref, sweeps = [], 0
    for _ in range(3):
        flush()
        box = [0]
        t_ref.append(time_region(torch, lambda: box.__setitem__(0, api.gebhart(
            ctx, pipe.F_it, pipe.eps, pipe.rho, SOLVE_PRECISION, tol=SOLVE_TOL, B=pipe.B)[1]), stream))
        sweeps = box[0]
    ms_r = statistics.median(t_ref)
    flops = 2.0 / 3.0 * N ** 3 + 2.0 * N * N * (N + 1) * (1 + sweeps)
    tf = flops / (ms_r * 1e-3) / 1e12
    bf = float(peaks.get("bf16_tflops", 1900.0))
    t_l, passes = [], 0
    for _ in range(3):
        F.copy_(pipe.F)
        flush()
        box = [0]
        t_l.append(time_region(torch, lambda: box.__setitem__(0, api.enforce_lsq(ctx, F, pipe.areas, nnr=True,
                                                                                  spva=True)), stream))
        passes = box[0]
    ms_l = statistics.median(t_l)
    lsq_flops = passes * (2.0 / 3.0 * N ** 3 + 2.0 * N * N * 4)
    tf_l = lsq_flops / (ms_l * 1e-3) / 1e12
    return {
        "enforce_lsq": {"kernel": "lsq_* + gemm_kernel (tcgen05) solve of the Schur complement", "bound": "tensor",
                        "achieved": round(tf_l, 3), "peak": bf, "unit": "TFLOP/s", "frac": round(tf_l / bf, 5),
                        "passes": passes, "ms": round(ms_l, 4),
                        "note": f"N={N}: launch- and latency-bound like the REF solve"},
        "enforce_iterative": {"kernel": "enforce_persistent", "bound": "hbm", "achieved": round(gbs, 1),
                              "peak": hbm, "unit": "GB/s", "frac": round(gbs / hbm, 4), "iterations": iters,
                              "ms": round(ms_e, 4),
                              "nonzero_tile_pairs": round(pf, 4),
                              "note": f"{enforce_bytes(N, iters, pf) / max(iters, 1) / 1e6:.1f} MB per iteration on "
                                      f"average, L2-resident at N={N}"},
        "gebhart": {"kernel": "gemm_kernel (tcgen05) + helpers", "bound": "tensor", "achieved": round(tf, 3),
                    "peak": bf, "unit": "TFLOP/s", "frac": round(tf / bf, 5), "sweeps": sweeps, "ms": round(ms_r, 4),
                    "note": f"N={N}: launch- and latency-bound ({SOLVE_PRECISION} peak = bf16 peak)"},
    }


def sided_stage(api, torch, ctx, flush, stream, synth, peaks):
    """Two-faced nodes (Sec. 5.2.4-5.2.5, App. C) on the plates mesh, outside the timed
    step: side-resolved MCRT at the full budget (1e6 rays per side, 1.024e9 rays), then the
    node view factors / view fractions and the node couplings of the 1,024 sides (HBM
    bound: 32 B read per node pair, 40 B written by the view factors and fractions, 24 B
    by the couplings)."""
    w = synth.workload("plates_sided")
    m = w["mesh"]
    N = m.n_faces
    mesh = api.Mesh.from_synth(ctx, m)
    counts = torch.zeros((2 * N, 2 * N + 1), dtype=torch.int64, device="cuda")
    api.trace_sided(ctx, mesh, w["rays"], w["seed"], counts=counts)        # warm-up
    t_tr = []
    for _ in range(3):
        counts.zero_()
        flush()
        t_tr.append(time_region(torch, lambda: api.trace_sided(ctx, mesh, w["rays"], w["seed"], counts=counts),
                                stream))
    rays = int(w["rays"].sum())
    F2 = api.counts_to_F(ctx, counts, torch.as_tensor(w["rays"], device="cuda"))
    C = torch.full((N,), 2, dtype=torch.int32, device="cuda")
    eps2 = torch.as_tensor(w["eps"][0], device="cuda")
    S = torch.as_tensor(mesh.face_areas(), device="cuda")
    api.node_view_factors(ctx, F2, C)
    api.node_couplings(ctx, F2, eps2, S, C)
    t_vf, t_gr = [], []
    for _ in range(5):
        flush()
        t_vf.append(time_region(torch, lambda: api.node_view_factors(ctx, F2, C), stream))
        flush()
        t_gr.append(time_region(torch, lambda: api.node_couplings(ctx, F2, eps2, S, C), stream))
    ms_tr, ms_vf, ms_gr = (statistics.median(t) for t in (t_tr, t_vf, t_gr))
    pairs = N * (N + 1)
    hbm = float(peaks.get("hbm_gbs", 6800.0))
    gb_vf = 72.0 * pairs / (ms_vf * 1e-3) / 1e9
    gb_gr = 56.0 * pairs / (ms_gr * 1e-3) / 1e9
    mesh.close()
    return {"workload": "plates mesh, both sides of the 512 sub-faces radiating (1,024 sides), 1e6 rays per side",
            "rays": rays, "trace_ms": round(ms_tr, 3), "rays_per_s": rays / (ms_tr * 1e-3),
            "node_view_factors": {"ms": round(ms_vf, 4), "bound": "hbm", "achieved": round(gb_vf, 1), "unit": "GB/s",
                                  "frac": round(gb_vf / hbm, 4)},
            "node_couplings": {"ms": round(ms_gr, 4), "bound": "hbm", "achieved": round(gb_gr, 1), "unit": "GB/s",
                               "frac": round(gb_gr / hbm, 4)},
            "note": "host-timed calls include their launch and one status read-back; 8.4 MB of side factors "
                    "at N=512 stay L2-sized, so these are latency-bound"}


def run_e2e(args, api, torch, pipe, stream):
    """The same metric through the public API from host buffers: every step builds the mesh
    and its BVH again from the host arrays (device builder), copies the ray budget, the 16
    eps / rho sets and the heat loads in from pinned memory, runs the path and reads F, the
    REFs of every set, the temperatures and both gradients back into pinned memory."""
    w = pipe.w
    m = w["mesh"]
    pin = lambda a: torch.as_tensor(np.ascontiguousarray(a)).pin_memory()  # noqa: E731
    host_in = {"rays": pin(w["rays"]), "eps": pin(w["eps"]), "rho": pin(w["rho"]), "Q": pin(w["Q"])}
    N, S = pipe.N, pipe.S
    h2d = (m.verts.nbytes + m.tris.nbytes + m.tri_face.nbytes + N * 8
           + sum(t.numel() * t.element_size() for t in host_in.values()))
    f64 = dict(dtype=torch.float64)
    outs = {"F_it": torch.empty((N, N + 1), **f64).pin_memory(), "B": torch.empty((S, N, N + 1), **f64).pin_memory(),
            "T": torch.empty((S, N), **f64).pin_memory(), "deps_B": torch.empty((S, N), **f64).pin_memory(),
            "deps_T": torch.empty((S, N), **f64).pin_memory(), "drho": torch.empty((S, N), **f64).pin_memory()}
    d2h = sum(t.numel() * t.element_size() for t in outs.values())

    def one():
        pipe.load_inputs(host_in)
        pipe.step()
        for k in outs:
            outs[k].copy_(getattr(pipe, k), non_blocking=True)

    one()
    torch.cuda.synchronize()
    n = max(1, min(args.steps, 3))
    vals = [time_region(torch, one, stream) for _ in range(n)]
    ms = statistics.mean(vals)
    return {"value": float(pipe.rays_per_step) / (ms * 1e-3), "unit": "rays/s", "ms_per_step": round(ms, 3),
            "steps": n, "h2d_bytes_per_step": int(h2d), "d2h_bytes_per_step": int(d2h),
            "note": "mesh + BVH rebuilt from host arrays (device builder) and face areas recomputed every step"}


# ------------------------------------------------------------------ CPU oracle
def oracle_inputs(w, threads=0):
    """A complete F for the oracle's downstream steps (500 rays per face, not timed): the
    timed pieces' costs do not depend on the values."""
    from oracle import mcrt
    m = w["mesh"]
    light = np.full(m.n_faces, 500, np.int64)
    c = mcrt.trace_counts(m.verts, m.tris, m.tri_face, m.n_faces, light, w["seed"], use_bvh=True, threads=threads)
    return mcrt.view_factors(c, light), mcrt.face_areas(m.verts, m.tris, m.tri_face, m.n_faces)


def oracle_sample(w, F, A, threads, name=HEADLINE):
    """One bounded CPU sample of the step, extrapolated to the whole step:
      MCRT   64 faces spread over the mesh (4 per host core at 16 cores), a quarter of each
             face's ray budget, C oracle with its own BVH on all cores -> x (total rays /
             sampled rays);
      enforcement  two iterations of the oracle's fp64 enforcer on the leading 5,120 faces
             (their 5,120 x 5,121 block, 210 MB: larger than the host's caches) -> x
             (iterations / 2) x (entries of the whole matrix / entries of the block);
      solves one LU-based solve of K^T for 128 rows of B (the oracle's gebhart_rows,
             LAPACK on all cores) -> its fp64 rate applied to the LU-equivalent flops of
             the step's solves (REFs, balances and both adjoints of every set).
    Returns (rays per second of the extrapolated step, details)."""
    from oracle import enforce as E
    from oracle import gebhart as G
    from oracle import mcrt
    m = w["mesh"]
    N = m.n_faces
    S = w["eps"].shape[0]
    rows = np.unique(np.linspace(0, N - 1, min(64, N)).astype(np.int64))
    budget = np.zeros(N, np.int64)
    budget[rows] = np.maximum(w["rays"][rows] // 4, 1)
    t0 = time.perf_counter()
    mcrt.trace_counts(m.verts, m.tris, m.tri_face, N, budget, w["seed"], use_bvh=True, threads=threads, faces=rows)
    t_trace = time.perf_counter() - t0
    ns = min(N, 5120)
    Fs = np.ascontiguousarray(np.concatenate([F[:ns, :ns], F[:ns, N:]], axis=1))
    t1 = time.perf_counter()
    E.iterative(Fs, A[:ns], tol=1e-12, maxit=2)
    t_enf = (time.perf_counter() - t1) / 2.0 * (N * (N + 1)) / (ns * (ns + 1))
    del Fs
    nr = min(128, N)
    t2 = time.perf_counter()
    G.gebhart_rows(F, w["eps"][0], w["rho"][0], range(0, N, max(1, N // nr)))
    t_rows = time.perf_counter() - t2
    rows_flops = 2.0 / 3.0 * N ** 3 + 2.0 * N * N * nr + 2.0 * nr * N * (N + 1)
    rate = rows_flops / t_rows
    sampled = int(budget.sum())
    total = int(w["rays"].sum())
    iters = ENFORCE_ITERS.get(name, 30)
    solve_flops = lu_equivalent_flops(N, S, 0)
    t_step = t_trace * total / sampled + t_enf * iters + solve_flops / rate
    detail = {"rays_sampled": sampled, "trace_s": round(t_trace, 3), "enforce_block": ns,
              "enforce_s_per_iteration": round(t_enf, 3),
              "enforce_iterations": iters, "lu_solve_s": round(t_rows, 3), "fp64_gflops": round(rate / 1e9, 1),
              "measured_s": round(time.perf_counter() - t0, 2), "extrapolated_step_s": round(t_step, 1)}
    return total / t_step, detail


def sample_text(d, w, cores):
    return (f"MCRT of 64 faces spread over the mesh at 1/4 of their budgets ({d['rays_sampled']:.3g} of "
            f"{w['rays'].sum():.3g} rays, C oracle with its own BVH, {cores} OpenMP threads) x ray count; 2 fp64 "
            f"enforcer iterations on the leading {d['enforce_block']} faces x entry count x "
            f"{d['enforce_iterations']} iterations; one LAPACK LU solve of K^T for 128 REF rows "
            f"({d['fp64_gflops']} GFLOP/s) applied to the LU-equivalent flops of the 16 sets' REFs, balances and "
            f"adjoints; {d['measured_s']} s measured, step extrapolated to {d['extrapolated_step_s']} s")


def cpu_baseline(w):
    from oracle import mcrt
    cores = len(os.sched_getaffinity(0))
    F, A = oracle_inputs(w, cores)
    value, d = oracle_sample(w, F, A, cores)
    return {"value": value, "unit": "rays/s", "cores": cores, "kind": "oracle", "sample": sample_text(d, w, cores),
            "detail": d, "threads_seen": mcrt.max_threads()}


def run_reference(args):
    rank = int(os.environ.get("RANK", 0))
    if rank != 0:
        return None
    w = load_workload(HEADLINE)
    cores = len(os.sched_getaffinity(0))
    F, A = oracle_inputs(w, cores)
    for _ in range(max(args.warmup, 0)):
        oracle_sample(w, F, A, cores)
    vals, details = [], []
    t0 = time.perf_counter()
    for _ in range(args.steps):
        v, d = oracle_sample(w, F, A, cores)
        vals.append(v)
        details.append(d)
    wall = time.perf_counter() - t0
    value = statistics.mean(vals)
    ms = float(w["rays"].sum()) / value * 1e3
    d = details[-1]
    return {"impl": "reference", "metric": METRIC, "value": value, "unit": "rays/s", "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(ms, 3),
            "ms_per_step_basis": "extrapolated from the bounded sample (see cpu_baseline.sample)",
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32 rays, i64 tallies, f64",
            "data": "synthetic",
            "config": {"workload": WORKLOADS[HEADLINE], "faces": w["mesh"].n_faces,
                       "triangles": int(w["mesh"].n_tris), "sets": int(w["eps"].shape[0]),
                       "rays_per_step": int(w["rays"].sum())},
            "wall_s_timed_samples": round(wall, 2),
            "cpu_baseline": {"value": value, "unit": "rays/s", "cores": cores, "kind": "oracle",
                             "sample": sample_text(d, w, cores)},
            "e2e": {"value": value, "unit": "rays/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}


def factorisation_comparison(torch, api, ctx, ev, name, F, eps, rho):
    """The factorisation the REF solve makes (the Newton-Schulz inverse M of K on tcgen05,
    fp16) and the per-sweep application of it (one correction product D = M R, n x n x (n+1)),
    beside an LU of the same K (cuSOLVER getrf through torch.linalg.lu_factor) and its
    per-sweep application (getrs with the n+1 right-hand sides, torch.linalg.lu_solve), in
    fp32 and fp64. Every figure is measured with CUDA events; the two totals are
    factorisation + sweeps x application, the sweeps being the ones the solve took."""
    n = F.shape[0]
    dev = F.device
    api.kernel_timer(ctx, True)
    _, sweeps, _ = api.gebhart(ctx, F, eps[:1], rho[:1], SOLVE_PRECISION, tol=SOLVE_TOL)
    api.kernel_timer(ctx, False)
    fa = api.kernel_timer_read(ctx, "factor")
    np_ = (n + 127) // 128 * 128
    dt16 = torch.float16 if SOLVE_PRECISION == "fp16" else torch.bfloat16
    Mi = torch.randn(np_, np_, device=dev).to(dt16)
    Rt = torch.randn(n + 1, np_, device=dev).to(dt16)
    C = torch.empty(np_, n + 1, dtype=torch.float32, device=dev)
    ms_corr = ev(lambda: api.tc_gemm(ctx, Mi, Rt, C), 5)
    del Mi, Rt, C
    res = {"workload": name, "n": n, "sweeps": int(sweeps),
           "newton_schulz": {"factor_ms": round(fa["ms"], 3), "apply_ms": round(ms_corr, 3),
                             "total_ms": round(fa["ms"] + sweeps * ms_corr, 3)}}
    Kd = torch.eye(n, dtype=torch.float64, device=dev) - F[:, :n] * rho[0][None, :]
    Ed = F.clone()
    Ed[:, :n] *= eps[0][None, :]
    prev = torch.backends.cuda.preferred_linalg_library()
    torch.backends.cuda.preferred_linalg_library("cusolver")
    try:
        for dt, key in ((torch.float32, "cusolver_lu_fp32"), (torch.float64, "cusolver_lu_fp64")):
            Kt, Et = Kd.to(dt), Ed.to(dt)
            try:
                box = {}
                ms_f = ev(lambda: box.__setitem__("lu", torch.linalg.lu_factor(Kt)), 3)
                LU, piv = box["lu"]
                ms_s = ev(lambda: torch.linalg.lu_solve(LU, piv, Et), 3)
                res[key] = {"factor_ms": round(ms_f, 3), "apply_ms": round(ms_s, 3),
                            "total_ms": round(ms_f + sweeps * ms_s, 3)}
                del LU, piv, box
            except RuntimeError as exc:
                res[key] = str(exc).splitlines()[0][:100]
            del Kt, Et
    finally:
        torch.backends.cuda.preferred_linalg_library(prev)
    del Kd, Ed
    return res


def solve_scaling(args):
    """REF solve + adjoint at the three solve sizes of the workloads (enforced MCRT F at a
    reduced ray budget), ours against torch.linalg.solve float64, and the tcgen05 GEMM
    rates the solves are built on. CUDA events, after one warm-up call each."""
    import torch
    import synth
    from paper_2511_04277_gb300 import api
    ctx = api.Context(0)
    dev = torch.device("cuda:0")

    def ev(fn, reps):
        fn()
        torch.cuda.synchronize()
        return statistics.median(time_region(torch, fn, torch.cuda.current_stream()) for _ in range(reps))

    out = {"kind": "solve_scaling", "precision": SOLVE_PRECISION, "gemm": [], "enforce": [], "solves": [],
           "factorisations": []}
    peaks = load_peaks()
    g = torch.Generator().manual_seed(0)
    for M, N, K in ((4096, 4096, 4096), (10240, 10240, 10240)):
        A = torch.randn(M, K, generator=g).to(torch.bfloat16).to(dev)
        B = torch.randn(N, K, generator=g).to(torch.bfloat16).to(dev)
        C = torch.zeros(M, N, dtype=torch.float32, device=dev)
        ms = ev(lambda: api.tc_gemm(ctx, A, B, C), 5)
        out["gemm"].append({"op": "bf16 A B^T -> fp32", "M": M, "N": N, "K": K, "ms": round(ms, 3),
                            "tflops": round(2 * M * N * K / ms / 1e9, 1)})
        del A, B, C
    for M, N, np_, levels in ((10240, 10241, 10240, 5),):
        # the refinement's exact level product: integer operands |x| <= 128 in bf16
        A = torch.randint(-128, 129, (M, 5 * np_), generator=g).to(torch.bfloat16).to(dev)
        B = torch.randint(-128, 129, (N, np_), generator=g).to(torch.bfloat16).to(dev)
        ms = ev(lambda: api.tc_gemm_exact(ctx, A, B, levels), 3)
        out["gemm"].append({"op": "rg_tc_gemm_exact: exact integer level product (5 levels), int32 sums, "
                                  "including the copy of the level sums to the caller's layout", "M": M, "N": N,
                            "K": levels * np_, "ms": round(ms, 3),
                            "tflops": round(2 * M * N * levels * np_ / ms / 1e9, 1)})
        del A, B
    torch.cuda.empty_cache()
    for name, scale, S in (("plates", 0.02, 1), ("small_sat", 0.02, 1), ("spacecraft", 0.01, 16)):
        w = synth.workload(name, rays_scale=scale)
        mesh = api.Mesh.from_synth(ctx, w["mesh"])
        rays = torch.as_tensor(w["rays"], device=dev)
        F = api.counts_to_F(ctx, api.trace(ctx, mesh, w["rays"], w["seed"]), rays)
        areas = torch.as_tensor(mesh.face_areas(), device=dev)
        n = F.shape[0]
        # the iterative enforcer on this F: HBM bound above N = 2,048 (16 B per entry in the
        # first iteration, per stored entry of the upper triangle after it), L2 sized below
        F0 = F.clone()
        t_e, iters = [], 0
        for _ in range(4):
            F.copy_(F0)
            torch.cuda.synchronize()
            box = {}
            t = time_region(torch, lambda: box.__setitem__("it", api.enforce_iterative(ctx, F, areas, tol=1e-12)),
                            torch.cuda.current_stream())
            t_e.append(t)
            iters = box["it"]
        ms_e = statistics.median(t_e[1:])
        pf = nonzero_pair_fraction(F)
        gbs = enforce_bytes(n, iters, pf) / (ms_e * 1e-3) / 1e9
        hbm = float(peaks.get("hbm_gbs", 6800.0))
        # the weighted enforcer (fractional-variance kappa, Eq. 3.23-3.25): kappa once, then
        # the iterations with per-pair weights (24 B per entry per iteration)
        K = api.kappa(ctx, rays, areas, "fractional_variance", F=F0)
        t_k, iters_k = [], 0
        for _ in range(3):
            F.copy_(F0)
            torch.cuda.synchronize()
            box = {}
            t_k.append(time_region(torch, lambda: box.__setitem__("it", api.enforce_iterative_kappa(
                ctx, F, areas, api.kappa(ctx, rays, areas, "fractional_variance", F=F0, K=K), tol=1e-12)),
                torch.cuda.current_stream()))
            iters_k = box["it"]
        ms_k = statistics.median(t_k[1:])
        del K
        out["enforce"].append({"workload": name, "n": n, "iterations": iters, "ms": round(ms_e, 3),
                               "ms_per_iteration": round(ms_e / iters, 4), "achieved_gbs": round(gbs, 1),
                               "peak_gbs": hbm, "frac": round(gbs / hbm, 4),
                               "bytes_per_iteration": round(enforce_bytes(n, iters, pf) / max(iters, 1)),
                               "nonzero_tile_pairs": round(pf, 4),
                               "bound": "hbm (whole call: also F -> eta and back, 28 B per entry once)",
                               "weighted": {"kappa": "fractional variance", "iterations": iters_k,
                                            "ms": round(ms_k, 3), "ms_per_iteration": round(ms_k / iters_k, 4)}})
        del F0
        eps = torch.as_tensor(w["eps"][:S], device=dev)
        rho = torch.as_tensor(w["rho"][:S], device=dev)
        reps = 1 if n > 4096 else 5
        box = {}
        store = api.gebhart_factor_store(n, S, SOLVE_PRECISION)
        ms_f = ev(lambda: box.__setitem__("B", api.gebhart(ctx, F, eps, rho, SOLVE_PRECISION, tol=SOLVE_TOL,
                                                           factors=store)), reps)
        B, sweeps, res = box["B"]
        dB = torch.ones_like(B)
        ms_a = ev(lambda: api.gebhart_adjoint(ctx, F, eps, rho, B, dB, SOLVE_PRECISION, tol=SOLVE_TOL,
                                              factors=store), reps)
        del dB, store
        Fn = F[:, :n]

        def fp64_pair():
            K = torch.eye(n, dtype=torch.float64, device=dev) - Fn * rho[0][None, :]
            E = F.clone()
            E[:, :n] *= eps[0][None, :]
            X = torch.linalg.solve(K, E)
            return torch.linalg.solve(K.T, torch.ones_like(X))
        try:
            ms64 = ev(fp64_pair, reps) * S
            Kd = torch.eye(n, dtype=torch.float64, device=dev) - Fn * rho[0][None, :]
            Ed = F.clone()
            Ed[:, :n] *= eps[0][None, :]
            B64 = torch.linalg.solve(Kd, Ed)
            err = float(((B[0] - B64).abs().amax(dim=-1) / B64.abs().amax(dim=-1)).max())
            del Kd, Ed, B64
        except RuntimeError as exc:
            ms64, err = None, str(exc).splitlines()[0][:120]
        out["factorisations"].append(factorisation_comparison(torch, api, ctx, ev, name, F, eps, rho))
        out["solves"].append({"workload": name, "n": n, "sets": S, "ours_ms": round(ms_f + ms_a, 2),
                              "refs_ms": round(ms_f, 2), "adjoint_ms": round(ms_a, 2), "sweeps": sweeps,
                              "residual": res, "fp64_ms": None if ms64 is None else round(ms64, 2),
                              "fp64_basis": "one set timed" + (f", x{S}" if S > 1 else ""),
                              "speedup": None if ms64 is None else round(ms64 / (ms_f + ms_a), 2),
                              "err_B_rownorm_set0": err})
        del B, F
        torch.cuda.empty_cache()
    ctx.close()
    return out


def bvh_build(args):
    """The host and the device BVH builder (the same tree): build time (median of 3, host
    wall clock around the call, uploads included) and the trace rate on each tree
    (FMA-free, the library's schedule choice), on the small-satellite and spacecraft
    meshes."""
    import torch
    import synth
    from paper_2511_04277_gb300 import api
    ctx = api.Context(0)
    stream = torch.cuda.current_stream()
    rows = []
    for name, scale in (("small_sat", 1.0), ("spacecraft", 0.1)):
        w = synth.workload(name, rays_scale=scale)
        m = w["mesh"]
        out = {"workload": name, "triangles": m.n_tris, "rays": int(w["rays"].sum())}
        for label, kw in (("host", {}), ("device", {"gpu_bvh": True})):
            api.Mesh.from_synth(ctx, m, **kw).close()
            times = []
            for _ in range(3):
                torch.cuda.synchronize()
                t0 = time.perf_counter()
                mesh = api.Mesh.from_synth(ctx, m, **kw)
                torch.cuda.synchronize()
                times.append(1e3 * (time.perf_counter() - t0))
                if _ < 2:
                    mesh.close()
            counts = torch.zeros((m.n_faces, m.n_faces + 1), dtype=torch.int64, device="cuda")
            api.trace(ctx, mesh, w["rays"], w["seed"], counts=counts)
            t_tr = []
            for _ in range(3):
                counts.zero_()
                t_tr.append(time_region(torch, lambda: api.trace(ctx, mesh, w["rays"], w["seed"], counts=counts),
                                        stream))
            info = mesh.info()
            _, tst = api.trace_stats(ctx, mesh, w["rays"], w["seed"])
            out[label] = {"build_ms": round(statistics.median(times), 2), "depth": info["bvh_depth"],
                          "box_tests_per_ray": round(tst["box_tests"] / tst["rays"], 3),
                          "tri_tests_per_ray": round(tst["tri_tests"] / tst["rays"], 3),
                          "nodes": info["bvh_nodes"], "sah_visits": round(info["sah_visits"], 3),
                          "refill": info["refill"], "trace_ms": round(statistics.median(t_tr), 3),
                          "rays_per_s": out["rays"] / (statistics.median(t_tr) * 1e-3)}
            mesh.close()
        rows.append(out)
    ctx.close()
    return {"kind": "bvh_build", "meshes": rows}


def enforce_once(n, iters):
    """One iterative enforcement of a seeded n x (n+1) matrix (rows summing to about 0.75,
    areas U[0.5, 2]) stopped after `iters` iterations: the small case of the enforcer's
    ncu captures (the tolerance is out of reach, so the call reports RG_ERR_NOT_CONVERGED
    after `iters` iterations, which is expected here)."""
    import torch
    from paper_2511_04277_gb300 import api
    from paper_2511_04277_gb300._native import RadgebError
    ctx = api.Context(0)
    g = torch.Generator(device="cuda").manual_seed(0)
    F = torch.rand((n, n + 1), dtype=torch.float64, device="cuda", generator=g) * (0.5 / n)
    F[:, n] = 0.5
    A = torch.rand(n, dtype=torch.float64, device="cuda", generator=g) * 1.5 + 0.5
    try:
        api.enforce_iterative(ctx, F, A, tol=1e-300, maxit=iters)
    except RadgebError as exc:
        if exc.code != "RG_ERR_NOT_CONVERGED":
            raise
    torch.cuda.synchronize()
    print(json.dumps({"kind": "enforce_once", "n": n, "iterations": iters}), flush=True)
    ctx.close()


def reflect_rates(args):
    """REFs by the MCRT reflection walk (rg_trace_reflect): paths per second on the plates
    (1e6 paths per sub-face, eps ~ U[0.1, 0.9], rho = 1 - eps) and the closed cube (1e6
    per face, eps = 0.8, rho = 0.2), with the mean bounces per path."""
    import torch
    import synth
    from paper_2511_04277_gb300 import api
    ctx = api.Context(0)
    stream = torch.cuda.current_stream()
    rows = []
    for name in ("plates", "cube"):
        w = synth.workload(name, rays_scale=1.0 if name == "plates" else 10.0)
        m = w["mesh"]
        mesh = api.Mesh.from_synth(ctx, m)
        eps, rho = w["eps"][0], w["rho"][0]
        counts = torch.zeros((m.n_faces, m.n_faces + 1), dtype=torch.int64, device="cuda")
        _, st = api.trace_reflect(ctx, mesh, w["rays"], eps, rho, w["seed"], counts=counts)
        ts = []
        for _ in range(3):
            counts.zero_()
            ts.append(time_region(torch, lambda: api.trace_reflect(ctx, mesh, w["rays"], eps, rho, w["seed"],
                                                                   counts=counts), stream))
        ms = statistics.median(ts)
        rows.append({"workload": name, "paths": st["rays"], "hits_per_path": round(st["hits"] / st["rays"], 3),
                     "ms": round(ms, 3), "paths_per_s": st["rays"] / (ms * 1e-3)})
        mesh.close()
    ctx.close()
    return {"kind": "reflect", "rows": rows}


def trace_once(scale, mesh_name="plates", sided=False):
    """One trace launch at `scale` x the workload's ray budget (FMA-free): the small case of
    the trace kernel's ncu captures."""
    import torch
    import synth
    from paper_2511_04277_gb300 import api
    ctx = api.Context(0)
    w = synth.workload("plates_sided" if sided else mesh_name, rays_scale=scale)
    mesh = api.Mesh.from_synth(ctx, w["mesh"])
    tr = api.trace_sided if sided else api.trace
    c = tr(ctx, mesh, w["rays"], w["seed"], fma_free=True)
    torch.cuda.synchronize()
    print(json.dumps({"kind": "trace_once", "mesh": w["mesh"].name, "rays": int(c.sum()), "bvh": mesh.info()}),
          flush=True)
    mesh.close()
    ctx.close()


class _RandomSystem:
    """A seeded random open system of n faces with the attributes of Pipeline that the
    solve stages use (no mesh)."""

    def __init__(self, ctx, n, n_sets, device, band=0):
        import torch
        import synth
        from paper_2511_04277_gb300 import api
        self.api, self.ctx, self.N, self.S = api, ctx, n, n_sets
        g = torch.Generator(device=device).manual_seed(0)
        F = torch.rand((n, n + 1), dtype=torch.float64, device=device, generator=g) * (1.5 / n)
        if band > 0:  # non-zero only within `band` of the diagonal (most 256 x 64 blocks zero)
            i = torch.arange(n, device=device)
            F[:, :n] *= ((i[:, None] - i[None, :]).abs() < band).double() * (n / (2.0 * band))
        F.diagonal()[:] = 0.0
        F[:, n] = 0.0
        F[:, n] = 1.0 - F.sum(dim=1)
        self.areas = torch.rand(n, dtype=torch.float64, device=device, generator=g) * 1.5 + 0.5
        self.F_it = F
        api.enforce_iterative(ctx, self.F_it, self.areas, tol=1e-12)
        eps, rho = synth.optical_sets(n, n_sets, 0.05, 0.9, seed=10)
        self.eps = torch.as_tensor(eps, device=device)
        self.rho = torch.as_tensor(rho, device=device)
        self.Q = torch.as_tensor(synth.heat_loads(n, seed=3), device=device)
        self.Qs = self.Q.expand(n_sets, n).contiguous()
        self.dT = torch.ones((n_sets, n), dtype=torch.float64, device=device)
        self.ones = torch.ones(n, dtype=torch.float64, device=device)
        f64 = dict(dtype=torch.float64, device=device)
        self.B = torch.empty((n_sets, n, n + 1), **f64)
        self.factors = api.gebhart_factor_store(n, n_sets, SOLVE_PRECISION, device=torch.device(device).index or 0)
        self.dB_a = torch.empty((n_sets, 2, n), **f64)
        self.dB_b = torch.empty((n_sets, 2, n + 1), **f64)
        self.T = torch.empty((n_sets, n), **f64)
        self.deps_T = torch.empty((n_sets, n), **f64)

    refs = Pipeline.refs
    thermal = Pipeline.thermal
    adjoint = Pipeline.adjoint


def solve_once(n_sets, n=None, band=0):
    """The spacecraft solves once for `n_sets` eps / rho sets on an enforced 1e7-ray F (or
    on a seeded random n-face system, banded when band > 0): REFs, steady temperatures and
    their adjoint per set, the REF adjoint (the case the solver's ncu captures use)."""
    import torch
    from paper_2511_04277_gb300 import api
    ctx = api.Context(0)
    if n is None:
        w = load_workload("spacecraft", rays_scale=0.01)
        w["eps"], w["rho"] = w["eps"][:n_sets], w["rho"][:n_sets]
        p = Pipeline(ctx, w, torch.device("cuda:0"))
        p.mcrt()
        p.enforce()
    else:
        p = _RandomSystem(ctx, n, n_sets, torch.device("cuda:0"), band=band)
    torch.cuda.synchronize()
    api.kernel_timer(ctx, True)
    t = time_region(torch, lambda: (p.refs(), p.thermal(), p.adjoint()), torch.cuda.current_stream())
    timer = {k: api.kernel_timer_read(ctx, k) for k in ("residual_gemm", "gemm", "factor")}
    api.kernel_timer(ctx, False)
    print(json.dumps({"kind": "solve_once", "n": p.N, "sets": n_sets, "ms": round(t, 2), "sweeps": p.sweeps,
                      "residual": p.resid, "closure_B": float((p.B.sum(dim=-1) - 1.0).abs().max()),
                      "kernel_timer": timer}), flush=True)
    if n is None:
        p.mesh.close()
    ctx.close()


def main():
    args = parse()
    if args.trace_once is not None:
        trace_once(args.trace_once, args.mesh, args.sided)
        return
    if args.solve_once is not None:
        solve_once(args.solve_once, args.solve_n, args.solve_band)
        return
    if args.solve_scaling:
        print(json.dumps(solve_scaling(args)), flush=True)
        return
    if args.enforce_once is not None:
        enforce_once(args.enforce_once[0], args.enforce_once[1])
        return
    if args.bvh_build:
        print(json.dumps(bvh_build(args)), flush=True)
        return
    if args.reflect:
        print(json.dumps(reflect_rates(args)), flush=True)
        return
    out = run_reference(args) if args.impl == "reference" else run_ours(args)
    if out is not None:
        print(json.dumps(out), flush=True)


if __name__ == "__main__":
    main()
