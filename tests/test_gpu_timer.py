"""The context's kernel timer (rg_kernel_timer / rg_kernel_timer_read): which launches it
records, per class, and that it records nothing while it is off."""
import numpy as np
import pytest
import torch

from paper_2511_04277_gb300 import api

pytestmark = pytest.mark.gpu


def _system(N, S, seed):
    rng = np.random.default_rng(seed)
    A = rng.uniform(0.5, 2.0, N)
    G = rng.random((N, N)) * (rng.random((N, N)) < 0.3)
    G = (G + G.T) / (2 * N) * 0.8
    np.fill_diagonal(G, 0.0)
    F = np.concatenate([G, (A - G.sum(axis=1))[:, None]], axis=1) / A[:, None]
    eps = rng.uniform(0.2, 0.9, (S, N))
    dev = lambda x: torch.as_tensor(x, dtype=torch.float64, device="cuda")
    return dev(F), dev(eps), dev(1.0 - eps), dev(A)


def test_timer_records_each_class_of_a_solve_and_nothing_while_off(rg_ctx):
    F, eps, rho, A = _system(300, 2, 3)
    api.gebhart(rg_ctx, F, eps, rho, "fp16", tol=1e-10)  # warm: kernels loaded, workspace sized
    api.kernel_timer(rg_ctx, True)
    _, sweeps, _ = api.gebhart(rg_ctx, F, eps, rho, "fp16", tol=1e-10)
    Fe = F.clone()
    api.enforce_iterative(rg_ctx, Fe, A, tol=1e-12)
    api.kernel_timer(rg_ctx, False)
    fac = api.kernel_timer_read(rg_ctx, "factor")
    gemm = api.kernel_timer_read(rg_ctx, "gemm")
    res = api.kernel_timer_read(rg_ctx, "residual_gemm")
    enf = api.kernel_timer_read(rg_ctx, "enforce")
    # one factorisation region per set, each holding at least one Newton-Schulz GEMM pair
    # unless the start iterate was already accurate enough
    assert fac["launches"] == 2 and fac["ms"] > 0.0
    assert fac["flops"] == 0.0 and fac["alg_flops"] == 0.0
    assert gemm["launches"] >= 2 and gemm["ms"] > 0.0 and gemm["flops"] == gemm["alg_flops"] > 0.0
    # at least one exact level product per sweep of the slowest set; its executed flops
    # count the levels each launch ran (0 for a speculative launch that skipped itself)
    assert res["launches"] >= sweeps and res["flops"] > 0.0 and res["alg_flops"] > 0.0
    assert enf["launches"] == 1 and enf["ms"] > 0.0 and enf["flops"] == 0.0
    # the timer is off: a further solve leaves the records as they were
    api.gebhart(rg_ctx, F, eps, rho, "fp16", tol=1e-10)
    again = api.kernel_timer_read(rg_ctx, "factor")
    assert again["launches"] == fac["launches"] and again["ms"] == fac["ms"]
    # switching it on clears the records
    api.kernel_timer(rg_ctx, True)
    api.kernel_timer(rg_ctx, False)
    assert api.kernel_timer_read(rg_ctx, "gemm")["launches"] == 0


def test_timer_rejects_an_unknown_class(rg_ctx):
    from paper_2511_04277_gb300._native import RadgebError
    import ctypes
    n, ms = ctypes.c_int64(), ctypes.c_double()
    st = rg_ctx.lib.rg_kernel_timer_read(rg_ctx.handle, 5, ctypes.byref(n), ctypes.byref(ms), None, None)
    assert st != 0
    with pytest.raises(RadgebError):
        rg_ctx.check(st, "rg_kernel_timer_read")
