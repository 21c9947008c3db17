"""The allocation-free enforcer entry point against the allocating one.

rg_enforce_iterative_noalloc exists for callers that must not allocate device memory
when they call in (software that plans all of its memory up front, or a host that owns
the device's memory pool). Its scratch is a fixed device array inside the library that
every call reuses, so the test makes two calls in a row, of different sizes, and checks
each against rg_enforce_iterative on the same input.
"""
import ctypes

import numpy as np
import pytest
import torch

from oracle import enforce as E
from paper_2511_04277_gb300 import _native, api

pytestmark = pytest.mark.gpu

TOL = 1e-12


def _random_F(N, rng, zeros=0.2):
    F = rng.random((N, N + 1))
    F[rng.random((N, N + 1)) < zeros] = 0.0
    np.fill_diagonal(F[:, :N], 0.0)
    F[:, N] += 0.05
    return F / F.sum(axis=1, keepdims=True)


def _noalloc(F, A):
    lib = _native.load()
    it = ctypes.c_int32(0)
    st = lib.rg_enforce_iterative_noalloc(F.shape[0], ctypes.c_void_p(A.data_ptr()), ctypes.c_void_p(F.data_ptr()),
                                          TOL, 10000, ctypes.byref(it),
                                          ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
    return st, it.value


# Two calls in a row per case. The first order fills the scratch's per-tile row sums
# completely (n = 4096 takes 64-wide tiles: 64 tiles x 4096 rows is the whole region) and
# then checks that a small call is unaffected by what that call left behind; the second
# starts just above the tile-width switch (n = 2049, 64-wide tiles) before a 32-wide one.
@pytest.mark.parametrize("sizes", [(4096, 300), (2049, 1000)], ids=["4096-then-300", "2049-then-1000"])
def test_noalloc_enforcer_matches_allocating_entry_point_on_two_calls(rg_ctx, sizes):
    rng = np.random.default_rng(42)
    for N in sizes:
        F = _random_F(N, rng)
        A = rng.uniform(0.5, 2.0, N)
        A_d = torch.as_tensor(A, device="cuda")
        F_ref = torch.as_tensor(F, device="cuda")
        it_ref = api.enforce_iterative(rg_ctx, F_ref, A_d, tol=TOL)
        F_na = torch.as_tensor(F, device="cuda")
        st, it = _noalloc(F_na, A_d)
        torch.cuda.synchronize()
        assert st == 0
        assert it == it_ref
        got, ref = F_na.cpu().numpy(), F_ref.cpu().numpy()
        assert np.abs(got - ref).max() <= 1e-12
        Fo, _, _ = E.iterative(F, A, tol=TOL)
        assert np.abs(got - Fo).max() <= 1e-12


def test_noalloc_enforcer_rejects_sizes_beyond_its_scratch(rg_ctx):
    tiny = torch.zeros(8, dtype=torch.float64, device="cuda")
    st, _ = _noalloc(torch.zeros((4097, 1), dtype=torch.float64, device="cuda").expand(4097, 4098), tiny)
    assert _native.STATUS[st] == "RG_ERR_UNSUPPORTED"
