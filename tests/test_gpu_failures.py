"""Failure detection without a GPU fault: the bounded device waits run out against a
flag that nothing sets and come back as a status, the context stays usable, and
non-finite inputs are reported instead of propagated silently."""
import numpy as np
import pytest
import torch

from oracle import gebhart as G
from paper_2511_04277_gb300 import api

pytestmark = pytest.mark.gpu


def _dev(x):
    return torch.as_tensor(np.ascontiguousarray(x), dtype=torch.float64).cuda()


def _small_system(N=40, seed=3):
    rng = np.random.default_rng(seed)
    A = rng.uniform(0.5, 2.0, N)
    S = rng.random((N, N)) * 0.4 / N
    S = S + S.T
    np.fill_diagonal(S, 0.0)
    F = np.concatenate([S, (A - S.sum(axis=1))[:, None]], axis=1) / A[:, None]
    return F, A, rng.uniform(0.2, 0.8, N)


def _context_still_works(rg_ctx):
    F, _, eps = _small_system()
    B, _, _ = api.gebhart(rg_ctx, _dev(F), _dev(eps), _dev(1 - eps), tol=1e-12)
    assert np.abs(B[0].cpu().numpy() - G.gebhart(F, eps, 1 - eps)).max() < 1e-7


@pytest.mark.parametrize("kind", ["mbarrier", "grid"])
def test_bounded_wait_runs_out_and_is_reported(rg_ctx, kind):
    with pytest.raises(api.RadgebError) as e:
        api.debug_wait_timeout(rg_ctx, kind, 0.01)
    assert e.value.code == "RG_ERR_CUDA" and "timed out" in str(e.value)
    torch.cuda.synchronize()
    _context_still_works(rg_ctx)


def test_non_finite_optical_properties_are_reported(rg_ctx):
    F, A, eps = _small_system()
    for e, r in ((np.where(np.arange(40) == 7, np.nan, eps), 1 - eps),
                 (eps, np.where(np.arange(40) == 3, np.nan, 1 - eps))):
        with pytest.raises(api.RadgebError) as err:
            api.gebhart(rg_ctx, _dev(F), _dev(e), _dev(r), tol=1e-12)
        assert err.value.code == "RG_ERR_NUMERIC"
    _context_still_works(rg_ctx)


def test_non_finite_view_factors_and_loads_are_reported(rg_ctx):
    F, A, eps = _small_system()
    Fn = F.copy()
    Fn[5, 9] = np.nan
    with pytest.raises(api.RadgebError) as err:
        api.enforce_iterative(rg_ctx, _dev(Fn), _dev(A))
    assert err.value.code == "RG_ERR_NUMERIC"
    B = G.gebhart(F, eps, 1 - eps)
    Q = np.full(40, 10.0)
    Q[2] = np.nan
    with pytest.raises(api.RadgebError) as err:
        api.temperatures(rg_ctx, _dev(B), _dev(eps), _dev(A), _dev(Q), 3.0)
    assert err.value.code == "RG_ERR_NUMERIC"
    _context_still_works(rg_ctx)



def test_invalid_radiative_balance_inputs_are_reported(rg_ctx):
    """A face with sigma eps A = 0 or a B row that sums to 0 has no radiative balance, and a
    heat load that drives T^4 below zero has no temperature: each is an error of the call,
    not a NaN in its output."""
    F, A, eps = _small_system()
    B = G.gebhart(F, eps, 1 - eps)
    Q = np.full(40, 10.0)
    To = G.temperatures(B, eps, A, Q, 3.0)
    e0 = eps.copy()
    e0[4] = 0.0
    B0 = B.copy()
    B0[6] = 0.0
    for Bx, ex in ((B, e0), (B0, eps)):
        with pytest.raises(api.RadgebError, match="no radiative exchange") as err:
            api.temperatures(rg_ctx, _dev(Bx), _dev(ex), _dev(A), _dev(Q), 3.0)
        assert err.value.code == "RG_ERR_NUMERIC"
        with pytest.raises(api.RadgebError, match="no radiative exchange") as err:
            api.temperatures_adjoint(rg_ctx, _dev(Bx), _dev(ex), _dev(A), 3.0, _dev(To), _dev(np.ones(40)))
        assert err.value.code == "RG_ERR_NUMERIC"
    Qn = Q.copy()
    Qn[9] = -1e12
    with pytest.raises(api.RadgebError, match="non-positive T") as err:
        api.temperatures(rg_ctx, _dev(B), _dev(eps), _dev(A), _dev(Qn), 3.0)
    assert err.value.code == "RG_ERR_NUMERIC"
    _context_still_works(rg_ctx)
