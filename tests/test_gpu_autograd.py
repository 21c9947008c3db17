"""torch.autograd wrappers of the REF and balance solves against the fp64 oracle."""
import numpy as np
import pytest
import torch

from oracle import gebhart as G
from paper_2511_04277_gb300 import autograd

pytestmark = pytest.mark.gpu

REL = 1e-6


def _dev(x):
    return torch.as_tensor(np.ascontiguousarray(x), dtype=torch.float64).cuda()


def _consistent_F(N, rng, density=0.3):
    A = rng.uniform(0.5, 2.0, N)
    S = rng.random((N, N)) * (rng.random((N, N)) < density)
    S = (S + S.T) / (2 * N) * 0.8
    np.fill_diagonal(S, 0.0)
    env = A - S.sum(axis=1)
    return np.concatenate([S, env[:, None]], axis=1) / A[:, None], A


def test_gebhart_function_gradients_of_three_sets(rg_ctx):
    rng = np.random.default_rng(31)
    N, S = 97, 3
    F, _ = _consistent_F(N, rng)
    eps0 = rng.uniform(0.1, 0.9, (S, N))
    rho0 = rng.uniform(0.0, 1.0, (S, N)) * (1 - eps0)     # semi-transparent-free, eps + rho <= 1
    W = rng.standard_normal((S, N, N + 1))
    eps = _dev(eps0).requires_grad_(True)
    rho = _dev(rho0).requires_grad_(True)
    B = autograd.gebhart(rg_ctx, _dev(F), eps, rho)
    (B * _dev(W)).sum().backward()
    for s in range(S):
        Bo = G.gebhart(F, eps0[s], rho0[s])
        assert np.abs(B[s].detach().cpu().numpy() - Bo).max() <= REL * np.abs(Bo).max()
        deo, dro = G.gebhart_adjoint(F, eps0[s], rho0[s], Bo, W[s])
        assert np.abs(eps.grad[s].cpu().numpy() - deo).max() <= REL * np.abs(deo).max()
        assert np.abs(rho.grad[s].cpu().numpy() - dro).max() <= REL * np.abs(dro).max()


def test_steady_temperatures_gradients_vs_oracle_and_differences(rg_ctx):
    rng = np.random.default_rng(32)
    N = 140
    F, A = _consistent_F(N, rng)
    eps0 = rng.uniform(0.1, 0.9, N)
    rho0 = 1 - eps0
    Q = rng.uniform(0, 50, N)
    wT = rng.standard_normal(N)
    eps = _dev(eps0).requires_grad_(True)
    rho = _dev(rho0).requires_grad_(True)
    T = autograd.steady_temperatures(rg_ctx, _dev(F), eps, rho, _dev(A), _dev(Q), 3.0)
    (T * _dev(wT)).sum().backward()
    ge, gr = eps.grad.cpu().numpy(), rho.grad.cpu().numpy()
    geo, gro = G.thermal_gradients(F, eps0, rho0, A, Q, 3.0, wT)
    assert np.abs(ge - geo).max() <= REL * np.abs(geo).max()
    assert np.abs(gr - gro).max() <= REL * np.abs(gro).max()

    def L(e, r):
        return float(np.sum(wT * G.temperatures(G.gebhart(F, e, r), e, A, Q, 3.0)))

    fe = G.central_difference(lambda e: L(e, rho0), eps0)
    fr = G.central_difference(lambda r: L(eps0, r), rho0)
    assert np.abs(ge - fe).max() <= 1e-5 * np.abs(fe).max()
    assert np.abs(gr - fr).max() <= 1e-5 * np.abs(fr).max()


def test_only_eps_requested(rg_ctx):
    rng = np.random.default_rng(33)
    N = 40
    F, A = _consistent_F(N, rng)
    eps0 = rng.uniform(0.2, 0.8, N)
    Q = rng.uniform(0, 50, N)
    eps = _dev(eps0).requires_grad_(True)
    T = autograd.steady_temperatures(rg_ctx, _dev(F), eps, _dev(1 - eps0), _dev(A), _dev(Q), 3.0)
    T.sum().backward()
    geo, _ = G.thermal_gradients(F, eps0, 1 - eps0, A, Q, 3.0, np.ones(N))
    assert np.abs(eps.grad.cpu().numpy() - geo).max() <= REL * np.abs(geo).max()


def test_gradients_of_constants_are_refused(rg_ctx):
    rng = np.random.default_rng(34)
    N = 20
    F, A = _consistent_F(N, rng)
    eps0 = rng.uniform(0.2, 0.8, N)
    Fd = _dev(F).requires_grad_(True)
    B = autograd.gebhart(rg_ctx, Fd, _dev(eps0), _dev(1 - eps0))
    with pytest.raises(NotImplementedError):
        B.sum().backward()
    Qd = _dev(rng.uniform(0, 50, N)).requires_grad_(True)
    Bo = _dev(G.gebhart(F, eps0, 1 - eps0))
    T = autograd.temperatures(rg_ctx, Bo, _dev(eps0), _dev(A), Qd, 3.0)
    with pytest.raises(NotImplementedError):
        T.sum().backward()
