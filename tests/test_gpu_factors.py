"""Stored factors of the REF solve (rg_gebhart's factor store, read by rg_gebhart_adjoint and
rg_gebhart_adjoint_factored): the adjoints with the store give the gradients the oracle
gives (App. B, Eq. B.8-B.11, differentiated), they factorise nothing, the stored matrices
are approximate inverses of K^T, and a store that does not fit the call is refused before
any launch."""
import numpy as np
import pytest
import torch

from oracle import gebhart as G
from paper_2511_04277_gb300 import api
from paper_2511_04277_gb300._native import RadgebError

pytestmark = pytest.mark.gpu


def _dev(x):
    return torch.as_tensor(np.ascontiguousarray(x), dtype=torch.float64, device="cuda")


def _system(N, S, seed):
    """Random open system with closure and reciprocity, S opaque (eps, rho = 1 - eps) sets."""
    rng = np.random.default_rng(seed)
    A = rng.uniform(0.5, 2.0, N)
    G_ = rng.random((N, N)) * (rng.random((N, N)) < 0.3)
    G_ = (G_ + G_.T) / (2 * N) * 0.8
    np.fill_diagonal(G_, 0.0)
    F = np.concatenate([G_, (A - G_.sum(axis=1))[:, None]], axis=1) / A[:, None]
    eps = rng.uniform(0.05, 0.9, (S, N))
    return F, eps, 1.0 - eps, rng


@pytest.mark.parametrize("N,S,prec", [(300, 3, "fp16"), (257, 2, "bf16")])
def test_adjoints_with_stored_factors_match_the_oracle_and_factorise_nothing(rg_ctx, N, S, prec):
    F, eps, rho, rng = _system(N, S, 70 + N)
    Fd, ed, rd = _dev(F), _dev(eps), _dev(rho)
    store = api.gebhart_factor_store(N, S, prec)
    B, _, _ = api.gebhart(rg_ctx, Fd, ed, rd, prec, tol=1e-12, factors=store)
    W = _dev(rng.standard_normal((S, N, N + 1)))
    a = _dev(rng.standard_normal((S, 2, N)))
    b = _dev(rng.standard_normal((S, 2, N + 1)))
    api.kernel_timer(rg_ctx, True)
    de, dr = api.gebhart_adjoint(rg_ctx, Fd, ed, rd, B, W, prec, tol=1e-12, factors=store)
    de_f, dr_f = api.gebhart_adjoint_factored(rg_ctx, Fd, ed, rd, B, a, b, prec, tol=1e-12, factors=store)
    api.kernel_timer(rg_ctx, False)
    assert api.kernel_timer_read(rg_ctx, "factor")["launches"] == 0
    # the same gradients without the store (K^T factorised afresh)
    de0, dr0 = api.gebhart_adjoint(rg_ctx, Fd, ed, rd, B, W, prec, tol=1e-12)
    de0_f, dr0_f = api.gebhart_adjoint_factored(rg_ctx, Fd, ed, rd, B, a, b, prec, tol=1e-12)
    for got, ref in ((de, de0), (dr, dr0), (de_f, de0_f), (dr_f, dr0_f)):
        assert (got - ref).abs().max().item() <= 1e-10 * ref.abs().max().item()
    Bh = B.cpu().numpy()
    ah, bh = a.cpu().numpy(), b.cpu().numpy()
    for s in range(S):
        deo, dro = G.gebhart_adjoint(F, eps[s], rho[s], Bh[s], W[s].cpu().numpy())
        assert np.abs(de[s].cpu().numpy() - deo).max() <= 1e-9 * np.abs(deo).max()
        assert np.abs(dr[s].cpu().numpy() - dro).max() <= 1e-9 * np.abs(dro).max()
        # the factored cotangent sum_r a_r b_r^T through the oracle's full adjoint
        deo, dro = G.gebhart_adjoint(F, eps[s], rho[s], Bh[s], ah[s].T @ bh[s])
        assert np.abs(de_f[s].cpu().numpy() - deo).max() <= 1e-9 * np.abs(deo).max()
        assert np.abs(dr_f[s].cpu().numpy() - dro).max() <= 1e-9 * np.abs(dro).max()


def test_stored_matrices_are_approximate_inverses_of_K_transposed(rg_ctx):
    """Set s of the store holds M^T with M ~ K^-1 (16-bit, np x np, after a 256-byte header):
    ||I - K^T M^T||_inf is small and its padding is the identity's."""
    N, S = 200, 2
    F, eps, rho, _ = _system(N, S, 5)
    store = api.gebhart_factor_store(N, S, "fp16")
    api.gebhart(rg_ctx, _dev(F), _dev(eps), _dev(rho), "fp16", tol=1e-12, factors=store)
    np_ = 256
    mats = store[256:256 + S * np_ * np_ * 2].view(torch.float16).reshape(S, np_, np_).double().cpu().numpy()
    for s in range(S):
        K = G.k_matrix(F, rho[s])
        Mt = mats[s]
        E = np.eye(N) - K.T @ Mt[:N, :N]
        assert np.abs(E).sum(axis=1).max() <= 0.02
        assert np.abs(Mt[:N, N:]).max() == 0.0 and np.abs(Mt[N:, :N]).max() == 0.0
        assert np.allclose(Mt[N:, N:], np.eye(np_ - N), atol=1e-3)


def test_a_store_of_another_system_changes_the_sweeps_not_the_gradients(rg_ctx):
    """The residual is refined exactly against the call's own F and rho: factors of a nearby
    system (rho scaled by 0.9) give the gradients the call's own factors give."""
    N, S = 240, 2
    F, eps, rho, rng = _system(N, S, 8)
    Fd, ed, rd = _dev(F), _dev(eps), _dev(rho)
    other = api.gebhart_factor_store(N, S, "fp16")
    api.gebhart(rg_ctx, Fd, ed, _dev(0.9 * rho), "fp16", tol=1e-12, factors=other)
    B, _, _ = api.gebhart(rg_ctx, Fd, ed, rd, "fp16", tol=1e-12)
    W = _dev(rng.standard_normal((S, N, N + 1)))
    de, dr = api.gebhart_adjoint(rg_ctx, Fd, ed, rd, B, W, "fp16", tol=1e-12, max_sweeps=24, factors=other)
    de0, dr0 = api.gebhart_adjoint(rg_ctx, Fd, ed, rd, B, W, "fp16", tol=1e-12)
    assert (de - de0).abs().max().item() <= 1e-10 * de0.abs().max().item()
    assert (dr - dr0).abs().max().item() <= 1e-10 * dr0.abs().max().item()


def _code(fn):
    with pytest.raises(RadgebError) as e:
        fn()
    return e.value.code


def test_stores_that_do_not_fit_the_call_are_refused(rg_ctx):
    N, S = 200, 2
    F, eps, rho, rng = _system(N, S, 11)
    Fd, ed, rd = _dev(F), _dev(eps), _dev(rho)
    nbytes = api.gebhart_workspace(N, S, "fp16", keep_factors=True)
    assert nbytes == 256 + S * 256 * 256 * 2 + S * 256 * 8
    store = api.gebhart_factor_store(N, S, "fp16")
    B, _, _ = api.gebhart(rg_ctx, Fd, ed, rd, "fp16", tol=1e-12, factors=store)
    W = _dev(rng.standard_normal((S, N, N + 1)))
    a = _dev(rng.standard_normal((S, 2, N)))
    b = _dev(rng.standard_normal((S, 2, N + 1)))
    adj = lambda prec="fp16", st=store, **kw: api.gebhart_adjoint(rg_ctx, Fd, ed, rd, B, W, prec, tol=1e-12,
                                                                  factors=st, **kw)
    # another precision: the stored inverse would be a GEMM operand of the other 16-bit type
    assert _code(lambda: adj("bf16")) == "RG_ERR_ARG"
    assert _code(lambda: api.gebhart_adjoint_factored(rg_ctx, Fd, ed, rd, B, a, b, "bf16", tol=1e-12,
                                                      factors=store)) == "RG_ERR_ARG"
    # more sets than stored
    e3, r3, B3, W3 = (torch.cat([x, x[:1]]) for x in (ed, rd, B, W))
    assert _code(lambda: api.gebhart_adjoint(rg_ctx, Fd, e3, r3, B3, W3, "fp16", tol=1e-12,
                                             factors=store)) == "RG_ERR_ARG"
    # a store never filled, a short one, a misaligned one
    blank = torch.zeros_like(store)
    assert _code(lambda: adj(st=blank)) == "RG_ERR_ARG"
    assert _code(lambda: adj(st=store[:-1])) == "RG_ERR_ARG"
    big = torch.zeros(nbytes + 512, dtype=torch.uint8, device="cuda")
    assert _code(lambda: api.gebhart(rg_ctx, Fd, ed, rd, "fp16", tol=1e-12, factors=big[16:16 + nbytes])) \
        == "RG_ERR_ARG"
    assert _code(lambda: api.gebhart(rg_ctx, Fd, ed, rd, "fp16", tol=1e-12, factors=store[:-1])) == "RG_ERR_ARG"
    # factors of another n (199 pads to the same 256 x 256 blocks: only the header tells)
    F2, eps2, rho2, _ = _system(N - 1, S, 12)
    s2 = api.gebhart_factor_store(N - 1, S, "fp16")
    assert s2.numel() == store.numel()
    api.gebhart(rg_ctx, _dev(F2), _dev(eps2), _dev(rho2), "fp16", tol=1e-12, factors=s2)
    assert _code(lambda: adj(st=s2)) == "RG_ERR_ARG"
    # the store still works after the refusals
    de, _ = adj()
    de0, _ = api.gebhart_adjoint(rg_ctx, Fd, ed, rd, B, W, "fp16", tol=1e-12)
    assert (de - de0).abs().max().item() <= 1e-10 * de0.abs().max().item()


@pytest.mark.parametrize("rank", [3, 8, 9, 64])
def test_factored_adjoint_ranks_across_the_narrow_and_wide_kernels(rg_ctx, rank):
    """Up to 8 right-hand sides the sweeps run one thread per row; from 9 on, four columns
    per lane with a ragged last lane (9 = 4 + 4 + 1). Both against the oracle's adjoint of
    dB = sum_r a_r b_r^T, with and without stored factors."""
    N, S = 333, 2
    F, eps, rho, rng = _system(N, S, 200 + rank)
    Fd, ed, rd = _dev(F), _dev(eps), _dev(rho)
    store = api.gebhart_factor_store(N, S, "fp16")
    B, _, _ = api.gebhart(rg_ctx, Fd, ed, rd, "fp16", tol=1e-12, factors=store)
    a = _dev(rng.standard_normal((S, rank, N)))
    b = _dev(rng.standard_normal((S, rank, N + 1)))
    de, dr = api.gebhart_adjoint_factored(rg_ctx, Fd, ed, rd, B, a, b, "fp16", tol=1e-12, factors=store)
    de0, dr0 = api.gebhart_adjoint_factored(rg_ctx, Fd, ed, rd, B, a, b, "fp16", tol=1e-12)
    assert (de - de0).abs().max().item() <= 1e-10 * de0.abs().max().item()
    assert (dr - dr0).abs().max().item() <= 1e-10 * dr0.abs().max().item()
    Bh, ah, bh = B.cpu().numpy(), a.cpu().numpy(), b.cpu().numpy()
    for s in range(S):
        deo, dro = G.gebhart_adjoint(F, eps[s], rho[s], Bh[s], ah[s].T @ bh[s])
        assert np.abs(de[s].cpu().numpy() - deo).max() <= 1e-9 * np.abs(deo).max()
        assert np.abs(dr[s].cpu().numpy() - dro).max() <= 1e-9 * np.abs(dro).max()


# ------------------------------------------------------------------ symmetric factorisation
@pytest.mark.parametrize("N", [2500, 3700])
def test_symmetric_factorisation_matches_the_oracle(rg_ctx, N):
    # (the step count of the symmetric form comes from the unscaled system's norms)
    """With the areas of a reciprocal F the REF solve builds its 16-bit inverse in the
    symmetric form D K D^-1 (D = diag(sqrt(A rho))), computing the tiles on and above the
    diagonal of the symmetric product X (2I - A X) of each Newton-Schulz step: 128-wide tiles
    at N = 2,500, CTA pairs (256-wide) at N = 3,700. B against the oracle, and against the
    general factorisation."""
    rng = np.random.default_rng(N)
    A = rng.uniform(0.5, 2.0, N)
    G_ = rng.random((N, N)) * (rng.random((N, N)) < 0.3)
    G_ = (G_ + G_.T) / (2 * N) * 0.8
    np.fill_diagonal(G_, 0.0)
    F = np.concatenate([G_, (A - G_.sum(axis=1))[:, None]], axis=1) / A[:, None]
    eps = rng.uniform(0.05, 0.9, (2, N))
    rho = 1.0 - eps
    Fd, ed, rd, Ad = _dev(F), _dev(eps), _dev(rho), _dev(A)
    B, sw, res = api.gebhart(rg_ctx, Fd, ed, rd, "fp16", tol=1e-12, areas=Ad)
    B0, sw0, _ = api.gebhart(rg_ctx, Fd, ed, rd, "fp16", tol=1e-12)
    assert res <= 1e-12 and sw <= sw0 + 1
    assert (B - B0).abs().max().item() <= 1e-10 * B0.abs().max().item()
    for s in (0, 1):
        Bo = G.gebhart(F, eps[s], rho[s])
        got = B[s].cpu().numpy()
        err = (np.abs(got - Bo).max(axis=1) / np.abs(Bo).max(axis=1)).max()
        assert err <= 1e-9


def test_stored_symmetric_inverse_and_the_adjoints(rg_ctx):
    """The store keeps M_sym and d for a set factorised symmetrically (M = D^-1 M_sym D is an
    approximate inverse of K); the adjoints through it match the oracle and the adjoints
    without a store. A set with a zero reflectivity takes the general factorisation (zero d)."""
    N, S = 3700, 2
    rng = np.random.default_rng(5)
    A = rng.uniform(0.5, 2.0, N)
    G_ = rng.random((N, N)) * (rng.random((N, N)) < 0.3)
    G_ = (G_ + G_.T) / (2 * N) * 0.8
    np.fill_diagonal(G_, 0.0)
    F = np.concatenate([G_, (A - G_.sum(axis=1))[:, None]], axis=1) / A[:, None]
    eps = rng.uniform(0.05, 0.9, (S, N))
    eps[1, 7] = 1.0  # a black face: rho = 0 -> the general factorisation for set 1
    rho = 1.0 - eps
    Fd, ed, rd, Ad = _dev(F), _dev(eps), _dev(rho), _dev(A)
    store = api.gebhart_factor_store(N, S, "fp16")
    B, _, _ = api.gebhart(rg_ctx, Fd, ed, rd, "fp16", tol=1e-12, factors=store, areas=Ad)
    np_ = 3712
    mats = store[256:256 + S * np_ * np_ * 2].view(torch.float16).reshape(S, np_, np_)
    dv = store[256 + S * np_ * np_ * 2:].view(torch.float64).reshape(S, np_)
    d0 = dv[0, :N].cpu().numpy()
    assert (d0 > 0).all() and abs(d0.max() - 1.0) < 1e-12 and not dv[1].any()
    Msym = mats[0, :N, :N].double().cpu().numpy()
    # mirrored tiles are exact transposes; diagonal tiles are symmetric to 16-bit rounding
    assert np.abs(Msym - Msym.T).max() <= 2e-3 * np.abs(Msym).max()
    K = G.k_matrix(F, rho[0])
    M = Msym * (d0[None, :] / d0[:, None])             # D^-1 M_sym D
    assert np.abs(np.eye(N) - K @ M).sum(axis=1).max() <= 0.05
    W = _dev(rng.standard_normal((S, N, N + 1)))
    a = _dev(rng.standard_normal((S, 2, N)))
    b = _dev(rng.standard_normal((S, 2, N + 1)))
    de, dr = api.gebhart_adjoint(rg_ctx, Fd, ed, rd, B, W, "fp16", tol=1e-12, factors=store)
    de0, dr0 = api.gebhart_adjoint(rg_ctx, Fd, ed, rd, B, W, "fp16", tol=1e-12)
    de_f, dr_f = api.gebhart_adjoint_factored(rg_ctx, Fd, ed, rd, B, a, b, "fp16", tol=1e-12, factors=store)
    de0_f, dr0_f = api.gebhart_adjoint_factored(rg_ctx, Fd, ed, rd, B, a, b, "fp16", tol=1e-12)
    for got, ref in ((de, de0), (dr, dr0), (de_f, de0_f), (dr_f, dr0_f)):
        assert (got - ref).abs().max().item() <= 1e-10 * ref.abs().max().item()
    Bh = B.cpu().numpy()
    deo, dro = G.gebhart_adjoint(F, eps[0], rho[0], Bh[0], W[0].cpu().numpy())
    assert np.abs(de[0].cpu().numpy() - deo).max() <= 1e-9 * np.abs(deo).max()
    assert np.abs(dr[0].cpu().numpy() - dro).max() <= 1e-9 * np.abs(dro).max()
