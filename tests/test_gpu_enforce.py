"""GPU enforcement and aggregation (rg_enforce_iterative, rg_aggregate) against the oracle."""
import numpy as np
import pytest
import torch

import synth
from oracle import enforce as E
from oracle import mcrt
from oracle import multinode as MN
from paper_2511_04277_gb300 import api
from tests.conftest import load_matrix

pytestmark = pytest.mark.gpu

TOL = 1e-12


def _dev(x, dtype=torch.float64):
    return torch.as_tensor(np.ascontiguousarray(x)).to(dtype=dtype, device="cuda")


def _random_F(N, rng, zeros=0.2):
    F = rng.random((N, N + 1))
    F[rng.random((N, N + 1)) < zeros] = 0.0
    np.fill_diagonal(F[:, :N], 0.0)
    F[:, N] += 0.05
    return F / F.sum(axis=1, keepdims=True)


def test_iterative_disc_example(rg_ctx):
    F1 = load_matrix("disc_F1_mcrt.txt")
    A = np.array([1.0, 4.0, 1.0, 4.0])
    Fd = _dev(F1)
    it = api.enforce_iterative(rg_ctx, Fd, _dev(A), tol=TOL)
    Fo, it_o, _ = E.iterative(F1, A, tol=TOL)
    got = Fd.cpu().numpy()
    assert np.abs(got - Fo).max() <= 1e-14
    assert abs(it - it_o) <= 1
    assert np.abs(got - load_matrix("disc_F6_iterative.txt")).max() <= 1e-6


@pytest.mark.parametrize("N", [1, 63, 64, 65, 200, 2048])
def test_iterative_random_sizes(rg_ctx, N):
    rng = np.random.default_rng(N)
    F = _random_F(N, rng)
    A = rng.uniform(0.5, 2.0, N)
    Fd = _dev(F)
    it = api.enforce_iterative(rg_ctx, Fd, _dev(A), tol=TOL)
    Fo, it_o, ok = E.iterative(F, A, tol=TOL)
    assert ok and abs(it - it_o) <= 1
    got = Fd.cpu().numpy()
    # row-normwise: max_j |F - F_ref| <= 1e-6 max_j |F_ref| (here far tighter)
    assert np.all(np.abs(got - Fo).max(axis=1) <= 1e-10 * np.abs(Fo).max(axis=1))


def test_iterative_not_converged_is_reported(rg_ctx):
    rng = np.random.default_rng(3)
    F = _random_F(50, rng)
    A = rng.uniform(0.5, 2.0, 50)
    Fd = _dev(F)
    with pytest.raises(api.RadgebError) as e:
        api.enforce_iterative(rg_ctx, Fd, _dev(A), tol=0.0, maxit=3)
    assert e.value.code == "RG_ERR_NOT_CONVERGED"
    Fo, _, _ = E.iterative(F, A, tol=0.0, maxit=3)
    assert np.abs(Fd.cpu().numpy() - Fo).max() < 1e-13   # holds the last iterate


def test_iterative_on_plates_mcrt(rg_ctx):
    """Config-sized: 512 sub-faces from GPU counts, enforced on the GPU and by the oracle."""
    m = synth.plates(16)
    rays = np.full(m.n_faces, 20000, np.int64)
    mesh = api.Mesh.from_synth(rg_ctx, m)
    c = api.trace(rg_ctx, mesh, rays, 0)
    F = api.counts_to_F(rg_ctx, c, _dev(rays, torch.int64))
    F0 = F.cpu().numpy()
    A = mesh.face_areas()
    api.enforce_iterative(rg_ctx, F, _dev(A), tol=TOL)
    Fo, _, _ = E.iterative(F0, A, tol=TOL)
    got = F.cpu().numpy()
    assert np.all(np.abs(got - Fo).max(axis=1) <= 1e-10 * np.abs(Fo).max(axis=1))
    assert np.abs(got.sum(axis=1) - 1).max() < 1e-13
    eta = A[:, None] * got[:, :512]
    assert np.abs(eta - eta.T).max() < 1e-11


def test_aggregate_plates(rg_ctx):
    m = synth.plates(16)
    rays = np.full(m.n_faces, 20000, np.int64)
    mesh = api.Mesh.from_synth(rg_ctx, m)
    F = api.counts_to_F(rg_ctx, api.trace(rg_ctx, mesh, rays, 0), _dev(rays, torch.int64))
    A = mesh.face_areas()
    api.enforce_iterative(rg_ctx, F, _dev(A))
    grp = m.patch_of_face.astype(np.int32)
    Fg, Sg = api.aggregate(rg_ctx, F, _dev(A), _dev(grp, torch.int32), 2)
    Fo, So = MN.surface_view_factors(F.cpu().numpy(), A, grp, 2)
    assert np.abs(Fg.cpu().numpy() - Fo).max() <= 1e-13
    assert np.abs(Sg.cpu().numpy() - So).max() <= 1e-13
    # whole plates: closed form 0.415253, within the MCRT error of 5.12e6 rays
    assert abs(Fo[0, 1] - 0.415253) < 1e-3


@pytest.mark.parametrize("N,G", [(37, 5), (300, 300), (1000, 17)])
def test_aggregate_random(rg_ctx, N, G):
    rng = np.random.default_rng(N + G)
    F = _random_F(N, rng)
    S = rng.uniform(0.5, 2.0, N)
    grp = rng.integers(0, G, N).astype(np.int32)
    grp[:G] = np.arange(G)
    Fg, _ = api.aggregate(rg_ctx, _dev(F), _dev(S), _dev(grp, torch.int32), G)
    Fo, _ = MN.surface_view_factors(F, S, grp, G)
    assert np.abs(Fg.cpu().numpy() - Fo).max() <= 1e-13


def test_aggregate_rejects_bad_group(rg_ctx):
    F = _random_F(8, np.random.default_rng(0))
    grp = np.array([0, 1, 2, 3, 0, 1, 2, 9], np.int32)
    with pytest.raises(api.RadgebError):
        api.aggregate(rg_ctx, _dev(F), _dev(np.ones(8)), _dev(grp, torch.int32), 4)


# ------------------------------------------------------------------ weighted reciprocity
def _plates_mcrt(rg_ctx, per_face=20000, seed=0):
    m = synth.plates(16)
    rays = np.full(m.n_faces, per_face, np.int64)
    rays[::7] = per_face // 4           # unequal ray budgets, so kappa is not 1/2
    mesh = api.Mesh.from_synth(rg_ctx, m)
    F = api.counts_to_F(rg_ctx, api.trace(rg_ctx, mesh, rays, seed), _dev(rays, torch.int64))
    return F, rays, mesh.face_areas()


@pytest.mark.parametrize("mode", ["triangulation", "fractional_variance"])
def test_kappa_matches_oracle(rg_ctx, mode):
    F, rays, A = _plates_mcrt(rg_ctx)
    K = api.kappa(rg_ctx, _dev(rays, torch.int64), _dev(A), mode, F=F).cpu().numpy()
    F0 = F.cpu().numpy()
    if mode == "triangulation":
        Ko = E.kappa_triangulation(rays, A, n=0.4)
    else:
        Ko = E.kappa_fractional_variance(F0, rays, A, z=1.96)
    assert np.abs(K - Ko).max() <= 1e-14
    assert np.abs(K - 0.5).max() > 0.1


@pytest.mark.parametrize("mode", ["triangulation", "fractional_variance"])
def test_iterative_kappa_vs_oracle(rg_ctx, mode):
    F, rays, A = _plates_mcrt(rg_ctx)
    F0 = F.cpu().numpy()
    K = api.kappa(rg_ctx, _dev(rays, torch.int64), _dev(A), mode, F=F)
    it = api.enforce_iterative_kappa(rg_ctx, F, _dev(A), K, tol=TOL)
    Fo, it_o, ok = E.iterative(F0, A, tol=TOL, kappa=K.cpu().numpy())
    assert ok and abs(it - it_o) <= 1
    got = F.cpu().numpy()
    assert np.all(np.abs(got - Fo).max(axis=1) <= 1e-10 * np.abs(Fo).max(axis=1))
    assert np.abs(got.sum(axis=1) - 1).max() < 1e-13
    eta = A[:, None] * got[:, :512]
    assert np.abs(eta - eta.T).max() < 1e-11


def test_iterative_kappa_one_half_is_the_default(rg_ctx):
    rng = np.random.default_rng(21)
    N = 200
    F = _random_F(N, rng)
    A = _dev(rng.uniform(0.5, 2.0, N))
    Fa, Fb = _dev(F), _dev(F)
    ia = api.enforce_iterative(rg_ctx, Fa, A, tol=TOL)
    ib = api.enforce_iterative_kappa(rg_ctx, Fb, A, torch.full((N, N), 0.5, dtype=torch.float64, device="cuda"),
                                     tol=TOL)
    # equal weights take the symmetric iterations (fixed-point row sums), a weight matrix
    # the full fp64 ones: the same iterates up to rounding
    assert abs(ia - ib) <= 1
    d = (Fa - Fb).abs().amax(dim=1) / Fb.abs().amax(dim=1)
    assert d.max().item() <= 1e-12


@pytest.mark.parametrize("N", [2049, 4160])
def test_iterative_wide_tiles(rg_ctx, N):
    """64-wide tiles (N > 2,048) with ragged last tiles."""
    rng = np.random.default_rng(N)
    F = _random_F(N, rng, zeros=0.5)
    A = rng.uniform(0.5, 2.0, N)
    Fd = _dev(F)
    it = api.enforce_iterative(rg_ctx, Fd, _dev(A), tol=TOL)
    Fo, it_o, ok = E.iterative(F, A, tol=TOL)
    assert ok and abs(it - it_o) <= 1
    got = Fd.cpu().numpy()
    assert np.all(np.abs(got - Fo).max(axis=1) <= 1e-10 * np.abs(Fo).max(axis=1))


@pytest.mark.parametrize("N", [300, 2500])
def test_iterative_wide_area_range(rg_ctx, N):
    """Areas over nine decades and rows that see only the environment: the per-row
    fixed-point exponents of the symmetric iterations follow each row's own scale."""
    rng = np.random.default_rng(7 * N)
    F = _random_F(N, rng, zeros=0.3)
    F[:5, :N] = 0.0
    F[:5, N] = 1.0
    F[:N, :5] = 0.0
    F = F / F.sum(axis=1, keepdims=True)
    A = 10.0 ** rng.uniform(-6, 3, N)
    # the stop rule is absolute (tol max Omega), so the small rows are not converged to
    # their own scale when it fires: compare the iterates after the same count
    _, it_o, ok = E.iterative(F, A, tol=TOL)
    assert ok
    Fo, _, _ = E.iterative(F, A, tol=0.0, maxit=it_o)
    Fd = _dev(F)
    with pytest.raises(api.RadgebError) as e:
        api.enforce_iterative(rg_ctx, Fd, _dev(A), tol=0.0, maxit=it_o)
    assert e.value.code == "RG_ERR_NOT_CONVERGED"
    got = Fd.cpu().numpy()
    assert np.all(np.abs(got - Fo).max(axis=1) <= 1e-10 * np.abs(Fo).max(axis=1))
    assert np.all(got[:5, :N] == 0.0)


def test_iterative_negative_entries_take_the_full_path(rg_ctx):
    """A negative entry keeps every iteration on the full fp64 path (the symmetric
    iterations need non-negative entries); the result still follows the oracle."""
    rng = np.random.default_rng(5)
    N = 150
    F = _random_F(N, rng)
    F[3, 7] = -1e-3
    F[40, 2] = -2e-4
    A = rng.uniform(0.5, 2.0, N)
    Fd = _dev(F)
    it = api.enforce_iterative(rg_ctx, Fd, _dev(A), tol=TOL)
    Fo, it_o, ok = E.iterative(F, A, tol=TOL)
    assert ok and abs(it - it_o) <= 1
    got = Fd.cpu().numpy()
    assert np.all(np.abs(got - Fo).max(axis=1) <= 1e-10 * np.abs(Fo).max(axis=1))


def test_iterative_already_enforced(rg_ctx):
    """An enforced F converges in the first (full) iteration and comes back unchanged
    up to rounding."""
    rng = np.random.default_rng(9)
    N = 2100
    F = _random_F(N, rng)
    A = rng.uniform(0.5, 2.0, N)
    Fo, _, ok = E.iterative(F, A, tol=1e-14)
    assert ok
    Fd = _dev(Fo)
    it = api.enforce_iterative(rg_ctx, Fd, _dev(A), tol=1e-12)
    assert it == 1
    assert np.abs(Fd.cpu().numpy() - Fo).max() <= 1e-15


def test_kappa_rejects_bad_input(rg_ctx):
    rays = torch.tensor([10, 0, 5], dtype=torch.int64, device="cuda")
    with pytest.raises(api.RadgebError) as e:
        api.kappa(rg_ctx, rays, torch.ones(3, dtype=torch.float64, device="cuda"), "triangulation")
    assert e.value.code == "RG_ERR_ARG"
    with pytest.raises(api.RadgebError):
        api.kappa(rg_ctx, rays.abs() + 1, torch.ones(3, dtype=torch.float64, device="cuda"), "fractional_variance")


def test_ref_enforcement_with_eps_area(rg_ctx):
    """REFs from an un-enforced F break Eq. 4.4; the iterative enforcer with Omega = eps A
    (Sec. 4.2.3) restores closure and eps_i A_i B_ij = eps_j A_j B_ji."""
    F, rays, A = _plates_mcrt(rg_ctx, per_face=5000)
    w = synth.workload("plates")
    eps = w["eps"][0]
    B, _, _ = api.gebhart(rg_ctx, F, _dev(eps), _dev(1 - eps), tol=1e-12)
    B0 = B[0].cpu().numpy()
    om = eps * A
    R0 = om[:, None] * B0[:, :512]
    assert np.abs(R0 - R0.T).max() > 1e-4 * np.abs(R0).max()       # not reciprocal before
    Bd = B[0].contiguous()
    api.enforce_iterative(rg_ctx, Bd, _dev(om), tol=TOL)
    Bo, _, ok = E.iterative(B0, om, tol=TOL)
    got = Bd.cpu().numpy()
    assert ok and np.all(np.abs(got - Bo).max(axis=1) <= 1e-10 * np.abs(Bo).max(axis=1))
    assert np.abs(got.sum(axis=1) - 1).max() < 1e-13
    R = om[:, None] * got[:, :512]
    assert np.abs(R - R.T).max() < 1e-11 * np.abs(R).max()
