"""GPU dense solves against the oracle: the tcgen05 GEMM on its own, REFs (App. B),
their adjoint, the steady radiative balance and its adjoint, and the least-squares
optimum enforcer with NNR / SPVA.

Floating-point bar: row-normwise max_j |X_ij - X_ref,ij| <= 1e-6 max_j |X_ref,ij| for
matrices, and ||g - g_ref||_inf <= 1e-6 ||g_ref||_inf for gradients.
"""
import numpy as np
import pytest
import torch

import synth
from oracle import enforce as E
from oracle import gebhart as G
from oracle import mcrt
from paper_2511_04277_gb300 import api
from tests.conftest import load_matrix

pytestmark = pytest.mark.gpu

REL = 1e-6


def _dev(x, dtype=torch.float64):
    return torch.as_tensor(np.ascontiguousarray(x)).to(dtype=dtype, device="cuda")


def _rownorm_err(got, ref):
    got, ref = np.asarray(got), np.asarray(ref)
    scale = np.maximum(np.abs(ref).max(axis=-1), 1e-300)
    return float((np.abs(got - ref).max(axis=-1) / scale).max())


def _consistent_F(N, rng, density=0.3):
    """Random open-system F with reciprocity and closure (areas returned)."""
    A = rng.uniform(0.5, 2.0, N)
    S = rng.random((N, N)) * (rng.random((N, N)) < density)
    S = (S + S.T) / (2 * N) * 0.8
    np.fill_diagonal(S, 0.0)
    env = A - S.sum(axis=1)
    assert env.min() > 0
    return np.concatenate([S, env[:, None]], axis=1) / A[:, None], A


# ------------------------------------------------------------------ GEMM
@pytest.mark.parametrize("M,N,K,dt", [(128, 128, 64, torch.bfloat16), (300, 200, 96, torch.bfloat16),
                                      (257, 513, 640, torch.float16), (1, 5, 8, torch.bfloat16)])
def test_tc_gemm_matches_fp64_of_rounded_operands(rg_ctx, M, N, K, dt):
    g = torch.Generator().manual_seed(M + N + K)
    A = torch.randn(M, K, generator=g).to(dt)
    B = torch.randn(N, K, generator=g).to(dt)
    C0 = torch.randn(M, N, generator=g, dtype=torch.float32)
    C = api.tc_gemm(rg_ctx, A.cuda(), B.cuda(), C0.clone().cuda(), alpha=-1.0, beta=1.0).cpu().double()
    ref = C0.double() - A.double() @ B.double().T
    err = (C - ref).abs().max().item()
    assert err <= 2e-5 * (A.double().abs() @ B.double().abs().T).max().item()


@pytest.mark.parametrize("dt", [torch.bfloat16, torch.float16])
@pytest.mark.parametrize("M", [5000, 4900])
def test_tc_gemm_wide_tiles_with_ragged_edges(rg_ctx, dt, M):
    """Enough tiles for the CTA-pair path (256 x 256 tiles, two CTAs each), with partial tiles on
    both edges: at N = 4,931 the odd CTA's half of B in the last column tile lies wholly
    beyond N, at M = 4,900 its rows in the last row tile lie wholly beyond M, and K = 200 ends
    in a partial K block."""
    N, K = 4931, 200
    g = torch.Generator().manual_seed(7)
    A = torch.randn(M, K, generator=g).to(dt)
    B = torch.randn(N, K, generator=g).to(dt)
    C0 = torch.randn(M, N, generator=g, dtype=torch.float32)
    C = api.tc_gemm(rg_ctx, A.cuda(), B.cuda(), C0.clone().cuda(), alpha=-1.0, beta=1.0).cpu().double()
    ref = C0.double() - A.double() @ B.double().T
    scale = (A.double().abs() @ B.double().abs().T).max().item()
    assert (C - ref).abs().max().item() <= 2e-5 * scale


# ------------------------------------------------------------------ REFs
def test_gebhart_plates_example(rg_ctx):
    F = load_matrix("plates_F.txt")
    eps = np.full(4, 0.5)
    B, sw, res = api.gebhart(rg_ctx, _dev(F), _dev(eps), _dev(1 - eps), tol=1e-13)
    assert np.abs(B[0].cpu().numpy() - load_matrix("plates_B.txt")).max() <= 5e-7
    assert res <= 1e-8


@pytest.mark.parametrize("N", [1, 6, 127, 128, 129, 300, 512])
@pytest.mark.parametrize("prec", ["bf16", "fp16"])
def test_gebhart_random_sizes(rg_ctx, N, prec):
    rng = np.random.default_rng(N)
    F, A = _consistent_F(N, rng)
    eps = rng.uniform(0.1, 0.9, N)
    B, sw, res = api.gebhart(rg_ctx, _dev(F), _dev(eps), _dev(1 - eps), precision=prec, tol=1e-12)
    Bo = G.gebhart(F, eps, 1 - eps)
    assert _rownorm_err(B[0].cpu().numpy(), Bo) <= REL
    assert _rownorm_err(B[0].cpu().numpy(), Bo) <= 1e-10
    # converged to tol (the residual is tracked exactly, so 1e-12 is reachable)
    assert res <= 1e-12 and sw >= 1


def test_gebhart_batched_sets_and_identities(rg_ctx):
    rng = np.random.default_rng(11)
    N, S = 200, 3
    F, A = _consistent_F(N, rng)
    eps = rng.uniform(0.05, 0.9, (S, N))
    rho = 1 - eps
    B, _, _ = api.gebhart(rg_ctx, _dev(F), _dev(eps), _dev(rho), tol=1e-12)
    Bg = B.cpu().numpy()
    for s in range(S):
        Bo = G.gebhart(F, eps[s], rho[s])
        assert _rownorm_err(Bg[s], Bo) <= REL
        # the identities hold to the refinement's exactly tracked residual (tol 1e-12)
        assert _rownorm_err(Bg[s], Bo) <= 1e-10
        assert np.abs(Bg[s].sum(axis=1) - 1).max() <= 1e-10                  # Eq. 4.3
        R = (eps[s] * A)[:, None] * Bg[s][:, :N]
        assert np.abs(R - R.T).max() <= 1e-10 * np.abs(R).max()               # Eq. 4.4


def test_gebhart_black_surfaces(rg_ctx):
    rng = np.random.default_rng(5)
    F, _ = _consistent_F(130, rng)
    eps = rng.uniform(0.1, 0.9, 130)
    B, sw, _ = api.gebhart(rg_ctx, _dev(F), _dev(eps), _dev(np.zeros(130)), tol=1e-13)
    # K = I: the refinement from a 16-bit first solve lands on E to near double precision
    assert np.abs(B[0].cpu().numpy() - G.e_matrix(F, eps)).max() <= 1e-12


def test_gebhart_cube_closed_forms(rg_ctx):
    # config-1 REFs from the closed-form cube view factors, closed system (env column 0)
    from tests import closed_forms as cf
    opp, adj = cf.parallel_opposed(1, 1, 1), cf.perpendicular_common_edge(1, 1, 1)
    F = np.full((6, 7), adj)
    F[:, 6] = 0.0
    for i in range(6):
        F[i, i] = 0.0
        F[i, i ^ 1] = opp
    eps = np.full(6, 0.8)
    B, _, _ = api.gebhart(rg_ctx, _dev(F), _dev(eps), _dev(1 - eps), tol=1e-13)
    Bo = G.gebhart(F, eps, 1 - eps)
    assert _rownorm_err(B[0].cpu().numpy(), Bo) <= 1e-9


def test_gebhart_plates_workload_full_size(rg_ctx):
    """N = 512 from GPU MCRT + GPU enforcement, eps ~ U[0.1, 0.9]: the bench's solve."""
    w = synth.workload("plates", rays_scale=0.02)
    m = w["mesh"]
    mesh = api.Mesh.from_synth(rg_ctx, m)
    F = api.counts_to_F(rg_ctx, api.trace(rg_ctx, mesh, w["rays"], 0), _dev(w["rays"], torch.int64))
    api.enforce_iterative(rg_ctx, F, _dev(mesh.face_areas()))
    B, sw, res = api.gebhart(rg_ctx, F, _dev(w["eps"]), _dev(w["rho"]), tol=1e-12)
    Bo = G.gebhart(F.cpu().numpy(), w["eps"][0], w["rho"][0])
    assert _rownorm_err(B[0].cpu().numpy(), Bo) <= REL


def test_gebhart_not_converged_is_reported(rg_ctx):
    rng = np.random.default_rng(8)
    F, _ = _consistent_F(256, rng)
    eps = rng.uniform(0.05, 0.1, 256)
    with pytest.raises(api.RadgebError) as e:
        api.gebhart(rg_ctx, _dev(F), _dev(eps), _dev(1 - eps), tol=1e-13, max_sweeps=1)
    assert e.value.code == "RG_ERR_NOT_CONVERGED"


# ------------------------------------------------------------------ adjoints
@pytest.mark.parametrize("N", [5, 140])
def test_gebhart_adjoint_vs_oracle(rg_ctx, N):
    rng = np.random.default_rng(100 + N)
    F, _ = _consistent_F(N, rng)
    eps = rng.uniform(0.1, 0.9, N)
    rho = 1 - eps
    W = rng.standard_normal((N, N + 1))
    Bo = G.gebhart(F, eps, rho)
    de, dr = api.gebhart_adjoint(rg_ctx, _dev(F), _dev(eps), _dev(rho), _dev(Bo), _dev(W), tol=1e-12)
    deo, dro = G.gebhart_adjoint(F, eps, rho, Bo, W)
    assert np.abs(de[0].cpu().numpy() - deo).max() <= REL * np.abs(deo).max()
    assert np.abs(dr[0].cpu().numpy() - dro).max() <= REL * np.abs(dro).max()


def test_temperatures_vs_oracle(rg_ctx):
    w = synth.workload("thermal", rays_scale=0.01)
    m = w["mesh"]
    mesh = api.Mesh.from_synth(rg_ctx, m)
    F = api.counts_to_F(rg_ctx, api.trace(rg_ctx, mesh, w["rays"], 0), _dev(w["rays"], torch.int64))
    A = mesh.face_areas()
    api.enforce_iterative(rg_ctx, F, _dev(A))
    eps = w["eps"][0]
    B, _, _ = api.gebhart(rg_ctx, F, _dev(eps), _dev(w["rho"][0]), tol=1e-12)
    T = api.temperatures(rg_ctx, B[0].contiguous(), _dev(eps), _dev(A), _dev(w["Q"]), w["T_sink"], tol=1e-13)
    To = G.temperatures(B[0].cpu().numpy(), eps, A, w["Q"], w["T_sink"])
    assert np.abs(T.cpu().numpy() - To).max() <= REL * To.max()


def test_temperatures_adjoint_vs_oracle(rg_ctx):
    rng = np.random.default_rng(21)
    N = 150
    F, A = _consistent_F(N, rng)
    eps = rng.uniform(0.1, 0.9, N)
    Q = rng.uniform(0, 50, N)
    Bo = G.gebhart(F, eps, 1 - eps)
    To = G.temperatures(Bo, eps, A, Q, 3.0)
    wT = rng.standard_normal(N)
    dB, deps = api.temperatures_adjoint(rg_ctx, _dev(Bo), _dev(eps), _dev(A), 3.0, _dev(To), _dev(wT), tol=1e-13)
    dBo, depso = G.temperatures_adjoint(Bo, eps, A, Q, 3.0, To, wT)
    assert np.abs(dB.cpu().numpy() - dBo).max() <= REL * np.abs(dBo).max()
    assert np.abs(deps.cpu().numpy() - depso).max() <= REL * np.abs(depso).max()


@pytest.mark.parametrize("prec", ["fp16", "bf16"])
def test_temperature_sets_vs_oracle_and_per_set_calls(rg_ctx, prec):
    """rg_temperatures_sets / rg_temperatures_adjoint_sets (one shared preconditioner for all
    sets) against the oracle's balance and adjoint of each set (Eq. 3.13, 4.2), and against
    the per-set entry points: the same equations, refined to the same tolerance."""
    rng = np.random.default_rng(33)
    N, S = 300, 3
    F, A = _consistent_F(N, rng)
    eps = rng.uniform(0.05, 0.9, (S, N))
    rho = 1 - eps
    Q = rng.uniform(0, 50, (S, N))
    B, _, _ = api.gebhart(rg_ctx, _dev(F), _dev(eps), _dev(rho), tol=1e-12)
    T = api.temperatures_sets(rg_ctx, _dev(F), B, _dev(eps), _dev(rho), _dev(A), _dev(Q), 3.0, precision=prec,
                              tol=1e-13)
    wT = rng.standard_normal((S, N))
    dB, deps = api.temperatures_adjoint_sets(rg_ctx, _dev(F), B, _dev(eps), _dev(rho), _dev(A), 3.0, T, _dev(wT),
                                             precision=prec, tol=1e-13)
    Bh = B.cpu().numpy()
    for s in range(S):
        To = G.temperatures(Bh[s], eps[s], A, Q[s], 3.0)
        assert np.abs(T[s].cpu().numpy() - To).max() <= 1e-10 * To.max()
        dBo, depso = G.temperatures_adjoint(Bh[s], eps[s], A, Q[s], 3.0, T[s].cpu().numpy(), wT[s])
        assert np.abs(dB[s].cpu().numpy() - dBo).max() <= 1e-9 * np.abs(dBo).max()
        assert np.abs(deps[s].cpu().numpy() - depso).max() <= 1e-9 * np.abs(depso).max()
        T1 = api.temperatures(rg_ctx, B[s].contiguous(), _dev(eps[s]), _dev(A), _dev(Q[s]), 3.0, precision=prec,
                              tol=1e-13)
        assert np.abs(T1.cpu().numpy() - T[s].cpu().numpy()).max() <= 1e-10 * To.max()


def test_factored_thermal_adjoint_vs_full_and_oracle(rg_ctx):
    """The calibration chain with the temperature cotangent in factored form: dL/dB of the
    balance is -nu_i (u_i - u_j), rank 2, and rg_gebhart_adjoint_factored solves K^T for its
    two left factors only. Against the full-dB chain (rg_temperatures_adjoint_sets ->
    rg_gebhart_adjoint) and the oracle's fp64 gradients of L = sum w o T."""
    rng = np.random.default_rng(44)
    N, S = 300, 3
    F, A = _consistent_F(N, rng)
    eps = rng.uniform(0.05, 0.9, (S, N))
    rho = 1 - eps
    Q = rng.uniform(0, 50, (S, N))
    wT = rng.standard_normal((S, N))
    Fd, ed, rd, Ad = _dev(F), _dev(eps), _dev(rho), _dev(A)
    B, _, _ = api.gebhart(rg_ctx, Fd, ed, rd, tol=1e-12)
    T = api.temperatures_sets(rg_ctx, Fd, B, ed, rd, Ad, _dev(Q), 3.0, tol=1e-13)
    (fa, fb), deps_T = api.temperatures_adjoint_sets(rg_ctx, Fd, B, ed, rd, Ad, 3.0, T, _dev(wT), tol=1e-13,
                                                      factored=True)
    dB, deps_T2 = api.temperatures_adjoint_sets(rg_ctx, Fd, B, ed, rd, Ad, 3.0, T, _dev(wT), tol=1e-13)
    # the factors reproduce the full cotangent
    full = torch.einsum("srn,srm->snm", fa, fb)
    assert (full - dB).abs().max().item() <= 1e-14 * dB.abs().max().item()
    assert torch.equal(deps_T, deps_T2)
    de_f, dr_f = api.gebhart_adjoint_factored(rg_ctx, Fd, ed, rd, B, fa, fb, tol=1e-12)
    de_full, dr_full = api.gebhart_adjoint(rg_ctx, Fd, ed, rd, B, dB, tol=1e-12)
    assert (de_f - de_full).abs().max().item() <= 1e-9 * de_full.abs().max().item()
    assert (dr_f - dr_full).abs().max().item() <= 1e-9 * dr_full.abs().max().item()
    for s in range(S):
        geo, gro = G.thermal_gradients(F, eps[s], rho[s], A, Q[s], 3.0, wT[s])
        g = (de_f[s] + deps_T[s]).cpu().numpy()
        assert np.abs(g - geo).max() <= 1e-8 * np.abs(geo).max()
        assert np.abs(dr_f[s].cpu().numpy() - gro).max() <= 1e-8 * np.abs(gro).max()


def test_temperature_sets_small_sat(rg_ctx):
    """The 2,048-face small satellite, two sets: the batched balance against the oracle."""
    w = synth.workload("small_sat", rays_scale=0.02)
    mesh = api.Mesh.from_synth(rg_ctx, w["mesh"])
    F = api.counts_to_F(rg_ctx, api.trace(rg_ctx, mesh, w["rays"], 0), _dev(w["rays"], torch.int64))
    A = mesh.face_areas()
    api.enforce_iterative(rg_ctx, F, _dev(A), tol=1e-12)
    N = F.shape[0]
    eps, rho = synth.optical_sets(N, 2, 0.05, 0.9, seed=40)
    Q = np.stack([synth.heat_loads(N, seed=3), synth.heat_loads(N, seed=4)])
    B, _, _ = api.gebhart(rg_ctx, F, _dev(eps), _dev(rho), tol=1e-12)
    T = api.temperatures_sets(rg_ctx, F, B, _dev(eps), _dev(rho), _dev(A), _dev(Q), 3.0, tol=1e-13)
    Bh = B.cpu().numpy()
    for s in range(2):
        To = G.temperatures(Bh[s], eps[s], A, Q[s], 3.0)
        assert np.abs(T[s].cpu().numpy() - To).max() <= 1e-10 * To.max()


# ------------------------------------------------------------------ least-squares optimum
def test_lsq_disc_example(rg_ctx):
    F1 = load_matrix("disc_F1_mcrt.txt")
    A = np.array([1.0, 4.0, 1.0, 4.0])
    for spva, name in ((False, "disc_F4_lsq_nnr.txt"), (True, "disc_F5_lsq_nnr_spva.txt")):
        Fd = _dev(F1)
        passes = api.enforce_lsq(rg_ctx, Fd, _dev(A), nnr=True, spva=spva)
        Fo, po = E.lsq_optimum(F1, A, nnr=True, spva=spva)
        got = Fd.cpu().numpy()
        assert np.abs(got - Fo).max() <= 1e-8
        assert passes == po
        assert np.abs(got - load_matrix(name)).max() <= 1e-6


def test_lsq_plates_config(rg_ctx):
    """512 sub-faces (config-sized) from GPU MCRT, LSQ + NNR + SPVA on the GPU and by the oracle."""
    m = synth.plates(16)
    rays = np.full(m.n_faces, 20000, np.int64)
    mesh = api.Mesh.from_synth(rg_ctx, m)
    F = api.counts_to_F(rg_ctx, api.trace(rg_ctx, mesh, rays, 0), _dev(rays, torch.int64))
    F0 = F.cpu().numpy()
    A = mesh.face_areas()
    api.enforce_lsq(rg_ctx, F, _dev(A), nnr=True, spva=True)
    Fo, _ = E.lsq_optimum(F0, A, nnr=True, spva=True)
    got = F.cpu().numpy()
    assert _rownorm_err(got, Fo) <= REL
    assert got.min() >= 0.0
    assert np.all(got[F0 == 0] == 0.0)
    assert np.abs(got.sum(axis=1) - 1).max() <= 1e-7
    eta = A[:, None] * got[:, :512]
    assert np.abs(eta - eta.T).max() <= 1e-7 * np.abs(eta).max()


def _banded_F(N, rng, band=384, extra=3):
    """A view-factor-like N x (N+1) matrix whose N x N block is non-zero only within `band`
    of the diagonal and in a few off-diagonal 512-wide squares: most 256 x 64 blocks of its
    slices are zero, as on the spacecraft (zero blocks skipped by the exact product)."""
    i = np.arange(N)
    M = np.abs(i[:, None] - i[None, :]) < band
    for _ in range(extra):
        a, b = rng.integers(0, N - 512, 2)
        M[a:a + 512, b:b + 512] = True
    F = np.zeros((N, N + 1))
    F[:, :N] = np.where(M, rng.random((N, N)) ** 3, 0.0)
    np.fill_diagonal(F[:, :N], 0.0)
    F[:, N] = 0.05 + 0.3 * rng.random(N)
    return F / F.sum(axis=1, keepdims=True)


def test_gebhart_block_sparse_vs_oracle(rg_ctx):
    """N = 4,608 (CTA-pair exact product) with mostly zero 256 x 64 blocks, and a first
    256-row tile whose faces see only the environment (no flagged block at all): the REFs and
    both gradients of a random cotangent against the oracle (Eq. B.11 and its adjoint)."""
    rng = np.random.default_rng(4608)
    N = 4608
    F = _banded_F(N, rng)
    F[:256, :N] = 0.0
    F[:256, N] = 1.0
    eps = rng.uniform(0.1, 0.9, N)
    rho = 1 - eps
    B, sweeps, _ = api.gebhart(rg_ctx, _dev(F), _dev(eps), _dev(rho), tol=1e-12)
    Bo = G.gebhart(F, eps, rho)
    got = B[0].cpu().numpy()
    assert np.all(got[:256, :N] == 0.0) and np.all(got[:256, N] == 1.0)  # faces that see nothing
    # the refinement's tolerance is normwise (max |R| / max |X|, and max |X| = 1 here)
    assert np.abs(got - Bo).max() <= 1e-10 * np.abs(Bo).max()
    assert np.all(np.abs(got - Bo).max(axis=1) <= 1e-8 * np.abs(Bo).max(axis=1))
    assert np.abs(got.sum(axis=1) - 1.0).max() <= 1e-10
    W = rng.standard_normal((N, N + 1))
    de, dr = api.gebhart_adjoint(rg_ctx, _dev(F), _dev(eps), _dev(rho), _dev(Bo), _dev(W), tol=1e-12)
    deo, dro = G.gebhart_adjoint(F, eps, rho, Bo, W)
    assert np.abs(de[0].cpu().numpy() - deo).max() <= REL * np.abs(deo).max()
    assert np.abs(dr[0].cpu().numpy() - dro).max() <= REL * np.abs(dro).max()
