"""Pins of the enforcement oracle: the thesis's printed two-disc example (Sec. 6.2,
Eq. 6.3-6.9, Table 6.1) and the invariants the enforcers must establish."""
import numpy as np
import pytest

from oracle import enforce as E
from tests.conftest import load_matrix, load_table

AREAS = np.array([1.0, 4.0, 1.0, 4.0])   # disc radii 1:2 and back faces (Eq. 6.1-6.3)


@pytest.fixture(scope="module")
def F1():
    return load_matrix("disc_F1_mcrt.txt")


@pytest.fixture(scope="module")
def Fa():
    return load_matrix("disc_F_analytical.txt")


def test_closure_only_matches_eq_6_5(F1):
    F2 = E.closure_open(F1, AREAS)
    assert np.abs(F2 - load_matrix("disc_F2_closure.txt")).max() <= 5e-7


def test_reciprocity_matches_eq_6_6(F1):
    F3 = E.reciprocity(F1, AREAS, kappa=0.5)
    assert np.abs(F3 - load_matrix("disc_F3_reciprocity.txt")).max() <= 5e-7
    rows = load_table("disc_iterations.txt")
    assert abs(F3[0].sum() - rows["rowsum_F3_row1"]) < 5e-6
    assert abs(F3[1].sum() - rows["rowsum_F3_row2"]) < 5e-6


def test_iterative_matches_eq_6_9(F1):
    F6, it, ok = E.iterative(F1, AREAS, tol=1e-12)
    assert ok
    printed = load_matrix("disc_F6_iterative.txt")
    assert np.abs(F6 - printed).max() <= 1e-6
    # after the 13 iterations the text reports, the iterate already matches to print precision
    F13, _, _ = E.iterative(F1, AREAS, tol=0.0, maxit=int(load_table("disc_iterations.txt")["iterations"]))
    assert np.abs(F13 - printed).max() <= 1e-6
    # invariants: exact closure (the last step is closure), reciprocity to tol
    assert np.allclose(F6.sum(axis=1), 1.0, atol=1e-14)
    eta = E.exchange(F6, AREAS)[:, :4]
    assert np.abs(eta - eta.T).max() <= 1e-11


def test_lsq_nnr_matches_eq_6_7(F1):
    F4, passes = E.lsq_optimum(F1, AREAS, nnr=True, spva=False)
    # printed to 6 decimals from an unrounded MCRT matrix: agreement to 1e-6
    assert np.abs(F4 - load_matrix("disc_F4_lsq_nnr.txt")).max() <= 1e-6
    assert passes > 1                       # NNR had negatives to remove
    assert F4.min() >= 0.0


def test_lsq_nnr_spva_matches_eq_6_8(F1):
    F5, _ = E.lsq_optimum(F1, AREAS, nnr=True, spva=True)
    assert np.abs(F5 - load_matrix("disc_F5_lsq_nnr_spva.txt")).max() <= 1e-6
    assert np.all(F5[F1 == 0] == 0.0)       # SPVA keeps the MCRT zeros


def test_table_6_1_mae(F1, Fa):
    t = load_table("disc_table_6_1_mae.txt")
    got = {
        "none": E.mae(F1, Fa),
        "closure": E.mae(E.closure_open(F1, AREAS), Fa),
        "reciprocity": E.mae(E.reciprocity(F1, AREAS), Fa),
        "lsq_nnr": E.mae(E.lsq_optimum(F1, AREAS, spva=False)[0], Fa),
        "lsq_nnr_spva": E.mae(E.lsq_optimum(F1, AREAS, spva=True)[0], Fa),
        "iterative": E.mae(E.iterative(F1, AREAS)[0], Fa),
    }
    # printed to 2-3 significant digits from matrices rounded to 6 decimals
    for k, v in got.items():
        assert abs(v - t[k]) <= 3e-7, (k, v, t[k])


def test_literal_eq_3_52_equals_projection(F1):
    for spva in (False, True):
        a, _ = E.lsq_optimum(F1, AREAS, spva=spva, literal=True)
        b, _ = E.lsq_optimum(F1, AREAS, spva=spva, literal=False)
        assert np.abs(a - b).max() < 1e-12


def test_restriction_matrix_shape_and_rows():
    N = 4
    A, b = E.restriction_system(N, AREAS, space="eta")
    assert A.shape == (N + N * (N - 1) // 2, N * (N + 1))   # Eq. 3.41-3.43
    D = np.asarray(A.todense())
    # first reciprocity row of Eq. 3.43: +1 at eta_12 (col 1), -1 at eta_21 (col 5)
    assert D[N, 1] == 1 and D[N, 5] == -1 and np.count_nonzero(D[N]) == 2
    assert np.all(D[:N].sum(axis=1) == N + 1)
    assert np.allclose(b[:N], AREAS) and np.all(b[N:] == 0)


def _random_F(N, rng, zeros=0.2):
    F = rng.random((N, N + 1))
    F[rng.random((N, N + 1)) < zeros] = 0.0
    np.fill_diagonal(F[:, :N], 0.0)
    F[:, N] += 0.05
    return F / F.sum(axis=1, keepdims=True)


def test_lsq_invariants_random():
    rng = np.random.default_rng(4)
    N = 12
    F = _random_F(N, rng)
    A = rng.uniform(0.5, 2.0, N)
    for spva in (False, True):
        Fh, _ = E.lsq_optimum(F, A, nnr=True, spva=spva)
        assert Fh.min() >= 0
        assert np.abs(Fh.sum(axis=1) - 1).max() < 1e-12
        eta = A[:, None] * Fh[:, :N]
        assert np.abs(eta - eta.T).max() < 1e-12
        if spva:
            assert np.all(Fh[F == 0] == 0)
    # without NNR the projection is the closest point: any feasible point is farther
    Fh, _ = E.lsq_optimum(F, A, nnr=False, spva=False)
    Fi, _, _ = E.iterative(F, A)
    assert np.linalg.norm(Fh - F) <= np.linalg.norm(Fi - F) + 1e-12


def test_iterative_invariants_random():
    rng = np.random.default_rng(5)
    N = 30
    F = _random_F(N, rng)
    A = rng.uniform(0.5, 2.0, N)
    Fh, it, ok = E.iterative(F, A, tol=1e-13)
    assert ok and it > 1
    assert np.abs(Fh.sum(axis=1) - 1).max() < 1e-13
    eta = A[:, None] * Fh[:, :N]
    assert np.abs(eta - eta.T).max() < 1e-12 * A.max()
    assert Fh.min() >= 0          # averaging and positive row scaling keep signs
    both_zero = (F[:, :N] == 0) & (F[:, :N].T == 0)
    assert np.all(Fh[:, :N][both_zero] == 0)      # pairs that MCRT never linked stay 0


def test_already_consistent_matrix_is_a_fixed_point():
    # symmetric eta with row sums Omega: every enforcer leaves it alone
    rng = np.random.default_rng(6)
    N = 8
    A = rng.uniform(0.5, 2.0, N)
    S = rng.random((N, N)); S = 0.05 * (S + S.T)
    env = A - S.sum(axis=1)
    assert env.min() > 0
    F = np.concatenate([S, env[:, None]], axis=1) / A[:, None]
    assert np.abs(E.iterative(F, A)[0] - F).max() < 1e-14
    assert np.abs(E.lsq_optimum(F, A)[0] - F).max() < 1e-12
    assert np.abs(E.reciprocity(F, A) - F).max() < 1e-15
    assert np.abs(E.closure_open(F, A) - F).max() < 1e-15


def test_kappa_variants():
    rays = np.array([100, 100, 100.0])
    om = np.array([1.0, 1.0, 1.0])
    # equal Omega/N -> Y = 0 -> kappa = 1/2 (Eq. 3.21-3.22)
    assert np.allclose(E.kappa_triangulation(rays, om), 0.5)
    # Omega_j/N_j >> Omega_i/N_i -> Y -> 1 -> kappa -> 1 (keep the better-sampled side)
    k = E.kappa_triangulation(np.array([1e6, 1.0]), np.array([1.0, 1.0]))
    assert k[0, 1] > 0.99 and abs(k[0, 1] + k[1, 0] - 1) < 1e-12
    # fractional variance: kappa_ij + kappa_ji = 1 and the minimum-variance weight
    F = np.array([[0, 0.3, 0.7], [0.2, 0, 0.8]])
    kf = E.kappa_fractional_variance(F, [1000, 4000], [1.0, 1.5])
    assert abs(kf[0, 1] + kf[1, 0] - 1) < 1e-12
    v01 = 1.0 ** 2 * (1 - 0.3) / (1000 * 0.3)
    v10 = 1.5 ** 2 * (1 - 0.2) / (4000 * 0.2)
    assert abs(kf[0, 1] - v10 / (v01 + v10)) < 1e-12


def test_kappa_triangulation_pins():
    rng = np.random.default_rng(11)
    N = 12
    rays = rng.integers(100, 10000, N).astype(np.float64)
    om = rng.uniform(0.2, 3.0, N)
    k = E.kappa_triangulation(rays, om)
    # Y_ji = -Y_ij (Eq. 3.22), so the two weights of a pair add up to one
    assert np.abs(k + k.T - 1.0).max() < 1e-15
    assert np.all(np.diag(k) == 0.5)
    # with the exponent n = 1, Eq. 3.21 collapses to r_j / (r_i + r_j), r = Omega / N
    r = om / rays
    k1 = E.kappa_triangulation(rays, om, n=1.0)
    assert np.abs(k1 - r[None, :] / (r[:, None] + r[None, :])).max() < 1e-14
    # n -> 0 keeps only the sign of Y: all weight on eta_ij where Omega_j/N_j > Omega_i/N_i
    k0 = E.kappa_triangulation(rays, om, n=1e-12)
    target = np.where(r[None, :] > r[:, None], 1.0, np.where(r[None, :] < r[:, None], 0.0, 0.5))
    assert np.abs(k0 - target).max() < 1e-9


def test_kappa_fractional_variance_pins():
    rng = np.random.default_rng(12)
    N = 10
    rays = rng.integers(1000, 100000, N).astype(np.float64)
    om = rng.uniform(0.5, 2.0, N)
    F = _random_F(N, rng, zeros=0.0)
    k = E.kappa_fractional_variance(F, rays, om)
    # Eq. 3.23 in its exchange-coefficient form: sigma_ij = z Omega_i sqrt((Omega_i - eta_ij) / (N_i eta_ij))
    eta = om[:, None] * F[:, :N]
    with np.errstate(divide="ignore", invalid="ignore"):
        sig2 = (1.96 * om[:, None]) ** 2 * (om[:, None] - eta) / (rays[:, None] * eta)
    off = ~np.eye(N, dtype=bool)

    def var(kk):  # Eq. 3.24
        return kk ** 2 * sig2 + (1 - kk) ** 2 * sig2.T

    # Eq. 3.25 minimises Eq. 3.24: moving kappa either way raises the estimator variance
    for d in (1e-3, -1e-3):
        assert np.all(var(k + d)[off] > var(k)[off])
    assert np.abs(k + k.T - 1.0)[off].max() < 1e-15
    # z cancels
    assert np.abs(E.kappa_fractional_variance(F, rays, om, z=3.0) - k).max() < 1e-15
    # a zero estimate has infinite variance: the other side is taken; both zero -> 1/2
    F0 = F.copy()
    F0[0, 1] = 0.0
    F0[2, 3] = F0[3, 2] = 0.0
    k0 = E.kappa_fractional_variance(F0, rays, om)
    assert k0[0, 1] == 0.0 and k0[1, 0] == 1.0
    assert k0[2, 3] == 0.5 and k0[3, 2] == 0.5


def test_iterative_with_kappa_weights():
    rng = np.random.default_rng(13)
    N = 25
    F = _random_F(N, rng)
    A = rng.uniform(0.5, 2.0, N)
    rays = rng.integers(1000, 50000, N)
    # constant 1/2 weights are the default enforcer
    Fh, it, _ = E.iterative(F, A, tol=1e-13)
    Fk, itk, _ = E.iterative(F, A, tol=1e-13, kappa=np.full((N, N), 0.5))
    assert it == itk and np.array_equal(Fh, Fk)
    # variance weights: closure and reciprocity still hold at the fixed point
    K = E.kappa_fractional_variance(F, rays, A)
    Fv, itv, ok = E.iterative(F, A, tol=1e-13, kappa=K)
    assert ok
    assert np.abs(Fv.sum(axis=1) - 1).max() < 1e-13
    eta = A[:, None] * Fv[:, :N]
    assert np.abs(eta - eta.T).max() < 1e-12 * A.max()
    assert np.abs(Fv - Fh).max() > 1e-6          # the weights change the result
