"""Pins of the Gebhart / temperature / adjoint oracle: the printed parallel-plates
example (Sec. 6.3, Eq. 6.10-6.11, Table 6.2), REF identities (Eq. 4.3-4.5),
special cases with closed forms and finite differences."""
import numpy as np
import pytest

from oracle import enforce as E
from oracle import gebhart as G
from tests.conftest import load_matrix, load_table


def test_plates_B_matches_eq_6_11():
    F = load_matrix("plates_F.txt")
    eps = np.full(4, 0.5)
    B = G.gebhart(F, eps, 1 - eps)
    assert np.abs(B - load_matrix("plates_B.txt")).max() <= 5e-7


def test_gebhart_rows_match_printed_plates_B_and_the_full_solve():
    F = load_matrix("plates_F.txt")
    eps = np.full(4, 0.5)
    assert np.abs(G.gebhart_rows(F, eps, 1 - eps, [3, 1]) - load_matrix("plates_B.txt")[[3, 1]]).max() <= 5e-7
    rng = np.random.default_rng(4)
    F, _ = _consistent_F(40, rng)
    eps = rng.uniform(0.05, 0.9, 40)
    rows = [0, 17, 39]
    assert np.abs(G.gebhart_rows(F, eps, 1 - eps, rows) - G.gebhart(F, eps, 1 - eps)[rows]).max() <= 1e-14


def test_table_6_2_temperatures():
    F = load_matrix("plates_F.txt")
    t = load_table("plates_table_6_2.txt")
    eps = np.full(4, 0.5)
    area = np.ones(4)
    B = G.gebhart(F, eps, 1 - eps)
    nodes = np.array([0, 0, 1, 1])          # each plate is one node, both faces at one T
    T_bot, T_env = t["T_bottom_C"] + 273.15, t["T_env_C"] + 273.15
    eps_env = np.concatenate([eps, [1.0]])   # the environment is black
    GR_vf = G.SIGMA * eps[:, None] * eps_env[None, :] * area[:, None] * F      # Eq. 3.11
    GR_ref = G.conductances(B, eps, area)                                      # Eq. 4.2
    T_vf = G.steady_temperatures_fixed(GR_vf, {0: T_bot}, nodes, T_env=T_env)[1] - 273.15
    T_ref = G.steady_temperatures_fixed(GR_ref, {0: T_bot}, nodes, T_env=T_env)[1] - 273.15
    # the table is printed to 0.01 C (truncated)
    assert 0.0 <= T_vf - t["T_top_view_factors_C"] < 0.01
    assert 0.0 <= T_ref - t["T_top_refs_C"] < 0.01


def _consistent_F(N, rng):
    """Random F with reciprocity A_i F_ij = A_j F_ji and closure, open system."""
    A = rng.uniform(0.5, 2.0, N)
    S = rng.random((N, N))
    S = 0.3 * (S + S.T) / N
    np.fill_diagonal(S, 0.0)
    env = A - S.sum(axis=1)
    assert env.min() > 0
    return np.concatenate([S, env[:, None]], axis=1) / A[:, None], A


def test_ref_closure_and_reciprocity():
    rng = np.random.default_rng(1)
    N = 20
    F, A = _consistent_F(N, rng)
    eps = rng.uniform(0.1, 0.9, N)
    B = G.gebhart(F, eps, 1 - eps)
    assert np.abs(B.sum(axis=1) - 1).max() < 1e-13            # Eq. 4.3 with the env column
    R = (eps * A)[:, None] * B[:, :N]
    assert np.abs(R - R.T).max() < 1e-14                      # Eq. 4.4
    assert G.recursion_residual(F, eps, 1 - eps, B) < 1e-14   # Eq. 4.5 / B.6


def test_closed_system_closure():
    rng = np.random.default_rng(2)
    N = 10
    S = rng.random((N, N)); S = S + S.T; np.fill_diagonal(S, 0)
    A = S.sum(axis=1)                    # A_i F_ij = S_ij symmetric, rows of F sum to 1
    F = S / A[:, None]
    eps = rng.uniform(0.2, 0.9, N)
    B = G.gebhart(F, eps, 1 - eps)
    assert B.shape == (N, N)
    assert np.abs(B.sum(axis=1) - 1).max() < 1e-13


def test_black_surfaces_give_B_equal_E():
    rng = np.random.default_rng(3)
    F, _ = _consistent_F(7, rng)
    eps = rng.uniform(0.1, 0.9, 7)
    B = G.gebhart(F, eps, np.zeros(7))
    assert np.abs(B - G.e_matrix(F, eps)).max() < 1e-15
    assert np.array_equal(B[:, -1], F[:, -1])


def test_two_plates_reflection_series():
    # two facing faces (2, 3) exchanging only with each other and the environment:
    # energy leaving face 2 that comes back after one reflection at 3 and is absorbed at 2,
    # summed over the repeated round trips: B_22 = eps rho F23 F32 / (1 - rho^2 F23 F32)
    F = load_matrix("plates_F.txt")
    e, r = 0.3, 0.7
    B = G.gebhart(F, np.full(4, e), np.full(4, r))
    a, b = F[1, 2], F[2, 1]
    assert abs(B[1, 1] - e * r * a * b / (1 - r * r * a * b)) < 1e-15
    assert abs(B[1, 2] - e * a / (1 - r * r * a * b)) < 1e-15


def test_enforced_mcrt_gives_reciprocal_refs():
    F1 = load_matrix("disc_F1_mcrt.txt")
    A = np.array([1.0, 4.0, 1.0, 4.0])
    F6, _, _ = E.iterative(F1, A)
    eps = np.array([0.3, 0.6, 0.8, 0.5])
    B = G.gebhart(F6, eps, 1 - eps)
    R = (eps * A)[:, None] * B[:, :4]
    assert np.abs(R - R.T).max() < 1e-11
    assert np.abs(B.sum(axis=1) - 1).max() < 1e-12


def test_temperatures_special_cases():
    rng = np.random.default_rng(7)
    N = 9
    F, A = _consistent_F(N, rng)
    eps = rng.uniform(0.1, 0.9, N)
    B = G.gebhart(F, eps, 1 - eps)
    # no heat load: everything sits at the sink temperature
    T = G.temperatures(B, eps, A, np.zeros(N), 50.0)
    assert np.abs(T - 50.0).max() < 1e-9
    # energy balance: total load = total radiated to the environment
    Q = rng.uniform(0, 50, N)
    T = G.temperatures(B, eps, A, Q, 3.0)
    loss = np.sum(G.SIGMA * eps * A * B[:, N] * (T ** 4 - 3.0 ** 4))
    assert abs(loss - Q.sum()) < 1e-9 * Q.sum()
    # one isolated black node: sigma A (T^4 - Ts^4) = Q
    Bi = np.zeros((1, 2)); Bi[0, 1] = 1.0
    Ti = G.temperatures(Bi, np.ones(1), np.array([2.0]), np.array([100.0]), 3.0)
    assert abs(G.SIGMA * 2.0 * (Ti[0] ** 4 - 81.0) - 100.0) < 1e-9


@pytest.mark.parametrize("N", [3, 8])
def test_gebhart_adjoint_vs_central_differences(N):
    rng = np.random.default_rng(10 + N)
    F, _ = _consistent_F(N, rng)
    eps = rng.uniform(0.1, 0.9, N)
    rho = 1 - eps
    W = rng.standard_normal((N, N + 1))
    loss = lambda e, r: float(np.sum(W * G.gebhart(F, e, r)))  # noqa: E731
    de, dr = G.gebhart_adjoint(F, eps, rho, G.gebhart(F, eps, rho), W)
    fe = G.central_difference(lambda e: loss(e, rho), eps)
    fr = G.central_difference(lambda r: loss(eps, r), rho)
    assert np.abs(de - fe).max() <= 1e-6 * np.abs(fe).max()
    assert np.abs(dr - fr).max() <= 1e-6 * np.abs(fr).max()


def test_gebhart_adjoint_2x2_by_hand():
    # closed-form 2x2 case: F = [[0, a], [b, 0]] plus env; B_12 = e2 a / (1 - r1 r2 a b)
    a, b = 0.4, 0.3
    F = np.array([[0, a, 1 - a], [b, 0, 1 - b]])
    e = np.array([0.6, 0.7]); r = 1 - e
    Wb = np.zeros((2, 3)); Wb[0, 1] = 1.0         # L = B_12
    de, dr = G.gebhart_adjoint(F, e, r, G.gebhart(F, e, r), Wb)
    D = 1 - r[0] * r[1] * a * b
    assert abs(de[1] - a / D) < 1e-14 and abs(de[0]) < 1e-14
    assert abs(dr[0] - e[1] * a * r[1] * a * b / D ** 2) < 1e-14
    assert abs(dr[1] - e[1] * a * r[0] * a * b / D ** 2) < 1e-14


def test_thermal_adjoint_vs_central_differences():
    rng = np.random.default_rng(21)
    N = 6
    F, A = _consistent_F(N, rng)
    eps = rng.uniform(0.1, 0.9, N)
    rho = 1 - eps
    Q = rng.uniform(0, 50, N)
    w = rng.standard_normal(N)

    def loss(e, r):
        B = G.gebhart(F, e, r)
        return float(np.sum(w * G.temperatures(B, e, A, Q, 3.0)))

    ge, gr = G.thermal_gradients(F, eps, rho, A, Q, 3.0, w)
    fe = G.central_difference(lambda e: loss(e, rho), eps)
    fr = G.central_difference(lambda r: loss(eps, r), rho)
    assert np.abs(ge - fe).max() <= 1e-6 * np.abs(fe).max()
    assert np.abs(gr - fr).max() <= 1e-6 * np.abs(fr).max()
