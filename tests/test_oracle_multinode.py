"""Pins of the multi-node relations (Ch. 5): closed forms for aggregated plates and the
closure/reciprocity preservation proved in Sec. 5.3 (Eq. 5.30-5.36)."""
import numpy as np

from oracle import gebhart as G
from oracle import multinode as MN
from tests import closed_forms as cf


def _plate_subfaces(n):
    """Exact sub-face view factors between two facing unit plates 0.5 apart, n x n each."""
    cells = [(i / n, (i + 1) / n, j / n, (j + 1) / n) for j in range(n) for i in range(n)]
    N = 2 * n * n
    F = np.zeros((N, N + 1))
    for a, (x1, x2, y1, y2) in enumerate(cells):
        for b, (u1, u2, v1, v2) in enumerate(cells):
            f = cf.parallel_rectangles(x1, x2, y1, y2, u1, u2, v1, v2, 0.5)
            F[a, n * n + b] = f
            F[n * n + b, a] = f            # equal areas: reciprocity is symmetry
    F[:, N] = 1.0 - F[:, :N].sum(axis=1)
    return F


def test_aggregated_subfaces_equal_whole_plate_closed_form():
    n = 4
    F = _plate_subfaces(n)
    S = np.full(2 * n * n, 1.0 / (n * n))
    grp = np.repeat([0, 1], n * n)
    Fs, S_surf = MN.surface_view_factors(F, S, grp, 2)
    whole = cf.parallel_opposed(1, 1, 0.5)
    assert abs(whole - 0.415253) < 1e-6
    assert abs(Fs[0, 1] - whole) < 1e-12 and abs(Fs[1, 0] - whole) < 1e-12
    assert Fs[0, 0] == 0 and abs(Fs[0, 2] - (1 - whole)) < 1e-12
    assert np.allclose(S_surf, 1.0)


def test_aggregation_preserves_closure_and_reciprocity():
    rng = np.random.default_rng(0)
    N = 24
    S = rng.uniform(0.5, 2.0, N)
    X = rng.random((N, N)); X = 0.4 * (X + X.T) / N
    env = S - X.sum(axis=1)
    F = np.concatenate([X, env[:, None]], axis=1) / S[:, None]   # S_i F_ij symmetric, closed rows
    grp = rng.integers(0, 5, N)
    grp[:5] = np.arange(5)
    Fs, Ss = MN.surface_view_factors(F, S, grp, 5)
    assert np.abs(Fs.sum(axis=1) - 1).max() < 1e-14                  # Eq. 5.32
    R = Ss[:, None] * Fs[:, :5]
    assert np.abs(R - R.T).max() < 1e-14                              # Eq. 5.35


def test_node_view_factors_cases():
    rng = np.random.default_rng(1)
    N = 5
    Fs = rng.random((N, 2, N, 2)) * 0.05
    Fe = rng.random((N, 2)) * 0.1
    C = np.array([2, 2, 1, 2, 1])
    Fs[C == 1, 1] = 0.0                   # one-faced nodes emit nothing from side B
    Fe[C == 1, 1] = 0.0
    Fn = MN.node_view_factors(Fs, Fe, C)
    i = 0
    assert abs(Fn[i, 3] - 0.5 * Fs[i, :, 3, :].sum()) < 1e-15          # Eq. 5.12
    assert abs(Fn[2, 4] - Fs[2, 0, 4, :].sum()) < 1e-15                # Eq. 5.15
    assert abs(Fn[2, N] - Fe[2, 0]) < 1e-15                            # Eq. 5.16
    f, fe = MN.view_fractions(Fs, Fe)
    assert np.allclose(f.sum(axis=(1, 3)), 1.0)                        # Eq. 5.27 sums to 1
    assert np.allclose(fe.sum(axis=1), 1.0)


def _sided_system(rng, N, C):
    """Side-resolved F [2N, 2N+1] of nodes with C_i faces of area S_i each: S F^{X->Y}_ij
    symmetric in (iX, jY) (Eq. 5.34), closed rows (Eq. 5.30), zero rows for the missing
    side B of one-faced nodes."""
    S = rng.uniform(0.5, 2.0, N)
    Sa = np.repeat(S, 2)
    active = np.ones(2 * N, bool)
    active[1::2] = np.asarray(C) == 2
    X = rng.random((2 * N, 2 * N)) * (rng.random((2 * N, 2 * N)) < 0.6)
    X = (X + X.T) * np.outer(active, active)
    np.fill_diagonal(X, 0.0)
    X *= 0.7 * Sa.min() / X.sum(axis=1).max()
    env = np.where(active, Sa - X.sum(axis=1), 0.0)
    F = np.concatenate([X, env[:, None]], axis=1) / Sa[:, None]
    return F, S, active


def test_sided_surface_aggregation_closed_form_and_relations():
    # the stacked-plates geometry of the side-resolved MCRT pins, split into n x n
    # sub-faces: aggregating the exact sub-face factors gives the whole-square factor
    n, gap = 3, 0.5
    cells = [(i / n, (i + 1) / n, j / n, (j + 1) / n) for j in range(n) for i in range(n)]
    k = n * n
    F2 = np.zeros((6 * k, 6 * k + 1))          # 3 plates x k sub-faces, sides A (up) / B (down)
    for a, (x1, x2, y1, y2) in enumerate(cells):
        for b, (u1, u2, v1, v2) in enumerate(cells):
            f = cf.parallel_rectangles(x1, x2, y1, y2, u1, u2, v1, v2, gap)
            for lo in (0, 1):                  # plate lo's side A faces plate lo+1's side B
                F2[2 * (lo * k + a), 2 * ((lo + 1) * k + b) + 1] = f
                F2[2 * ((lo + 1) * k + b) + 1, 2 * (lo * k + a)] = f
    F2[:, -1] = 1.0 - F2[:, :-1].sum(axis=1)
    S = np.full(3 * k, 1.0 / k)
    grp = np.repeat([0, 1, 2], k)
    Fs, S_surf = MN.surface_view_factors_sided(F2, S, grp, 3)
    whole = cf.parallel_opposed(1, 1, gap)
    assert abs(Fs[0, 3] - whole) < 1e-12 and abs(Fs[3, 0] - whole) < 1e-12   # bottom A <-> middle B
    assert abs(Fs[2, 5] - whole) < 1e-12 and abs(Fs[5, 2] - whole) < 1e-12   # middle A <-> top B
    assert abs(Fs[1, 6] - 1.0) < 1e-14 and abs(Fs[4, 6] - 1.0) < 1e-14
    # Eq. 5.32 and Eq. 5.35 on a random reciprocal, closed side-resolved system
    rng = np.random.default_rng(4)
    F, S, _ = _sided_system(rng, 20, np.full(20, 2))
    grp = rng.integers(0, 4, 20)
    grp[:4] = np.arange(4)
    Fs, Ss = MN.surface_view_factors_sided(F, np.repeat(S, 1), grp, 4)
    assert np.abs(Fs.sum(axis=1) - 1).max() < 1e-14
    R = np.repeat(Ss, 2)[:, None] * Fs[:, :8]
    assert np.abs(R - R.T).max() < 1e-14


def test_node_couplings_equal_faces_and_one_faced_nodes():
    rng = np.random.default_rng(5)
    N = 6
    C = np.array([2, 1, 2, 2, 1, 2])
    F, S, active = _sided_system(rng, N, C)
    B2 = G.gebhart(F, np.where(active, 0.6, 0.0), np.where(active, 0.4, 0.0))
    eps2 = np.repeat(rng.uniform(0.2, 0.9, N), 2)               # eps^A = eps^B on every node
    eps2[1::2][C == 1] = 0.0
    GR, Bn, epn = MN.node_couplings(B2, eps2, S, C)
    mask = Bn > 0
    assert np.abs(epn[mask] - np.repeat(eps2[0::2], N + 1).reshape(N, N + 1)[mask]).max() < 1e-14   # Eq. C.4
    # a one-faced node: eps_ij = eps^A_i and GR_ij = eps^A_i S_i (B^{AA} + B^{AB}) (Eq. C.3, C = 1)
    eps2 = rng.uniform(0.2, 0.9, 2 * N)
    GR, Bn, epn = MN.node_couplings(B2, eps2, S, C)
    i = 1
    row = B2[2 * i, :2 * N].reshape(N, 2).sum(axis=1)
    assert np.allclose(GR[i, :N], eps2[2 * i] * S[i] * row, rtol=1e-14, atol=0)
    assert np.allclose(epn[i][Bn[i] > 0], eps2[2 * i], rtol=1e-14)


def test_node_couplings_two_routes_agree_and_keep_closure_and_reciprocity():
    rng = np.random.default_rng(6)
    N = 9
    C = np.full(N, 2)
    F, S, _ = _sided_system(rng, N, C)
    eps2 = rng.uniform(0.1, 0.9, 2 * N)
    B2 = G.gebhart(F, eps2, 1 - eps2)
    GR, Bn, epn = MN.node_couplings(B2, eps2, S, C)
    # Eq. C.3 (GR from the faces) against Eq. C.1 with the node emissivity of Eq. C.4
    assert np.abs(GR - epn * (C * S)[:, None] * Bn).max() <= 1e-14 * GR.max()
    # the faces' REFs close (Eq. 4.3), so each node's couplings add up to its emitters
    assert np.abs(GR.sum(axis=1) - S * (eps2[0::2] + eps2[1::2])).max() < 1e-13
    # face-level reciprocity (Eq. 4.4) makes the node couplings symmetric
    assert np.abs(GR[:, :N] - GR[:, :N].T).max() < 1e-14 * GR.max()
    assert not np.allclose(epn[:, :N], epn[:, :N].T)             # the emissivities themselves are not
