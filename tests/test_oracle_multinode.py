"""Pins of the multi-node relations (Ch. 5): closed forms for aggregated plates and the
closure/reciprocity preservation proved in Sec. 5.3 (Eq. 5.30-5.36)."""
import numpy as np

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
