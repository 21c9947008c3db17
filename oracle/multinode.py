"""Multi-node surface relations (Ch. 5, Eq. 5.28-5.29).

TEST INFRASTRUCTURE ONLY (see the package docstring). Plain numpy, fp64.
"""
from __future__ import annotations

import numpy as np


def surface_view_factors(F_sub, sub_area, sub_to_surf, n_surf):
    """Surface view factors from sub-surface view factors (Eq. 5.6-5.7).

    F_nm = sum_{i in n} sum_{j in m} F_{n_i m_j} S_{n_i} / S_n, and
    F_n,inf = sum_{i in n} F_{n_i,inf} S_{n_i} / S_n. Written as plain loops.
    """
    F_sub = np.asarray(F_sub, np.float64)
    n_sub = F_sub.shape[0]
    S = np.asarray(sub_area, np.float64)
    grp = np.asarray(sub_to_surf)
    S_surf = np.zeros(n_surf)
    for i in range(n_sub):
        S_surf[grp[i]] += S[i]
    out = np.zeros((n_surf, n_surf + 1))
    for i in range(n_sub):
        n = grp[i]
        w = S[i] / S_surf[n]
        for j in range(n_sub):
            out[n, grp[j]] += F_sub[i, j] * w
        out[n, n_surf] += F_sub[i, n_sub] * w
    return out, S_surf


def node_view_factors(F_sides, F_env_sides, n_faces_per_node):
    """Node view factors from side-resolved sub-surface view factors (Eq. 5.17).

    F_sides[i, X, j, Y] = F^{X->Y}_{n_i m_j}; F_env_sides[i, X] = F^{X->inf}_{n_i}; C_n = number
    of faces of node i (1 or 2; a one-faced node has zeros on side B).
    """
    Fs = np.asarray(F_sides, np.float64)
    Fe = np.asarray(F_env_sides, np.float64)
    C = np.asarray(n_faces_per_node, np.float64)
    N = Fs.shape[0]
    out = np.zeros((N, N + 1))
    out[:, :N] = Fs.sum(axis=(1, 3)) / C[:, None]
    out[:, N] = Fe.sum(axis=1) / C
    return out


def view_fractions(F_sides, F_env_sides):
    """View fractions f^{X->Y} (Eq. 5.27/5.29); 0 where the pair exchanges nothing."""
    Fs = np.asarray(F_sides, np.float64)
    Fe = np.asarray(F_env_sides, np.float64)
    tot = Fs.sum(axis=(1, 3), keepdims=True)
    tot_e = Fe.sum(axis=1, keepdims=True)
    with np.errstate(invalid="ignore", divide="ignore"):
        f = np.where(tot > 0, Fs / tot, 0.0)
        fe = np.where(tot_e > 0, Fe / tot_e, 0.0)
    return f, fe
