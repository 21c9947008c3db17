"""Multi-node surface relations (Ch. 5, Eq. 5.28-5.29) and node optical properties (App. C).

TEST INFRASTRUCTURE ONLY (see the package docstring). Plain numpy, fp64.

Side-resolved matrices use the layout of the side-resolved MCRT counts: row 2i+X is side
X (0 = A, 1 = B) of face i, column 2j+Y side Y of face j, column 2N the environment.
``split_sides`` turns that into the 4-index form F[i, X, j, Y] used below.
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


def split_sides(M2):
    """[2N, 2N+1] side-resolved layout -> (M[i, X, j, Y], M_env[i, X])."""
    M2 = np.asarray(M2, np.float64)
    N = M2.shape[0] // 2
    return M2[:, :2 * N].reshape(N, 2, N, 2), M2[:, 2 * N].reshape(N, 2)


def surface_view_factors_sided(F2, sub_area, sub_to_surf, n_surf):
    """Side-resolved surface view factors from sub-surface ones (Eq. 5.6-5.7, first two
    lines of Eq. 5.28): F^{X->Y}_nm = sum_i sum_j F^{X->Y}_{n_i m_j} S_{n_i} / S_n and
    F^{X->inf}_n = sum_i F^{X->inf}_{n_i} S_{n_i} / S_n, in the [2n, 2n+1] layout.
    Written as plain loops."""
    Fs, Fe = split_sides(F2)
    n_sub = Fs.shape[0]
    S = np.asarray(sub_area, np.float64)
    grp = np.asarray(sub_to_surf)
    S_surf = np.zeros(n_surf)
    for i in range(n_sub):
        S_surf[grp[i]] += S[i]
    out = np.zeros((2 * n_surf, 2 * n_surf + 1))
    for i in range(n_sub):
        n = grp[i]
        w = S[i] / S_surf[n]
        for X in range(2):
            for j in range(n_sub):
                for Y in range(2):
                    out[2 * n + X, 2 * grp[j] + Y] += Fs[i, X, j, Y] * w
            out[2 * n + X, 2 * n_surf] += Fe[i, X] * w
    return out, S_surf


def node_couplings(B2, eps2, face_area, n_faces_per_node):
    """Radiative couplings and emissivities of nodes with two optically different faces (App. C).

    B2: side-resolved REFs [2N, 2N+1] (the Gebhart factors of the system whose faces are
    the nodes' sides); eps2[2i+X] = eps^X_i; face_area[i] = S_i, the area of each face of
    node i; n_faces_per_node[i] = C_i (1: side B of node i emits nothing).
    Returns GR [N, N+1] with GR_ij = S_i * sum_X eps^X_i sum_Y B^{X->Y}_{ij} (Eq. C.3, last
    line; column N: the environment, sum over X only), the node REFs B [N, N+1] with
    C_i B_ij = sum_{X,Y} B^{X->Y}_{ij} (Eq. C.3, first line, as Eq. 5.17), and the node
    emissivity of each pair eps_ij = eps^A_i (f^{AA} + f^{AB}) + eps^B_i (f^{BA} + f^{BB})
    (Eq. C.4) from the view fractions of B (Eq. 5.27), 0 where B_ij = 0.
    """
    Bs, Be = split_sides(B2)
    N = Bs.shape[0]
    e = np.asarray(eps2, np.float64).reshape(N, 2)
    S = np.asarray(face_area, np.float64)
    C = np.asarray(n_faces_per_node, np.float64)
    GR = np.zeros((N, N + 1))
    GR[:, :N] = S[:, None] * (e[:, 0, None] * Bs[:, 0].sum(axis=2) + e[:, 1, None] * Bs[:, 1].sum(axis=2))
    GR[:, N] = S * (e[:, 0] * Be[:, 0] + e[:, 1] * Be[:, 1])
    Bn = node_view_factors(Bs, Be, C)
    f, fe = view_fractions(Bs, Be)
    eps_n = np.zeros((N, N + 1))
    eps_n[:, :N] = e[:, 0, None] * (f[:, 0, :, 0] + f[:, 0, :, 1]) + e[:, 1, None] * (f[:, 1, :, 0] + f[:, 1, :, 1])
    eps_n[:, N] = e[:, 0] * fe[:, 0] + e[:, 1] * fe[:, 1]
    return GR, Bn, eps_n
