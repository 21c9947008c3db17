"""Closure and reciprocity enforcement of MCRT view factors (Sec. 3.5.3-3.5.5, App. A).

TEST INFRASTRUCTURE ONLY (see the package docstring). Plain numpy/scipy, fp64.

Matrices are N x (N+1): column N is the environment (Sec. 2.4.12). ``omega`` is
Omega_i (= A_i for view factors, eps_i*A_i for REFs, Sec. 4.2.3).

Readings of the text taken here (the paper is silent or garbled there):
* reciprocity weight kappa = 1/2 by default: the printed F^(3) and F^(6) of the
  disc example (Eq. 6.6, 6.9) are reproduced only with equal weights;
* Eq. 3.40 prints eta-hat in the numerator of lambda_i; substituting Eq. 3.39
  into g_i = 0 gives eta, so lambda_i = (Omega_i - sum_j eta_ij) / sum_j w_ij;
* the least-squares optimum works on F with restriction rows sum_j F_ij = 1 and
  A_i F_ij - A_j F_ji = 0 (``space="F"``), which reproduces the printed F^(4)
  and F^(5) (Eq. 6.7, 6.8); ``space="eta"`` is the literal eta-space statement
  (rows of ones, c_C = Omega, +-1 reciprocity rows) and is kept for comparison;
* the iterative enforcer stops when both the reciprocity defect of the previous
  iterate and the closure defect after symmetrisation are <= tol * max(Omega).
"""
from __future__ import annotations

import numpy as np
import scipy.linalg
import scipy.sparse
import scipy.sparse.linalg


def exchange(F, omega):
    """eta_ij = Omega_i * F_ij (Eq. 3.18)."""
    return np.asarray(omega, np.float64)[:, None] * np.asarray(F, np.float64)


def from_exchange(eta, omega):
    return np.asarray(eta, np.float64) / np.asarray(omega, np.float64)[:, None]


def kappa_triangulation(rays, omega, n=0.4):
    """Matrix-triangulation weights kappa_ij (Eq. 3.21-3.22)."""
    r = np.asarray(omega, np.float64) / np.asarray(rays, np.float64)
    Y = (r[None, :] - r[:, None]) / (r[None, :] + r[:, None])
    return 0.5 * (1.0 + np.sign(Y) * np.abs(Y) ** n)


def kappa_fractional_variance(F, rays, omega, z=1.96):
    """Fractional-variance weights (Eq. 3.23-3.25) on the N x N block.

    sigma^2_ij = z^2 Omega_i^2 (1 - F_ij) / (N_i F_ij); a zero estimate has infinite
    variance, so the other side is taken; both zero -> kappa = 1/2 (nothing to average).
    """
    F = np.asarray(F, np.float64)
    N = F.shape[0]
    Fn = F[:, :N]
    om = np.asarray(omega, np.float64)
    nr = np.asarray(rays, np.float64)
    with np.errstate(divide="ignore", invalid="ignore"):
        var = z * z * om[:, None] ** 2 * (1.0 - Fn) / (nr[:, None] * Fn)
    var = np.where(Fn > 0, var, np.inf)
    vt = var.T
    kappa = np.full((N, N), 0.5)
    both_inf = np.isinf(var) & np.isinf(vt)
    one_inf = np.isinf(var) & ~np.isinf(vt)
    other_inf = ~np.isinf(var) & np.isinf(vt)
    fin = ~np.isinf(var) & ~np.isinf(vt)
    with np.errstate(invalid="ignore", divide="ignore"):
        kappa[fin] = (vt[fin] / (var[fin] + vt[fin]))
    kappa[one_inf] = 0.0
    kappa[other_inf] = 1.0
    kappa[both_inf] = 0.5
    return kappa


def reciprocity(F, omega, kappa=0.5):
    """Reciprocity on the N x N block: eta-hat_ij = kappa eta_ij + (1-kappa) eta_ji (Eq. 3.20).

    The environment column is left as it is (Sec. 3.5.3, open systems).
    """
    F = np.asarray(F, np.float64)
    N = F.shape[0]
    eta = exchange(F, omega)
    k = np.broadcast_to(np.asarray(kappa, np.float64), (N, N))
    out = eta.copy()
    out[:, :N] = k * eta[:, :N] + (1.0 - k) * eta[:, :N].T
    return from_exchange(out, omega)


def closure_open(F, omega):
    """Least-squares smoothing for open systems with w_ij = eta_ij (Eq. 3.36-3.40).

    lambda_i = (Omega_i - sum_j eta_ij) / sum_j w_ij and eta-hat_ij = eta_ij + w_ij lambda_i,
    which with w = eta is a scaling of row i by Omega_i / sum_j eta_ij.
    """
    F = np.asarray(F, np.float64)
    om = np.asarray(omega, np.float64)
    eta = exchange(F, om)
    w = eta
    lam = (om - eta.sum(axis=1)) / w.sum(axis=1)
    return from_exchange(eta + w * lam[:, None], om)


def iterative(F, omega, tol=1e-12, maxit=10000, kappa=0.5):
    """Iterative closure + reciprocity enforcer for open systems (Sec. 3.5.5).

    Each iteration: reciprocity on the N x N block (Eq. 3.20) with the environment
    column carried over from the previous iterate, then open-system least-squares
    closure (Eq. 3.39-3.40, w = eta). Returns (F-hat, iterations, converged).
    """
    om = np.asarray(omega, np.float64)
    eta = exchange(F, om)
    N = eta.shape[0]
    scale = float(om.max())
    for it in range(1, maxit + 1):
        H = eta.copy()
        sq = eta[:, :N]
        H[:, :N] = kappa * sq + (1.0 - kappa) * sq.T
        d_recip = float(np.max(np.abs(sq - sq.T))) * 0.5 if N > 0 else 0.0
        rows = H.sum(axis=1)
        d_close = float(np.max(np.abs(rows - om)))
        lam = (om - rows) / H.sum(axis=1)
        eta = H + H * lam[:, None]
        if max(d_recip, d_close) <= tol * scale:
            return from_exchange(eta, om), it, True
    return from_exchange(eta, om), maxit, False


# ----------------------------------------------------------------------------
# Least-squares optimum for open systems (Sec. 3.5.5, Eq. 3.41-3.52) + NNR + SPVA
# ----------------------------------------------------------------------------

def restriction_system(N, omega, space="F"):
    """A = [R_C; R_R] and b = [c_C; c_R] (Eq. 3.41-3.43) as sparse matrices.

    Unknowns are the N(N+1) entries in row-major order (the environment column
    included, Eq. 3.42). Reciprocity rows run over pairs i < j (Eq. 3.43).
    space="F": rows sum_j F_ij = 1 and A_i F_ij - A_j F_ji = 0.
    space="eta": rows sum_j eta_ij = Omega_i and eta_ij - eta_ji = 0 (literal text).
    """
    om = np.asarray(omega, np.float64)
    M = N + 1
    rows, cols, vals = [], [], []
    for i in range(N):
        for j in range(M):
            rows.append(i); cols.append(i * M + j); vals.append(1.0)
    r = N
    for i in range(N):
        for j in range(i + 1, N):
            a_i, a_j = (om[i], om[j]) if space == "F" else (1.0, 1.0)
            rows += [r, r]; cols += [i * M + j, j * M + i]; vals += [a_i, -a_j]
            r += 1
    A = scipy.sparse.csr_matrix((vals, (rows, cols)), shape=(r, N * M))
    b = np.zeros(r)
    b[:N] = 1.0 if space == "F" else om
    return A, b


def project_literal(A, b, x):
    """Eq. 3.47-3.52 written out with dense matrices (tiny systems only).

    x_r = A^T (A A^T)^+ b, N_b = basis of null(A), w = (N_b^T N_b)^-1 N_b^T (x - x_r),
    x-hat = x_r + N_b w.
    """
    A = np.asarray(A.todense() if scipy.sparse.issparse(A) else A, np.float64)
    x_r = A.T @ (np.linalg.pinv(A @ A.T) @ b)
    Nb = scipy.linalg.null_space(A)
    if Nb.shape[1] == 0:
        return x_r
    w = np.linalg.solve(Nb.T @ Nb, Nb.T @ (x - x_r))
    return x_r + Nb @ w


def project(A, b, x):
    """Orthogonal projection of x onto {A x = b}: x - A^+ (A x - b).

    This is Eq. 3.52: x_r + N_b (N_b^T N_b)^-1 N_b^T (x - x_r) with x_r = A^+ b equals
    P_null x + A^+ b = x - A^+ (A x - b). The minimum-norm least-squares solution
    A^+ r is computed by LSQR (Paige & Saunders 1982) to full double precision.
    """
    A = scipy.sparse.csr_matrix(A)
    r = A @ x - b
    z = scipy.sparse.linalg.lsqr(A, r, atol=1e-16, btol=1e-16, conlim=1e14, iter_lim=100000)[0]
    return x - z


def lsq_optimum(F, omega, nnr=True, spva=True, space="F", literal=False, max_passes=1000):
    """Least-squares optimum for open systems with NNR (App. A.1) and SPVA (App. A.2).

    SPVA: MCRT zeros are removed from the unknowns (fixed at 0), then restriction
    rows left without unknowns are dropped (App. A.2 steps 1-5).
    NNR: after each projection, negative entries are set to 0 and removed from the
    unknowns, rows left without unknowns are dropped, and the original MCRT values
    of the remaining unknowns are projected again, until no entry is negative.
    Returns (F-hat, passes).
    """
    F = np.asarray(F, np.float64)
    om = np.asarray(omega, np.float64)
    N = F.shape[0]
    A_full, b_full = restriction_system(N, om, space)
    x0 = (F if space == "F" else exchange(F, om)).reshape(-1)
    active = np.ones(x0.size, dtype=bool)
    if spva:
        active &= x0 != 0.0
    passes = 0
    while True:
        passes += 1
        A = A_full[:, np.flatnonzero(active)]
        keep = np.diff(A.tocsr().indptr) > 0
        A = A[keep]
        b = b_full[keep]
        xa = x0[active]
        xh = project_literal(A, b, xa) if literal else project(A, b, xa)
        x = np.zeros_like(x0)
        x[active] = xh
        neg = x < 0.0
        if not nnr or not neg.any() or passes >= max_passes:
            break
        active &= ~neg
    out = x.reshape(N, N + 1)
    return (out if space == "F" else from_exchange(out, om)), passes


def mae(F, F_ref):
    """Mean absolute error over all N(N+1) entries (Table 6.1 metric)."""
    return float(np.mean(np.abs(np.asarray(F) - np.asarray(F_ref))))
