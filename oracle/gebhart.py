"""Gebhart radiative exchange factors, steady radiative balance and their adjoints.

TEST INFRASTRUCTURE ONLY (see the package docstring). Plain numpy, fp64.

* REFs: K B = E with K = I - F diag(rho) (Eq. B.3/B.9), E = [F diag(eps) | F_inf]
  (Eq. B.8), B = K^-1 E (Eq. B.11); closed systems have no environment column
  (Eq. B.1-B.5). The last row of K in Eq. B.3/B.9 prints -rho_2 F_2N where
  -rho_2 F_N2 is meant (the matrix is I - F diag(rho), as Eq. 4.5 states).
* Steady radiative balance of every node: sum_j GR_ij (T_i^4 - T_j^4) = Q_i
  (Eq. 3.13) with GR_ij = sigma eps_i A_i B_ij (Eq. 4.2) and the environment as a
  node of fixed temperature T_sink; linear in u = T^4.
* Adjoints: derived from B = K^-1 E. With Lambda = K^-T dL/dB:
  dL/deps_j = sum_i Lambda_ij F_ij (j <= N) and
  dL/drho_k = sum_i F_ik (Lambda B^T)_ik.
  For the temperatures M u = r with M = diag(sigma eps A)(diag(s) - B_NN),
  s_i = sum_{j != i} B_ij + B_i,inf (plus the B_ii term that cancels),
  r = Q + sigma eps A B_inf u_sink; mu = M^-T dL/du and
  dL/dB_ij = -mu_i sigma eps_i A_i (u_i - u_j) (u_{N+1} = u_sink),
  dL/deps_i (direct) = -mu_i sigma A_i sum_j B_ij (u_i - u_j).
"""
from __future__ import annotations

import numpy as np

SIGMA = 5.67e-8  # W m^-2 K^-4, the value the thesis prints


def k_matrix(F, rho):
    """K = I - F_NN diag(rho) (Eq. B.9)."""
    F = np.asarray(F, np.float64)
    N = F.shape[0]
    return np.eye(N) - F[:, :N] * np.asarray(rho, np.float64)[None, :]


def e_matrix(F, eps):
    """E = [F_NN diag(eps) | F_inf] (Eq. B.8); for a closed N x N F, F_NN diag(eps) (Eq. B.2)."""
    F = np.asarray(F, np.float64)
    N = F.shape[0]
    E = F.copy()
    E[:, :N] = F[:, :N] * np.asarray(eps, np.float64)[None, :]
    return E


def gebhart(F, eps, rho):
    """B = K^-1 E (Eq. B.5 / B.11). F is N x N (closed) or N x (N+1) (open)."""
    return np.linalg.solve(k_matrix(F, rho), e_matrix(F, eps))


def gebhart_rows(F, eps, rho, rows):
    """Selected rows of B = K^-1 E (Eq. B.11): B[rows] = Y^T E with K^T Y = I[:, rows]."""
    K = k_matrix(F, rho)
    Y = np.linalg.solve(K.T, np.eye(K.shape[0])[:, list(rows)])
    return Y.T @ e_matrix(F, eps)


def gebhart_batched(F, eps_sets, rho_sets):
    """One REF matrix per (eps, rho) set: [S, N, N+1]."""
    return np.stack([gebhart(F, e, r) for e, r in zip(eps_sets, rho_sets)])


def recursion_residual(F, eps, rho, B):
    """max |B_ij - eps_j F_ij - sum_k F_ik rho_k B_kj| (Eq. 4.5; Eq. B.6 for the env column)."""
    F = np.asarray(F, np.float64)
    N = F.shape[0]
    rhs = e_matrix(F, eps) + (F[:, :N] * np.asarray(rho)[None, :]) @ B
    return float(np.max(np.abs(B - rhs)))


def gebhart_adjoint(F, eps, rho, B, Bbar):
    """Gradients (dL/deps, dL/drho) of L(B) given Bbar = dL/dB."""
    F = np.asarray(F, np.float64)
    N = F.shape[0]
    K = k_matrix(F, rho)
    Lam = np.linalg.solve(K.T, np.asarray(Bbar, np.float64))
    FN = F[:, :N]
    deps = np.sum(Lam[:, :N] * FN, axis=0)
    drho = np.sum(FN * (Lam @ np.asarray(B, np.float64).T), axis=0)
    return deps, drho


def conductances(B, eps, area, sigma=SIGMA):
    """GR_ij = sigma eps_i A_i B_ij (Eq. 4.2), N x (N+1)."""
    return sigma * (np.asarray(eps) * np.asarray(area))[:, None] * np.asarray(B, np.float64)


def balance_system(B, eps, area, Q, T_sink, sigma=SIGMA):
    """M, r of the steady balance sum_j GR_ij (u_i - u_j) = Q_i in u = T^4 (Eq. 3.13)."""
    B = np.asarray(B, np.float64)
    N = B.shape[0]
    g = sigma * np.asarray(eps, np.float64) * np.asarray(area, np.float64)
    BN = B[:, :N]
    off = BN - np.diag(np.diag(BN))
    s = off.sum(axis=1) + B[:, N]
    M = g[:, None] * (np.diag(s) - off)
    r = np.asarray(Q, np.float64) + g * B[:, N] * T_sink ** 4
    return M, r


def temperatures(B, eps, area, Q, T_sink, sigma=SIGMA):
    """Steady node temperatures from the REFs (Eq. 3.13 with Eq. 4.2), K."""
    M, r = balance_system(B, eps, area, Q, T_sink, sigma)
    u = np.linalg.solve(M, r)
    return u ** 0.25


def temperatures_adjoint(B, eps, area, Q, T_sink, T, Tbar, sigma=SIGMA):
    """(dL/dB [N, N+1], dL/deps direct [N]) of L(T) given Tbar = dL/dT."""
    B = np.asarray(B, np.float64)
    N = B.shape[0]
    M, _ = balance_system(B, eps, area, Q, T_sink, sigma)
    u = np.asarray(T, np.float64) ** 4
    ubar = np.asarray(Tbar, np.float64) / (4.0 * np.asarray(T, np.float64) ** 3)
    mu = np.linalg.solve(M.T, ubar)
    g = sigma * np.asarray(eps) * np.asarray(area)
    uu = np.concatenate([u, [T_sink ** 4]])
    diff = u[:, None] - uu[None, :]           # u_i - u_j, j over N+1 columns
    Bbar = -(mu * g)[:, None] * diff
    deps_direct = -mu * sigma * np.asarray(area) * np.sum(B * diff, axis=1)
    return Bbar, deps_direct


def thermal_gradients(F, eps, rho, area, Q, T_sink, Tbar, sigma=SIGMA):
    """dL/deps, dL/drho of L(T(B(eps, rho), eps)) through both adjoints."""
    B = gebhart(F, eps, rho)
    T = temperatures(B, eps, area, Q, T_sink, sigma)
    Bbar, deps_direct = temperatures_adjoint(B, eps, area, Q, T_sink, T, Tbar, sigma)
    deps_b, drho = gebhart_adjoint(F, eps, rho, B, Bbar)
    return deps_b + deps_direct, drho


def steady_temperatures_fixed(GR, fixed_T, node_of_face=None, Q=None, T_env=None):
    """Steady temperatures of a network with some nodes held at fixed temperatures.

    GR is N x (N+1) (column N = environment at T_env); faces sharing a node
    (``node_of_face``) share one temperature; ``fixed_T`` maps node -> K. Each free
    node balances sum over its faces of sum_j GR_ij (u_i - u_j) = Q_node (Eq. 3.13).
    Used for the parallel-plates example (Table 6.2).
    """
    GR = np.asarray(GR, np.float64)
    N = GR.shape[0]
    nodes = np.arange(N) if node_of_face is None else np.asarray(node_of_face)
    n_nodes = int(nodes.max()) + 1
    P = np.zeros((N, n_nodes))
    P[np.arange(N), nodes] = 1.0
    # per-face flow out: sum_j GR_ij (u_i - u_j) = (rowsum_i) u_i - sum_j GR_ij u_j - GR_i,env u_env
    L = np.diag(GR.sum(axis=1)) - GR[:, :N]
    Ln = P.T @ L @ P                       # node-level operator
    env = P.T @ GR[:, N]                   # node coupling to environment
    q = np.zeros(n_nodes) if Q is None else np.asarray(Q, np.float64).copy()
    q = q + env * (T_env ** 4 if T_env is not None else 0.0)
    free = [n for n in range(n_nodes) if n not in fixed_T]
    fixed = sorted(fixed_T)
    u_fix = np.array([fixed_T[n] ** 4 for n in fixed])
    A = Ln[np.ix_(free, free)]
    rhs = q[free] - (Ln[np.ix_(free, fixed)] @ u_fix if fixed else 0.0)
    u = np.zeros(n_nodes)
    u[free] = np.linalg.solve(A, rhs)
    u[fixed] = u_fix
    return u ** 0.25


def central_difference(fn, x, h=1e-6):
    """Central finite differences of a scalar function, one coordinate at a time."""
    x = np.asarray(x, np.float64)
    g = np.zeros_like(x)
    for k in range(x.size):
        xp = x.copy(); xp.flat[k] += h
        xm = x.copy(); xm.flat[k] -= h
        g.flat[k] = (fn(xp) - fn(xm)) / (2.0 * h)
    return g
