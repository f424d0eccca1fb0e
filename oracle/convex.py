"""Brute-force solves of the entropic OT problems on tiny inputs.

TEST INFRASTRUCTURE ONLY.  This module is not a Sinkhorn iteration: it maximises
the smooth dual of

    min_P  <P, C> + reg * sum_ij P_ij (log P_ij - 1)
    s.t.   P 1 = p,  P^T 1 = q                     (sum p == sum q)

with a damped Newton method on the dual variables (phi, psi), psi_M pinned to
0 to remove the one-dimensional degeneracy.  The primal optimum is
``P_ij = exp((phi_i + psi_j - C_ij)/reg)``.  The oracle's Sinkhorn iteration
(Section 2.1) is pinned to this solve at its fixed point: the limit of the
literal rule is the balanced plan between rescaled marginals (see
``fixed_point_marginals``).
"""

from __future__ import annotations

import numpy as np


def fixed_point_marginals(a, b, fi: float):
    """Marginals of the limit of the literal row-then-column rule.

    At a fixed point of "row step, then column step" every row factor equals a
    constant ``k`` and every column factor ``1/k``; the row sums are
    ``a k^(-1/fi)`` and the column sums ``b k^(1/fi - 1)``.  Equal total mass
    gives ``k = (m_a/m_b)^(fi/(2-fi))``.  Returns ``(p, q, k)``.
    """
    a = np.asarray(a, np.float64)
    b = np.asarray(b, np.float64)
    ma, mb = a.sum(), b.sum()
    k = (ma / mb) ** (fi / (2.0 - fi))
    p = a * k ** (-1.0 / fi)
    q = b * k ** (1.0 / fi - 1.0)
    return p, q, k


def entropic_ot_newton(C, p, q, reg: float, tol: float = 1e-14, max_iter: int = 500):
    """Balanced entropic OT plan by Newton's method on the dual (see module doc)."""
    C = np.asarray(C, np.float64)
    p = np.asarray(p, np.float64)
    q = np.asarray(q, np.float64)
    N, M = C.shape
    if abs(p.sum() - q.sum()) > 1e-12 * max(p.sum(), 1.0):
        raise ValueError("balanced problem needs equal masses")
    phi = np.zeros(N)
    psi = np.zeros(M)

    def plan(phi, psi):
        return np.exp((phi[:, None] + psi[None, :] - C) / reg)

    def dual(phi, psi):
        return phi @ p + psi @ q - reg * plan(phi, psi).sum()

    for _ in range(max_iter):
        P = plan(phi, psi)
        g = np.concatenate([p - P.sum(axis=1), (q - P.sum(axis=0))[: M - 1]])
        if np.max(np.abs(g)) <= tol * max(p.max(), q.max()):
            break
        # Hessian of the (concave) dual, restricted to (phi, psi[:M-1]).
        H = np.zeros((N + M - 1, N + M - 1))
        H[:N, :N] = np.diag(P.sum(axis=1))
        H[N:, N:] = np.diag(P.sum(axis=0)[: M - 1])
        H[:N, N:] = P[:, : M - 1]
        H[N:, :N] = P[:, : M - 1].T
        H *= -1.0 / reg
        step = np.linalg.solve(H, -g)
        d_phi, d_psi = step[:N], np.concatenate([step[N:], [0.0]])
        base = dual(phi, psi)
        s = 1.0
        while s > 1e-12:
            if dual(phi + s * d_phi, psi + s * d_psi) >= base - 1e-15 * abs(base):
                break
            s *= 0.5
        phi = phi + s * d_phi
        psi = psi + s * d_psi
    return plan(phi, psi)


def uot_objective(P, C, a, b, reg: float, reg_m: float) -> float:
    """``<P,C> + reg sum P (log P - 1) + reg_m KL(P1|a) + reg_m KL(P^T 1|b)`` with
    the generalised ``KL(x|y) = sum x log(x/y) - x + y`` (``reg_m = inf``:
    the marginal terms become constraints and are left out)."""
    P = np.asarray(P, np.float64)
    r, c = P.sum(axis=1), P.sum(axis=0)

    def kl(x, y):
        return float(np.sum(x * np.log(x / y) - x + y))

    val = float(np.sum(P * C) + reg * np.sum(P * (np.log(P) - 1.0)))
    if np.isfinite(reg_m):
        val += reg_m * (kl(r, a) + kl(c, b))
    return val


def uot_newton(C, a, b, reg: float, reg_m: float, tol: float = 1e-13, max_iter: int = 200):
    """Minimiser of ``uot_objective`` over positive plans by Newton's method in
    the plan entries themselves (N*M unknowns; tiny problems only).

    Gradient ``C_ij + reg log P_ij + reg_m log(r_i/a_i) + reg_m log(c_j/b_j)``;
    Hessian ``reg/P_ij`` on the diagonal plus ``reg_m/r_i`` between entries of
    row i and ``reg_m/c_j`` between entries of column j (positive definite).
    Steps are cut to keep every entry positive and to decrease the objective.
    """
    C = np.asarray(C, np.float64)
    a = np.asarray(a, np.float64)
    b = np.asarray(b, np.float64)
    if not np.isfinite(reg_m):
        raise ValueError("reg_m must be finite (the balanced case is entropic_ot_newton)")
    N, M = C.shape
    P = np.full((N, M), np.sqrt(a.sum() * b.sum()) / (N * M))
    rows = np.repeat(np.arange(N), M)
    cols = np.tile(np.arange(M), N)
    same_row = (rows[:, None] == rows[None, :]).astype(np.float64)
    same_col = (cols[:, None] == cols[None, :]).astype(np.float64)
    for _ in range(max_iter):
        r, c = P.sum(axis=1), P.sum(axis=0)
        g = (C + reg * np.log(P) + reg_m * np.log(r / a)[:, None]
             + reg_m * np.log(c / b)[None, :]).ravel()
        if np.max(np.abs(g)) <= tol:
            break
        p = P.ravel()
        H = np.diag(reg / p) + reg_m * same_row / r[rows][:, None] + reg_m * same_col / c[cols][:, None]
        step = np.linalg.solve(H, -g)
        # Stay inside the positive orthant, then backtrack on the objective.
        neg = step < 0
        smax = min(1.0, 0.99 * float(np.min(-p[neg] / step[neg]))) if neg.any() else 1.0
        base = uot_objective(P, C, a, b, reg, reg_m)
        s = smax
        while s > 1e-14:
            Pn = (p + s * step).reshape(N, M)
            if uot_objective(Pn, C, a, b, reg, reg_m) <= base + 1e-15 * abs(base):
                break
            s *= 0.5
        P = (p + s * step).reshape(N, M)
    return P
