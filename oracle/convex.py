"""Brute-force solve of the balanced entropic OT problem on tiny inputs.

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
