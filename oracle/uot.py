"""Plain FP64 oracle of the Sinkhorn-UOT iteration (Section 2.1).

TEST INFRASTRUCTURE ONLY: used by ``tests/``, ``__graft_entry__.smoke()`` and
``bench.py``'s CPU baseline.  It shares no code with the CUDA path.

Notation: the plan ``P`` is N x M, row-major; ``a`` (length N) is the row
target (the paper's RPD), ``b`` (length M) the column target (CPD).  The
paper's own matrix ``A`` has M rows and N columns; only the names differ.

Readings of points the paper leaves open (each is also listed in the design
notes of the repository):

* ``fi = er/(er+ep)`` (Section 2.1) with ``er = reg_m`` (marginal weight) and
  ``ep = reg`` (entropic weight); ``reg_m = inf`` gives ``fi = 1`` (balanced).
* Order: a row step, then a column step, per iteration (Section 2.1 states
  this order; Algorithm 1 is written column-first and the paper says the order
  does not change the limit).  The output is the plan after the column step of
  the last iteration.
* Initial plan: ``P0 = exp(-C/reg)`` (the paper only says "given matrix").
* Degenerate factors: target 0 gives factor 0; a zero sum with a positive
  target gives factor 1 and raises ``STATUS_ZERO_SUM``; a non-finite sum or
  factor raises ``STATUS_NONFINITE``.
* Stopping error (undefined in the paper): the relative L1 change of the row
  sums, ``err_t = sum_i |r_t,i - r_{t-1},i| / sum_i r_t,i``, checked after the
  column step of iteration ``t`` when ``tol > 0``, ``t >= 2`` and
  ``t % check_every == 0``.

Parity status: no function here can be pinned to numbers printed in the paper
(it prints none).  ``sinkhorn_pot`` is pinned by the brute-force minimiser of the
unbalanced objective, by the 1x1 closed form and by ``sinkhorn`` at ``fi = 1``.
``sinkhorn`` is pinned by closed forms (1x1, rank-one cost),
the textbook balanced Sinkhorn at ``fi = 1``, the closed-form fixed point
checked by a brute-force convex solve, per-step identities and symmetries;
``sinkhorn_grad`` by FP64 central differences and by torch autograd of the
plain unrolled loop.
"""

from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

STATUS_ZERO_SUM = 1
STATUS_NONFINITE = 2


def fi_exponent(reg: float, reg_m: float) -> float:
    """Exponent of the rescaling factors, ``fi = er/(er+ep)`` (Section 2.1)."""
    if reg <= 0 or not math.isfinite(reg):
        raise ValueError("reg must be a positive finite number")
    if reg_m <= 0:
        raise ValueError("reg_m must be positive (inf = balanced)")
    if math.isinf(reg_m):
        return 1.0
    return reg_m / (reg_m + reg)


def init_plan(C, reg: float) -> np.ndarray:
    """Initial plan ``P0 = exp(-C/reg)`` in FP64 from the given cost values."""
    C = np.asarray(C, dtype=np.float64)
    return np.exp(-C / reg)


def scaling_factor(target, total, fi: float):
    """Rescaling factor ``(target/total)^fi`` of Section 2.1, elementwise.

    Returns ``(factor, status)``.  Degenerate readings: ``target == 0`` gives 0,
    ``total == 0 < target`` gives 1 (``STATUS_ZERO_SUM``).
    """
    target = np.asarray(target, dtype=np.float64)
    total = np.asarray(total, dtype=np.float64)
    status = 0
    factor = np.empty_like(total)
    zero_t = target == 0.0
    zero_s = (total == 0.0) & ~zero_t
    ok = ~zero_t & ~zero_s
    factor[zero_t] = 0.0
    factor[zero_s] = 1.0
    if zero_s.any():
        status |= STATUS_ZERO_SUM
    factor[ok] = np.power(target[ok] / total[ok], fi)
    if not np.all(np.isfinite(factor)) or not np.all(np.isfinite(total)):
        status |= STATUS_NONFINITE
    return factor, status


def row_step(P: np.ndarray, a, fi: float):
    """Row rescaling: ``r_i = sum_j P_ij``, ``alpha_i = (a_i/r_i)^fi``,
    ``P_ij *= alpha_i`` (Section 2.1).  ``P`` is updated in place."""
    r = P.sum(axis=1)
    alpha, status = scaling_factor(a, r, fi)
    P *= alpha[:, None]
    return r, alpha, status


def col_step(P: np.ndarray, b, fi: float):
    """Column rescaling: ``c_j = sum_i P_ij``, ``beta_j = (b_j/c_j)^fi``,
    ``P_ij *= beta_j`` (Section 2.1).  ``P`` is updated in place."""
    c = P.sum(axis=0)
    beta, status = scaling_factor(b, c, fi)
    P *= beta[None, :]
    return c, beta, status


@dataclass
class OracleResult:
    plan: np.ndarray
    iters_done: int
    err: float
    status: int
    # Per-iteration records when ``record=True``: row sums r_t, row factors
    # alpha_t, column sums c_t, column factors beta_t (t = 1..iters_done).
    r: list = field(default_factory=list)
    alpha: list = field(default_factory=list)
    c: list = field(default_factory=list)
    beta: list = field(default_factory=list)


def sinkhorn(P0, a, b, reg: float, reg_m: float, iters: int, tol: float = 0.0,
             check_every: int = 1, order: str = "row_first",
             record: bool = False) -> OracleResult:
    """The baseline UOT Sinkhorn iteration of Section 2.1, applied literally.

    Each iteration rescales every row by ``(a_i/rowsum_i)^fi`` and then every
    column by ``(b_j/colsum_j)^fi`` (``order="col_first"`` swaps the two, for
    the transpose-symmetry pin).  MAP-UOT (Section 4, Algorithm 1) reaches the
    same iterate with one sweep per iteration; this oracle keeps the plain
    two-step form.
    """
    if iters < 0:
        raise ValueError("iters must be >= 0")
    if check_every < 1:
        raise ValueError("check_every must be >= 1")
    fi = fi_exponent(reg, reg_m)
    P = np.array(P0, dtype=np.float64, copy=True)
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    res = OracleResult(plan=P, iters_done=0, err=math.inf, status=0)
    r_prev = None
    for t in range(1, iters + 1):
        if order == "row_first":
            r, alpha, s1 = row_step(P, a, fi)
            c, beta, s2 = col_step(P, b, fi)
        elif order == "col_first":
            c, beta, s2 = col_step(P, b, fi)
            r, alpha, s1 = row_step(P, a, fi)
        else:
            raise ValueError(order)
        res.status |= s1 | s2
        res.iters_done = t
        if record:
            res.r.append(r)
            res.alpha.append(alpha)
            res.c.append(c)
            res.beta.append(beta)
        if r_prev is not None:
            den = r.sum()
            res.err = float(np.abs(r - r_prev).sum() / den) if den > 0 else math.inf
        r_prev = r
        if tol > 0 and t >= 2 and t % check_every == 0 and res.err <= tol:
            break
    return res


def sinkhorn_pot(K, a, b, reg: float, reg_m: float, iters: int, tol: float = 0.0,
                 check_every: int = 1) -> OracleResult:
    """The scaling-vector form of the unbalanced iteration (the update of POT's
    ``sinkhorn_unbalanced``), row step first:

        u <- (a / (K v))^fi,    then    v <- (b / (K^T u))^fi,

    with the plan ``diag(u) K diag(v)`` and ``u = v = 1`` at the start, ``K``
    the initial plan.  It is NOT the rule Section 2.1 prints: written as a
    rescale of the plan, its row factor is the printed ``(a_i/rowsum_i)^fi``
    times ``u_i^(fi-1)``, so the two agree only when ``fi = 1``.  Its fixed
    point minimises ``<P,C> + reg sum P (log P - 1) + reg_m KL(P1|a) +
    reg_m KL(P^T 1|b)`` (see ``convex.uot_newton``).  The degenerate readings of
    ``scaling_factor`` apply to the ratios ``a/(Kv)`` and ``b/(K^T u)``; the
    stopping error is the one of ``sinkhorn`` (row sums of the plan before each
    row step).
    """
    if iters < 0:
        raise ValueError("iters must be >= 0")
    if check_every < 1:
        raise ValueError("check_every must be >= 1")
    fi = fi_exponent(reg, reg_m)
    K = np.asarray(K, dtype=np.float64)
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    u = np.ones(K.shape[0])
    v = np.ones(K.shape[1])
    res = OracleResult(plan=K.copy(), iters_done=0, err=math.inf, status=0)
    r_prev = None
    for t in range(1, iters + 1):
        Kv = K @ v
        r = u * Kv
        u, s1 = scaling_factor(a, Kv, fi)
        Ktu = K.T @ u
        v, s2 = scaling_factor(b, Ktu, fi)
        res.status |= s1 | s2
        res.iters_done = t
        if r_prev is not None:
            den = r.sum()
            res.err = float(np.abs(r - r_prev).sum() / den) if den > 0 else math.inf
        r_prev = r
        if tol > 0 and t >= 2 and t % check_every == 0 and res.err <= tol:
            break
    res.plan = u[:, None] * K * v[None, :]
    return res


def transport_cost(P, C) -> float:
    """Transport cost ``<P, C> = sum_ij P_ij C_ij`` accumulated in FP64."""
    return float(np.sum(np.asarray(P, np.float64) * np.asarray(C, np.float64)))


def kernel_form_scalings(res: OracleResult):
    """Cumulative scalings ``U = prod_t alpha_t`` and ``V = prod_t beta_t`` of a
    recorded run, so that the plan equals ``diag(U) P0 diag(V)`` (exactly, in
    real arithmetic).  Used to check the read-only kernel-form storage."""
    if not res.alpha:
        raise ValueError("run sinkhorn(..., record=True) first")
    U = np.prod(np.stack(res.alpha), axis=0)
    V = np.prod(np.stack(res.beta), axis=0)
    return U, V


def sinkhorn_grad(C, a, b, reg: float, reg_m: float, iters: int):
    """Value and gradient of ``L = <P_T, C>`` w.r.t. ``C``, ``a`` and ``b``.

    The iteration of Section 2.1 is written in log space: ``l = -C/reg``,
    ``f_0 = g_0 = 0``,
      ``r_t = rowsum(exp(l + f_{t-1} (+) g_{t-1}))``, ``f_t = f_{t-1} + fi (log a - log r_t)``,
      ``c_t = colsum(exp(l + f_t (+) g_{t-1}))``,   ``g_t = g_{t-1} + fi (log b - log c_t)``,
    with ``P_T = exp(l + f_T (+) g_T)``.  Reverse mode through these steps
    (the paper has no adjoint; this is plain calculus on its update rule):
    with ``R_t = exp(l + f_{t-1} (+) g_{t-1})`` and ``Q_t = exp(l + f_t (+) g_{t-1})``,
    start from ``dl = P_T * C``, ``F = rowsum(dl)``, ``G = colsum(dl)`` and for
    ``t = T..1``
      column step: ``w = -fi G / c_t``, ``db += fi G / b``, ``F += Q_t w``,
                   ``dl += Q_t * w[None, :]``, ``G = (1 - fi) G``;
      row step:    ``z = -fi F / r_t``, ``da += fi F / a``, ``G += R_t^T z``,
                   ``dl += R_t * z[:, None]``, ``F = (1 - fi) F``.
    Finally ``dC = P_T - dl / reg``.  All arithmetic in FP64.  Requires strictly
    positive ``a`` and ``b`` (the log-space form has no degenerate factors).
    """
    fi, l, f, g, rs, cs = _log_forward(C, a, b, reg, reg_m, iters, "sinkhorn_grad")
    a = np.asarray(a, np.float64)
    b = np.asarray(b, np.float64)
    C = np.asarray(C, np.float64)
    N, M = C.shape
    P = np.exp(l + f[-1][:, None] + g[-1][None, :])
    value = float(np.sum(P * C))
    dl = P * C
    F = dl.sum(axis=1)
    G = dl.sum(axis=0)
    da = np.zeros(N)
    db = np.zeros(M)
    for t in range(iters, 0, -1):
        Q = np.exp(l + f[t][:, None] + g[t - 1][None, :])
        R = np.exp(l + f[t - 1][:, None] + g[t - 1][None, :])
        w = -fi * G / cs[t - 1]
        db += fi * G / b
        F = F + Q @ w
        dl += Q * w[None, :]
        G = (1.0 - fi) * G
        z = -fi * F / rs[t - 1]
        da += fi * F / a
        G = G + R.T @ z
        dl += R * z[:, None]
        F = (1.0 - fi) * F
    dC = P - dl / reg
    return value, dC, da, db


def _log_forward(C, a, b, reg: float, reg_m: float, iters: int, who: str):
    """The log-space forward of ``sinkhorn_grad``: ``fi``, ``l = -C/reg`` and
    the lists ``f_t``, ``g_t`` (t = 0..iters), ``r_t``, ``c_t`` (t = 1..iters)."""
    fi = fi_exponent(reg, reg_m)
    C = np.asarray(C, np.float64)
    a = np.asarray(a, np.float64)
    b = np.asarray(b, np.float64)
    if np.any(a <= 0) or np.any(b <= 0):
        raise ValueError(f"{who} needs strictly positive marginals")
    l = -C / reg
    N, M = C.shape
    f = [np.zeros(N)]
    g = [np.zeros(M)]
    rs, cs = [], []
    for _ in range(iters):
        r = np.exp(l + f[-1][:, None] + g[-1][None, :]).sum(axis=1)
        f.append(f[-1] + fi * (np.log(a) - np.log(r)))
        c = np.exp(l + f[-1][:, None] + g[-1][None, :]).sum(axis=0)
        g.append(g[-1] + fi * (np.log(b) - np.log(c)))
        rs.append(r)
        cs.append(c)
    return fi, l, f, g, rs, cs


def sinkhorn_grad_magnitude(C, a, b, reg: float, reg_m: float, iters: int):
    """Magnitudes of the terms each gradient entry of ``sinkhorn_grad`` is
    formed from: the same reverse recurrence with every term taken by its
    absolute value (``w = +fi G / c``, ``z = +fi F / r`` on the magnitudes,
    ``dC = P + dl / reg``).  Rounding errors of any evaluation of the adjoint
    scale with these, not with the gradient itself, which can be far smaller
    where terms of opposite sign cancel.  Returns ``(dC_mag, da_mag, db_mag)``,
    each elementwise >= the absolute value of the gradient."""
    fi, l, f, g, rs, cs = _log_forward(C, a, b, reg, reg_m, iters, "sinkhorn_grad_magnitude")
    a = np.asarray(a, np.float64)
    b = np.asarray(b, np.float64)
    C = np.asarray(C, np.float64)
    N, M = C.shape
    P = np.exp(l + f[-1][:, None] + g[-1][None, :])
    dl = P * np.abs(C)
    F = dl.sum(axis=1)
    G = dl.sum(axis=0)
    da = np.zeros(N)
    db = np.zeros(M)
    for t in range(iters, 0, -1):
        Q = np.exp(l + f[t][:, None] + g[t - 1][None, :])
        R = np.exp(l + f[t - 1][:, None] + g[t - 1][None, :])
        w = fi * G / cs[t - 1]
        db += fi * G / b
        F = F + Q @ w
        dl += Q * w[None, :]
        G = (1.0 - fi) * G
        z = fi * F / rs[t - 1]
        da += fi * F / a
        G = G + R.T @ z
        dl += R * z[:, None]
        F = (1.0 - fi) * F
    return P + dl / reg, da, db


def sinkhorn_tensor3(P0, a, b, c, reg: float, reg_m: float, iters: int) -> np.ndarray:
    """The rule of Section 2.1 on a three-way plan (the paper notes the method
    applies to higher-dimensional tensors; this is the reading used): every
    iteration rescales along mode 1, then mode 2, then mode 3, each time by
    ``(target / marginal sum)^fi`` with the degenerate readings of
    ``scaling_factor``.  ``P0`` is n1 x n2 x n3; ``a``, ``b``, ``c`` are the
    mode targets.  Returns the plan after the mode-3 step of the last
    iteration (FP64)."""
    fi = fi_exponent(reg, reg_m)
    P = np.array(P0, dtype=np.float64, copy=True)
    for _ in range(iters):
        f1, _ = scaling_factor(a, P.sum(axis=(1, 2)), fi)
        P *= f1[:, None, None]
        f2, _ = scaling_factor(b, P.sum(axis=(0, 2)), fi)
        P *= f2[None, :, None]
        f3, _ = scaling_factor(c, P.sum(axis=(0, 1)), fi)
        P *= f3[None, None, :]
    return P
