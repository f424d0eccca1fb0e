"""Pins of the FP64 oracle against closed forms, textbook routines, a convex
solve and invariants of the Section 2.1 update rule (CPU only)."""

import json
import math
import os

import numpy as np
import pytest

import oracle
from oracle import convex

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def rand_problem(seed, n, m, lo=0.5, hi=1.5, mass_a=1.0, mass_b=1.5, scale=1.0):
    rng = np.random.default_rng(seed)
    C = rng.random((n, m)) * scale
    a = rng.uniform(lo, hi, n)
    a *= mass_a / a.sum()
    b = rng.uniform(lo, hi, m)
    b *= mass_b / b.sum()
    return C, a, b


def test_fi_exponent_reading():
    # fi = er/(er+ep) with er = reg_m, ep = reg (Section 2.1).
    assert oracle.fi_exponent(0.05, 1.0) == pytest.approx(1.0 / 1.05, rel=1e-15)
    assert oracle.fi_exponent(0.1, 0.5) == pytest.approx(0.5 / 0.6, rel=1e-15)
    assert oracle.fi_exponent(0.3, math.inf) == 1.0
    with pytest.raises(ValueError):
        oracle.fi_exponent(0.0, 1.0)
    with pytest.raises(ValueError):
        oracle.fi_exponent(0.1, -1.0)


@pytest.mark.parametrize("fi_pair", [(0.05, 1.0), (0.3, 0.5), (1.0, 0.2), (0.7, math.inf)])
def test_one_by_one_closed_form(fi_pair):
    """1x1: with x = log P each iteration is x <- (1-fi)x + fi log a followed
    by x <- (1-fi)x + fi log b, so x_T = q^T x0 + d (1 - q^T)/(1 - q) with
    q = (1-fi)^2 and d = (1-fi) fi log a + fi log b."""
    reg, reg_m = fi_pair
    fi = oracle.fi_exponent(reg, reg_m)
    a, b, p0 = 0.37, 2.9, 0.011
    q = (1 - fi) ** 2
    d = (1 - fi) * fi * math.log(a) + fi * math.log(b)
    for T in range(0, 41):
        res = oracle.sinkhorn([[p0]], [a], [b], reg, reg_m, T)
        if q == 0.0:
            x = math.log(p0) if T == 0 else d
        else:
            x = q**T * math.log(p0) + d * (1 - q**T) / (1 - q)
        assert res.plan[0, 0] == pytest.approx(math.exp(x), rel=1e-12)


def test_rank_one_cost_factorises():
    """C_ij = p_i + q_j makes P0 = u v^T rank one; the literal rule keeps it
    rank one and reduces to recurrences on u (rows) and v (columns)."""
    rng = np.random.default_rng(3)
    N, M, reg, reg_m, T = 9, 6, 0.2, 0.7, 25
    p, q = rng.random(N), rng.random(M)
    _, a, b = rand_problem(4, N, M)
    C = p[:, None] + q[None, :]
    fi = oracle.fi_exponent(reg, reg_m)
    u, v = np.exp(-p / reg), np.exp(-q / reg)
    for _ in range(T):
        u = u * (a / (u * v.sum())) ** fi
        v = v * (b / (v * u.sum())) ** fi
    res = oracle.sinkhorn(oracle.init_plan(C, reg), a, b, reg, reg_m, T)
    np.testing.assert_allclose(res.plan, np.outer(u, v), rtol=1e-12)


def test_balanced_case_is_textbook_sinkhorn():
    """reg_m = inf (fi = 1): the literal rule is the classical Sinkhorn-Knopp
    scaling u = a / (K v), v = b / (K^T u); after each iteration the column
    sums equal b."""
    C, a, b = rand_problem(5, 11, 7)
    reg = 0.25
    K = np.exp(-C / reg)
    v = np.ones(7)
    for T in range(1, 15):
        u = a / (K @ v)
        v = b / (K.T @ u)
        res = oracle.sinkhorn(K, a, b, reg, math.inf, T)
        np.testing.assert_allclose(res.plan, u[:, None] * K * v[None, :], rtol=1e-12)
        np.testing.assert_allclose(res.plan.sum(axis=0), b, rtol=1e-12)


@pytest.mark.parametrize("reg,reg_m", [(0.5, 1.0), (0.3, 0.4), (1.0, 5.0)])
def test_fixed_point_matches_convex_solve(reg, reg_m):
    """The limit of row-then-column rescaling is the balanced entropic-OT plan
    between the rescaled marginals a k^(-1/fi) and b k^(1/fi-1), solved here
    independently by Newton's method on the dual; the factors settle at
    alpha = k and beta = 1/k with k = (m_a/m_b)^(fi/(2-fi))."""
    C, a, b = rand_problem(7, 7, 5, mass_a=1.0, mass_b=1.7)
    fi = oracle.fi_exponent(reg, reg_m)
    res = oracle.sinkhorn(oracle.init_plan(C, reg), a, b, reg, reg_m, 4000, record=True)
    p, q, k = convex.fixed_point_marginals(a, b, fi)
    ref = convex.entropic_ot_newton(C, p, q, reg)
    np.testing.assert_allclose(res.plan, ref, rtol=1e-9)
    np.testing.assert_allclose(res.alpha[-1], k, rtol=1e-9)
    np.testing.assert_allclose(res.beta[-1], 1.0 / k, rtol=1e-9)


def test_fixed_point_golden_fixture():
    """Stored convex-solve plan (written by tests/golden/make_golden.py, which
    calls only oracle.convex) against the oracle's limit."""
    with open(os.path.join(GOLDEN, "fixed_point_6x4.json")) as fh:
        g = json.load(fh)
    C = np.array(g["C"])
    res = oracle.sinkhorn(oracle.init_plan(C, g["reg"]), g["a"], g["b"], g["reg"],
                          g["reg_m"], 5000)
    np.testing.assert_allclose(res.plan, np.array(g["plan"]), rtol=1e-9)


def test_step_identities():
    """After the row step the row sums are a^fi r^(1-fi); after the column step
    the column sums are b^fi c^(1-fi) (r, c: sums before the step)."""
    C, a, b = rand_problem(8, 13, 10)
    reg, reg_m = 0.2, 0.6
    fi = oracle.fi_exponent(reg, reg_m)
    P = oracle.init_plan(C, reg)
    for _ in range(5):
        r, _, _ = oracle.row_step(P, a, fi)
        np.testing.assert_allclose(P.sum(axis=1), a**fi * r ** (1 - fi), rtol=1e-13)
        c, _, _ = oracle.col_step(P, b, fi)
        np.testing.assert_allclose(P.sum(axis=0), b**fi * c ** (1 - fi), rtol=1e-13)
    res = oracle.sinkhorn(oracle.init_plan(C, reg), a, b, reg, reg_m, 5, record=True)
    np.testing.assert_allclose(res.plan, P, rtol=1e-14)


def test_transpose_symmetry():
    """(C^T, b, a) run row-first equals (C, a, b) run column-first, transposed."""
    C, a, b = rand_problem(9, 8, 5)
    reg, reg_m = 0.3, 0.8
    t1 = oracle.sinkhorn(oracle.init_plan(C.T, reg), b, a, reg, reg_m, 17)
    t2 = oracle.sinkhorn(oracle.init_plan(C, reg), a, b, reg, reg_m, 17, order="col_first")
    np.testing.assert_allclose(t1.plan, t2.plan.T, rtol=1e-13)


def test_permutation_equivariance():
    C, a, b = rand_problem(10, 9, 12)
    reg, reg_m = 0.15, 2.0
    rng = np.random.default_rng(0)
    pr, pc = rng.permutation(9), rng.permutation(12)
    base = oracle.sinkhorn(oracle.init_plan(C, reg), a, b, reg, reg_m, 30).plan
    perm = oracle.sinkhorn(oracle.init_plan(C[pr][:, pc], reg), a[pr], b[pc], reg, reg_m, 30).plan
    np.testing.assert_allclose(perm, base[pr][:, pc], rtol=1e-13)


def test_resume_equals_single_call():
    """The state is the plan alone: t1 then t2 iterations equal t1 + t2."""
    C, a, b = rand_problem(11, 6, 9)
    reg, reg_m = 0.2, 1.0
    P0 = oracle.init_plan(C, reg)
    one = oracle.sinkhorn(P0, a, b, reg, reg_m, 12).plan
    two = oracle.sinkhorn(oracle.sinkhorn(P0, a, b, reg, reg_m, 5).plan, a, b, reg, reg_m, 7).plan
    np.testing.assert_allclose(one, two, rtol=1e-14)


def test_degenerate_factors():
    C, a, b = rand_problem(12, 5, 4)
    a[2] = 0.0
    P0 = oracle.init_plan(C, 0.3)
    P0[4, :] = 0.0  # zero row sum with a positive target
    res = oracle.sinkhorn(P0, a, b, 0.3, 1.0, 3)
    assert np.all(res.plan[2] == 0.0)
    assert np.all(res.plan[4] == 0.0)
    assert res.status & oracle.STATUS_ZERO_SUM
    assert np.all(np.isfinite(res.plan))
    f, st = oracle.scaling_factor([0.0, 1.0, 2.0], [3.0, 0.0, 8.0], 0.5)
    np.testing.assert_allclose(f, [0.0, 1.0, 0.5])
    assert st == oracle.STATUS_ZERO_SUM
    _, st = oracle.scaling_factor([1.0], [np.nan], 0.5)
    assert st & oracle.STATUS_NONFINITE


def test_stopping_rule():
    C, a, b = rand_problem(13, 20, 15)
    reg, reg_m = 0.5, 1.0
    P0 = oracle.init_plan(C, reg)
    full = oracle.sinkhorn(P0, a, b, reg, reg_m, 2000, record=True)
    tol = 1e-8
    res = oracle.sinkhorn(P0, a, b, reg, reg_m, 2000, tol=tol)
    assert 2 <= res.iters_done < 2000
    assert res.err <= tol
    r = full.r
    t = res.iters_done
    assert np.abs(r[t - 1] - r[t - 2]).sum() / r[t - 1].sum() <= tol
    assert np.abs(r[t - 2] - r[t - 3]).sum() / r[t - 2].sum() > tol
    np.testing.assert_allclose(res.plan, oracle.sinkhorn(P0, a, b, reg, reg_m, t).plan, rtol=1e-14)
    # check_every=7: the stop lands on a multiple of 7
    res7 = oracle.sinkhorn(P0, a, b, reg, reg_m, 2000, tol=tol, check_every=7)
    assert res7.iters_done % 7 == 0 and res7.iters_done >= t


def test_transport_cost_is_a_plain_double_sum():
    C, a, b = rand_problem(14, 4, 3)
    P = oracle.sinkhorn(oracle.init_plan(C, 0.2), a, b, 0.2, 1.0, 4).plan
    s = 0.0
    for i in range(4):
        for j in range(3):
            s += P[i, j] * C[i, j]
    assert oracle.transport_cost(P, C) == pytest.approx(s, rel=1e-15)


def test_kernel_form_scalings_reproduce_plan():
    """diag(U) P0 diag(V) with U, V the cumulative factors equals the plan."""
    C, a, b = rand_problem(15, 10, 8)
    P0 = oracle.init_plan(C, 0.1)
    res = oracle.sinkhorn(P0, a, b, 0.1, 0.5, 20, record=True)
    U, V = oracle.kernel_form_scalings(res)
    np.testing.assert_allclose(U[:, None] * P0 * V[None, :], res.plan, rtol=1e-12)


def test_grad_matches_central_differences():
    """Adjoint of the unrolled iteration vs FP64 central differences."""
    N, M, T = 16, 16, 30
    C, a, b = rand_problem(16, N, M)
    reg, reg_m = 0.3, 1.0
    val, dC, da, db = oracle.sinkhorn_grad(C, a, b, reg, reg_m, T)
    ref = oracle.sinkhorn(oracle.init_plan(C, reg), a, b, reg, reg_m, T).plan
    assert val == pytest.approx(oracle.transport_cost(ref, C), rel=1e-12)

    def L(C_, a_, b_):
        P = oracle.sinkhorn(oracle.init_plan(C_, reg), a_, b_, reg, reg_m, T).plan
        return oracle.transport_cost(P, C_)

    h = 1e-6
    rng = np.random.default_rng(0)
    for _ in range(6):
        i, j = rng.integers(N), rng.integers(M)
        Cp, Cm = C.copy(), C.copy()
        Cp[i, j] += h
        Cm[i, j] -= h
        fd = (L(Cp, a, b) - L(Cm, a, b)) / (2 * h)
        assert dC[i, j] == pytest.approx(fd, rel=1e-6, abs=1e-10)
    for i in range(0, N, 5):
        ap, am = a.copy(), a.copy()
        ap[i] += h
        am[i] -= h
        assert da[i] == pytest.approx((L(C, ap, b) - L(C, am, b)) / (2 * h), rel=1e-6, abs=1e-10)
    for j in range(0, M, 5):
        bp, bm = b.copy(), b.copy()
        bp[j] += h
        bm[j] -= h
        assert db[j] == pytest.approx((L(C, a, bp) - L(C, a, bm)) / (2 * h), rel=1e-6, abs=1e-10)


@pytest.mark.parametrize("N,M,T", [(12, 9, 20), (256, 256, 200)])
def test_grad_matches_torch_autograd(N, M, T):
    """Adjoint vs torch CPU FP64 autograd of the plain unrolled literal loop."""
    torch = pytest.importorskip("torch")
    C, a, b = rand_problem(17 + N, N, M)
    reg, reg_m = 0.05 if N > 100 else 0.2, 1.0
    fi = oracle.fi_exponent(reg, reg_m)
    val, dC, da, db = oracle.sinkhorn_grad(C, a, b, reg, reg_m, T)
    Ct = torch.tensor(C, dtype=torch.float64, requires_grad=True)
    at = torch.tensor(a, dtype=torch.float64, requires_grad=True)
    bt = torch.tensor(b, dtype=torch.float64, requires_grad=True)
    P = torch.exp(-Ct / reg)
    for _ in range(T):
        P = P * ((at / P.sum(1)) ** fi)[:, None]
        P = P * ((bt / P.sum(0)) ** fi)[None, :]
    loss = (P * Ct).sum()
    loss.backward()
    assert val == pytest.approx(loss.item(), rel=1e-12)
    np.testing.assert_allclose(dC, Ct.grad.numpy(), rtol=1e-8, atol=1e-12 * np.abs(dC).max())
    np.testing.assert_allclose(da, at.grad.numpy(), rtol=1e-8, atol=1e-12 * np.abs(da).max())
    np.testing.assert_allclose(db, bt.grad.numpy(), rtol=1e-8, atol=1e-12 * np.abs(db).max())


def test_grad_magnitude_closed_forms_1x1():
    """Magnitudes of the adjoint's terms for one entry, by hand.  T = 0:
    dC = P - P C / reg from terms P and P C / reg.  T = 1: the value is
    dC = P - (1-fi)^2 P C / reg, da = fi (1-fi) P C / a, db = fi P C / b;
    the column step's correction -fi P C and the row step's -fi (1-fi) P C
    count positively in the magnitudes, which become P + (1+fi)^2 P C / reg,
    fi (1+fi) P C / a and fi P C / b."""
    C = np.array([[0.7]])
    a, b = np.array([0.3]), np.array([1.9])
    reg, reg_m = 0.5, 0.8
    fi = oracle.fi_exponent(reg, reg_m)
    dC0, da0, db0 = oracle.sinkhorn_grad_magnitude(C, a, b, reg, reg_m, 0)
    P0 = np.exp(-0.7 / reg)
    assert dC0[0, 0] == pytest.approx(P0 + P0 * 0.7 / reg, rel=1e-14)
    assert da0[0] == 0.0 and db0[0] == 0.0
    val, dC, da, db = oracle.sinkhorn_grad(C, a, b, reg, reg_m, 1)
    P = oracle.sinkhorn(oracle.init_plan(C, reg), a, b, reg, reg_m, 1).plan[0, 0]
    PC = P * 0.7
    assert dC[0, 0] == pytest.approx(P - (1 - fi) ** 2 * PC / reg, rel=1e-12)
    assert da[0] == pytest.approx(fi * (1 - fi) * PC / 0.3, rel=1e-12)
    assert db[0] == pytest.approx(fi * PC / 1.9, rel=1e-12)
    mC, ma, mb = oracle.sinkhorn_grad_magnitude(C, a, b, reg, reg_m, 1)
    assert mC[0, 0] == pytest.approx(P + (1 + fi) ** 2 * PC / reg, rel=1e-12)
    assert ma[0] == pytest.approx(fi * (1 + fi) * PC / 0.3, rel=1e-12)
    assert mb[0] == pytest.approx(fi * PC / 1.9, rel=1e-12)


def test_grad_magnitude_dominates_gradient():
    """Every entry's magnitude bounds the gradient entry (triangle
    inequality), and exceeds it by far where terms cancel."""
    C, a, b = rand_problem(18, 20, 15)
    for reg, reg_m, T in [(0.2, 1.0, 25), (0.1, 0.3, 10), (0.3, math.inf, 15)]:
        _, dC, da, db = oracle.sinkhorn_grad(C, a, b, reg, reg_m, T)
        mC, ma, mb = oracle.sinkhorn_grad_magnitude(C, a, b, reg, reg_m, T)
        for g, mg in ((dC, mC), (da, ma), (db, mb)):
            assert np.all(np.abs(g) <= mg * (1 + 1e-12))
        assert np.max(mC / np.abs(dC)) > 10.0


# --- the scaling-vector (POT) form of the unbalanced iteration -------------


@pytest.mark.parametrize("reg,reg_m", [(0.5, 1.0), (0.3, 0.4), (1.0, 5.0)])
def test_pot_rule_fixed_point_minimises_uot_objective(reg, reg_m):
    """The limit of u <- (a/Kv)^fi, v <- (b/K^T u)^fi is the minimiser of
    <P,C> + reg sum P(log P - 1) + reg_m KL(P1|a) + reg_m KL(P^T1|b), found
    here independently by Newton's method on the plan entries."""
    C, a, b = rand_problem(11, 7, 5, mass_a=1.0, mass_b=1.7)
    res = oracle.sinkhorn_pot(oracle.init_plan(C, reg), a, b, reg, reg_m, 4000)
    ref = convex.uot_newton(C, a, b, reg, reg_m)
    np.testing.assert_allclose(res.plan, ref, rtol=1e-9)
    f_ref = convex.uot_objective(ref, C, a, b, reg, reg_m)
    rng = np.random.default_rng(0)
    for _ in range(5):  # a local minimum: nearby plans cost more
        Pn = ref * np.exp(1e-3 * rng.standard_normal(ref.shape))
        assert convex.uot_objective(Pn, C, a, b, reg, reg_m) > f_ref


@pytest.mark.parametrize("reg,reg_m", [(0.05, 1.0), (0.3, 0.5), (1.0, 0.2)])
def test_pot_rule_one_by_one_closed_form(reg, reg_m):
    """1x1 with K = k: x = log u, y = log v obey x_t = fi (A - y_{t-1}),
    y_t = fi (B - x_t) with A = log(a/k), B = log(b/k), y_0 = 0, so
    y_T = d (1 - q^T)/(1 - q) with q = fi^2, d = fi B - fi^2 A."""
    fi = oracle.fi_exponent(reg, reg_m)
    a, b, k = 0.37, 2.9, 0.011
    A, B = math.log(a / k), math.log(b / k)
    q, d = fi * fi, fi * B - fi * fi * A
    for T in range(1, 41):
        y_prev = d * (1 - q ** (T - 1)) / (1 - q)
        x = fi * (A - y_prev)
        y = fi * (B - x)
        res = oracle.sinkhorn_pot([[k]], [a], [b], reg, reg_m, T)
        assert res.plan[0, 0] == pytest.approx(k * math.exp(x + y), rel=1e-12)


def test_pot_rule_balanced_case_equals_the_printed_rule():
    """fi = 1: both rules are balanced Sinkhorn, iterate by iterate."""
    C, a, b = rand_problem(5, 6, 9, mass_a=1.3, mass_b=1.3)
    P0 = oracle.init_plan(C, 0.2)
    for T in (1, 2, 7, 30):
        lit = oracle.sinkhorn(P0, a, b, 0.2, math.inf, T)
        pot = oracle.sinkhorn_pot(P0, a, b, 0.2, math.inf, T)
        np.testing.assert_allclose(pot.plan, lit.plan, rtol=1e-12)


def test_pot_rule_differs_from_the_printed_rule():
    """fi < 1: the printed rule and the scaling-vector rule have different
    limits (the printed rule's is balanced between rescaled marginals)."""
    C, a, b = rand_problem(9, 7, 5, mass_a=1.0, mass_b=1.5)
    P0 = oracle.init_plan(C, 0.3)
    lit = oracle.sinkhorn(P0, a, b, 0.3, 0.5, 3000).plan
    pot = oracle.sinkhorn_pot(P0, a, b, 0.3, 0.5, 3000).plan
    assert np.max(np.abs(lit - pot) / pot) > 0.05
    # The printed rule's limit has equal row and column mass; the
    # scaling-vector rule's generally does not.
    assert lit.sum(axis=1).sum() == pytest.approx(lit.sum(axis=0).sum(), rel=1e-12)


def test_pot_rule_zero_target_and_stopping():
    C, a, b = rand_problem(2, 5, 4)
    a[2] = 0.0
    res = oracle.sinkhorn_pot(oracle.init_plan(C, 0.3), a, b, 0.3, 1.0, 200, tol=1e-9)
    assert np.all(res.plan[2] == 0.0) and res.status == 0
    assert res.iters_done < 200 and res.err <= 1e-9


# --- the three-way (multi-marginal) form ------------------------------------


def test_tensor3_single_entry_closed_form():
    """1x1x1: with x = log P the iteration is x <- (1-fi) x + fi log a, then
    with log b, then with log c."""
    reg, reg_m, T = 0.4, 1.3, 9
    fi = oracle.fi_exponent(reg, reg_m)
    a, b, c = 0.7, 2.2, 0.35
    x = -0.9 / reg
    for _ in range(T):
        for t in (a, b, c):
            x = (1 - fi) * x + fi * math.log(t)
    got = oracle.sinkhorn_tensor3(np.exp(np.array([[[-0.9 / reg]]])), [a], [b], [c], reg, reg_m,
                                  T)
    assert got[0, 0, 0] == pytest.approx(math.exp(x), rel=1e-13)


def test_tensor3_with_one_mode_of_size_one_is_the_matrix_rule():
    """n3 = 1, fi = 1 and c = sum(b): after the mode-2 (column) step the total
    mass is sum(b), so the mode-3 factor is exactly 1 and the three-way rule
    is textbook Sinkhorn on the n1 x n2 matrix."""
    C, a, b = rand_problem(21, 9, 7)
    reg, T = 0.3, 25
    P0 = oracle.init_plan(C, reg)
    got = oracle.sinkhorn_tensor3(P0[:, :, None], a, b, [b.sum()], reg, math.inf, T)[:, :, 0]
    ref = oracle.sinkhorn(P0, a, b, reg, math.inf, T).plan
    np.testing.assert_allclose(got, ref, rtol=1e-12)


def test_tensor3_rank_one_cost_decouples():
    """C_ijk = p_i + q_j + r_k: the plan stays an outer product x (x) y (x) z,
    and each mode step rescales one vector by (target / (vector * product of
    the other two totals))^fi -- three vector recurrences written out here."""
    rng = np.random.default_rng(5)
    p, q, r = rng.random(4), rng.random(3), rng.random(5)
    C = p[:, None, None] + q[None, :, None] + r[None, None, :]
    a, b, c = rng.uniform(0.5, 1.5, 4), rng.uniform(0.5, 1.5, 3), rng.uniform(0.5, 1.5, 5)
    reg, reg_m, T = 0.5, 0.8, 12
    fi = oracle.fi_exponent(reg, reg_m)
    got = oracle.sinkhorn_tensor3(np.exp(-C / reg), a, b, c, reg, reg_m, T)
    x, y, z = np.exp(-p / reg), np.exp(-q / reg), np.exp(-r / reg)
    for _ in range(T):
        x = x * (a / (x * y.sum() * z.sum())) ** fi
        y = y * (b / (y * x.sum() * z.sum())) ** fi
        z = z * (c / (z * x.sum() * y.sum())) ** fi
    np.testing.assert_allclose(got, x[:, None, None] * y[None, :, None] * z[None, None, :],
                               rtol=1e-12)


def test_tensor3_mode_marginal_after_each_step():
    """Per-step identity: after the last (mode-3) step the mode-3 sums are
    c^fi s^(1-fi), s the sums before it; with fi = 1 they equal c."""
    rng = np.random.default_rng(6)
    P0 = rng.random((5, 4, 6))
    a, b, c = rng.random(5), rng.random(4), rng.random(6) + 0.5
    got = oracle.sinkhorn_tensor3(P0, a, b, c, 0.2, math.inf, 3)
    np.testing.assert_allclose(got.sum(axis=(0, 1)), c, rtol=1e-12)
