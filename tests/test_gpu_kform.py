"""Kernel form diag(U) K diag(V) (read-only K) against the FP64 oracle.

FP32 K: plan entries, U, V and cost within 1e-5 (the FP32 tolerance).
BF16/FP16 K: K is rounded once (relative 2^-8 / 2^-11) and U, V stay FP32,
so entries stay within about one rounding of K; the tolerance is 1e-2 on plan
entries and cost, on the 8192^2 instance of the reduced-precision workload
(2-D uniform points, reg 0.1, reg_m 1.0, 300 iterations).
"""

import math

import numpy as np
import pytest

import oracle
from oracle import convex
from paper_2412_11079_gb300 import workloads

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

FP32_TOL = 1e-5
LOW_TOL = 1e-2


@pytest.fixture(scope="module")
def uot():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2412_11079_gb300 import build, uot as u
    build.build()
    u.load()
    return u


def rel_err(got, ref):
    got = np.asarray(got, np.float64)
    floor = 1e-6 * np.abs(ref).max()
    return float(np.max(np.abs(got - ref) / np.maximum(np.abs(ref), floor)))


def dev(x):
    return torch.from_numpy(np.ascontiguousarray(x)).cuda()


def kform_gpu(uot, p, dtype=torch.float32, log2_scale=0, iters=None, tol=0.0, ld=None, rule=0,
              schedule=0):
    n, m = p.C.shape
    C = dev(p.C)
    store = torch.zeros((n, ld or m), dtype=dtype, device="cuda")
    K = store[:, :m]
    opt = uot.options(uot.dtype_code(dtype), rule=rule, schedule=schedule)
    uot.uot_init_kernel_scaled(C, K, p.reg, log2_scale, opt)
    U, V, res = uot.uot_sinkhorn_kform(K, dev(p.a), dev(p.b), p.reg, p.reg_m,
                                       p.iters if iters is None else iters, tol, log2_scale,
                                       opt=opt)
    plan = uot.uot_kform_plan(K, U, V)
    cost = uot.uot_kform_cost(K, U, V, C).item()
    torch.cuda.synchronize()
    return plan.double().cpu().numpy(), cost, U.double().cpu().numpy(), \
        V.double().cpu().numpy(), res


@pytest.mark.parametrize("n,m", [(1, 1), (3, 5), (33, 31), (127, 1000), (1000, 1025),
                                 (257, 4099), (65, 16387), (40, 40000)])
@pytest.mark.parametrize("schedule", [1, 0], ids=["passes", "auto"])
def test_fp32_kernel_form_matches_oracle(uot, n, m, schedule):
    p = workloads.uniform2d(seed=n * 31 + m, n=n, m=m, reg=0.1, reg_m=0.7, iters=15)
    plan, cost, U, V, res = kform_gpu(uot, p, schedule=schedule)
    ref = oracle.sinkhorn(oracle.init_plan(p.C, p.reg), p.a, p.b, p.reg, p.reg_m, p.iters,
                          record=True)
    Ur, Vr = oracle.kernel_form_scalings(ref)
    assert res.iters_done == p.iters and res.dev_status == 0
    assert rel_err(plan, ref.plan) <= FP32_TOL
    # U, V are the oracle's cumulative factors up to one exact power of two.
    g = 2.0 ** np.round(np.log2(np.median(U / Ur)))
    np.testing.assert_allclose(U, Ur * g, rtol=FP32_TOL)
    np.testing.assert_allclose(V, Vr / g, rtol=FP32_TOL)
    c_ref = oracle.transport_cost(ref.plan, p.C)
    assert abs(cost - c_ref) <= FP32_TOL * abs(c_ref)


@pytest.mark.parametrize("dtype,tol", [(torch.float32, FP32_TOL), (torch.bfloat16, LOW_TOL)])
def test_balanced_kernel_form(uot, dtype, tol):
    """reg_m = inf (fi = 1): balanced Sinkhorn, the special case the paper's
    introduction names for the same interleaving.  The kernel form follows the
    oracle, and the plan's column sums equal b after the last iteration in
    either storage precision (V is formed from the stored K's own sums)."""
    p = workloads.uniform2d(seed=21, n=700, m=1500, reg=0.1, reg_m=math.inf, iters=30)
    plan, cost, U, V, res = kform_gpu(uot, p, dtype=dtype)
    ref = oracle.sinkhorn(oracle.init_plan(p.C, p.reg), p.a, p.b, p.reg, math.inf, p.iters)
    assert res.dev_status == 0 and res.iters_done == p.iters
    assert rel_err(plan, ref.plan) <= tol
    np.testing.assert_allclose(plan.sum(axis=0), p.b, rtol=2e-5)


def test_balanced_limit_is_entropic_ot(uot):
    """fi = 1 and equal masses: the kernel form's limit is the entropic OT
    plan, here from Newton's method on the dual (no Sinkhorn step shared)."""
    p = workloads.uniform2d(seed=22, n=40, m=30, reg=0.1, reg_m=math.inf, iters=300)
    p.b = (p.b.astype(np.float64) * (p.a.astype(np.float64).sum()
                                     / p.b.astype(np.float64).sum())).astype(np.float32)
    plan, cost, U, V, res = kform_gpu(uot, p)
    a = p.a.astype(np.float64)
    b = p.b.astype(np.float64)
    b *= a.sum() / b.sum()
    ref = convex.entropic_ot_newton(p.C.astype(np.float64), a, b, p.reg)
    assert res.dev_status == 0
    assert rel_err(plan, ref) <= FP32_TOL


def test_kernel_form_misaligned_ld_and_scale(uot):
    """ld*4 % 16 != 0 takes the path without bulk copies; a storage scale of
    2^5 must be undone by U."""
    p = workloads.uniform2d(seed=3, n=200, m=301, reg=0.1, reg_m=1.0, iters=20)
    plan, _, _, _, _ = kform_gpu(uot, p, ld=303, log2_scale=5)
    ref = oracle.sinkhorn(oracle.init_plan(p.C, p.reg), p.a, p.b, p.reg, p.reg_m, p.iters)
    assert rel_err(plan, ref.plan) <= FP32_TOL


def test_kernel_form_stopping_rule(uot):
    p = workloads.uniform2d(seed=9, n=200, m=150, reg=0.3, reg_m=1.0, iters=3000)
    tol = 1e-6
    ref = oracle.sinkhorn(oracle.init_plan(p.C, p.reg), p.a, p.b, p.reg, p.reg_m, p.iters, tol=tol)
    plan, _, _, _, res = kform_gpu(uot, p, tol=tol)
    assert abs(res.iters_done - ref.iters_done) <= 2
    ref2 = oracle.sinkhorn(oracle.init_plan(p.C, p.reg), p.a, p.b, p.reg, p.reg_m,
                           res.iters_done)
    assert rel_err(plan, ref2.plan) <= FP32_TOL


def test_gauge_keeps_scalings_in_range(uot):
    """Masses 1 and 1.5: the cumulative factors drift as k^t, k ~ 0.69, so
    without the gauge U would underflow FP32 within ~250 iterations."""
    p = workloads.uniform2d(seed=6, n=64, m=80, reg=0.2, reg_m=1.0, iters=2000)
    plan, _, U, V, res = kform_gpu(uot, p)
    assert res.dev_status == 0
    assert np.all(np.isfinite(U)) and np.all(np.isfinite(V))
    assert 1e-30 < np.abs(U).max() < 1e30 and 1e-30 < np.abs(V).max() < 1e30
    ref = oracle.sinkhorn(oracle.init_plan(p.C, p.reg), p.a, p.b, p.reg, p.reg_m, p.iters)
    assert rel_err(plan, ref.plan) <= FP32_TOL


def test_scaled_fp16_init(uot):
    p = workloads.uniform2d(seed=4, n=70, m=90, reg=0.1)
    C = dev(p.C)
    K = torch.empty(C.shape, dtype=torch.float16, device="cuda")
    uot.uot_init_kernel_scaled(C, K, p.reg, 15, uot.options(uot.UOT_F16))
    ref = torch.from_numpy(np.exp(-p.C.astype(np.float64) / p.reg) * 2.0 ** 15)
    got = K.double().cpu()
    assert torch.all(torch.isfinite(got))
    assert ((got - ref).abs() <= ref.abs() * 2.0 ** -11 * 1.01).all()


@pytest.fixture(scope="module")
def precision_ref():
    """FP64 oracle on the 8192^2 instance of the reduced-precision workload."""
    p = workloads.precision_case(seed=0, n=8192, m=8192, iters=300)
    ref = oracle.sinkhorn(oracle.init_plan(p.C, p.reg), p.a, p.b, p.reg, p.reg_m, p.iters)
    return p, ref.plan, oracle.transport_cost(ref.plan, p.C)


@pytest.mark.slow
@pytest.mark.parametrize("dtype,scale,tol", [("float32", 0, FP32_TOL), ("bfloat16", 0, LOW_TOL),
                                             ("float16", 15, LOW_TOL)])
def test_precision_case_8192(uot, precision_ref, dtype, scale, tol):
    p, ref_plan, ref_cost = precision_ref
    plan, cost, _, _, res = kform_gpu(uot, p, getattr(torch, dtype), scale)
    assert res.iters_done == 300 and res.dev_status == 0
    assert rel_err(plan, ref_plan) <= tol
    assert abs(cost - ref_cost) <= tol * abs(ref_cost)


def test_kernel_form_rejects_bad_arguments(uot):
    p = workloads.uniform2d(seed=5, n=10, m=12, iters=2)
    K = torch.ones((10, 12), device="cuda")
    with pytest.raises(uot.UotError):
        uot.uot_sinkhorn_kform(K, dev(p.a), dev(p.b), p.reg, p.reg_m, 2, k_log2_scale=0.5)
    with pytest.raises(uot.UotError):
        uot.uot_sinkhorn_kform(K, dev(p.a), dev(p.b), p.reg, p.reg_m, 2,
                               opt=uot.options(algo=uot.UOT_ALGO_MULTIPASS))


# --- the scaling-vector (POT) rule -------------------------------------------


@pytest.mark.parametrize("n,m", [(1, 1), (3, 5), (33, 31), (127, 1000), (1000, 1025),
                                 (65, 16387), (40, 40000)])
def test_pot_rule_fp32_kernel_form_matches_oracle(uot, n, m):
    """u <- (a/Kv)^fi, v <- (b/K^T u)^fi on read-only K against the FP64
    oracle of the same rule (FP32 tolerance), rows from 1 to 40000 wide
    (clusters of CTAs per row above 16384)."""
    p = workloads.uniform2d(seed=n * 17 + m, n=n, m=m, reg=0.1, reg_m=0.7, iters=25)
    plan, cost, U, V, res = kform_gpu(uot, p, rule=uot.UOT_RULE_POT)
    ref = oracle.sinkhorn_pot(oracle.init_plan(p.C, p.reg), p.a, p.b, p.reg, p.reg_m, p.iters)
    assert res.iters_done == p.iters and res.dev_status == 0
    assert rel_err(plan, ref.plan) <= FP32_TOL
    c_ref = oracle.transport_cost(ref.plan, p.C)
    assert abs(cost - c_ref) <= FP32_TOL * abs(c_ref)


@pytest.mark.parametrize("dtype,log2_scale", [(torch.bfloat16, 0), (torch.float16, 15)])
def test_pot_rule_reduced_precision_kernel_form(uot, dtype, log2_scale):
    """16-bit K (FP16 stored x 2^15, the scale folded into U) under the
    scaling-vector rule, on a 2048^2 instance of the reduced-precision
    generator; 1e-2 on plan entries and cost."""
    p = workloads.precision_case(seed=5, n=2048, m=2048, iters=100)
    plan, cost, U, V, res = kform_gpu(uot, p, dtype=dtype, log2_scale=log2_scale,
                                      rule=uot.UOT_RULE_POT)
    ref = oracle.sinkhorn_pot(oracle.init_plan(p.C, p.reg), p.a, p.b, p.reg, p.reg_m, p.iters)
    assert res.dev_status == 0
    assert rel_err(plan, ref.plan) <= LOW_TOL
    c_ref = oracle.transport_cost(ref.plan, p.C)
    assert abs(cost - c_ref) <= LOW_TOL * abs(c_ref)


def test_pot_rule_stopping_rule(uot):
    """The device stopping rule under the scaling-vector rule stops where the
    oracle of that rule stops."""
    p = workloads.uniform2d(seed=3, n=300, m=200, reg=0.2, reg_m=2.0, iters=400)
    tol = 1e-6
    plan, cost, U, V, res = kform_gpu(uot, p, tol=tol, rule=uot.UOT_RULE_POT)
    ref = oracle.sinkhorn_pot(oracle.init_plan(p.C, p.reg), p.a, p.b, p.reg, p.reg_m, p.iters,
                              tol=tol)
    assert ref.iters_done < p.iters
    assert abs(res.iters_done - ref.iters_done) <= 1 and res.err <= tol
    ref2 = oracle.sinkhorn_pot(oracle.init_plan(p.C, p.reg), p.a, p.b, p.reg, p.reg_m,
                               res.iters_done)
    assert rel_err(plan, ref2.plan) <= FP32_TOL


def test_pot_rule_rejected_where_unsupported(uot):
    """In-place plans keep no scalings, and the adjoint is for the printed
    rule: both refuse the scaling-vector rule."""
    p = workloads.uniform2d(seed=4, n=16, m=12, iters=3)
    P = torch.from_numpy(oracle.init_plan(p.C, p.reg).astype(np.float32)).cuda()
    with pytest.raises(uot.UotError, match="unsupported"):
        uot.uot_sinkhorn(P, dev(p.a), dev(p.b), p.reg, p.reg_m, 3, 0.0,
                         opt=uot.options(rule=uot.UOT_RULE_POT))
    K = torch.from_numpy(oracle.init_plan(p.C, p.reg).astype(np.float32)).cuda()
    with pytest.raises(uot.UotError, match="unsupported"):
        uot.uot_sinkhorn_kform_save(K, dev(p.a), dev(p.b), p.reg, p.reg_m, 3,
                                    opt=uot.options(rule=uot.UOT_RULE_POT))
