"""uot_sinkhorn's two storages and its deterministic mode, through the C ABI,
against the FP64 oracle.

* The large workload's generator (64-D Gaussian clouds, C / max, Dirichlet
  marginals of masses 1 and 2, reg 0.1, reg_m 0.5) run for the full 500
  iterations from P0 at N = 2048, M = 16384: 16384 columns take the same
  fused configuration (one 512-thread CTA per row, 8 vectors per thread),
  grid, ring and row schedule as the 16384^2 benchmark, and the oracle
  finishes in about half a minute.  Plan entries and cost within 1e-5.
* Kernel-form storage (the buffer kept as K, read-only, with FP32
  scalings) on ragged shapes, rows wider than one CTA, the path without bulk
  copies, the stopping rule, the scaling-vector rule and BF16.
* Deterministic mode: two runs give the same bits (plan, and U, V of the
  kernel form), in both storages and with the stopping rule.
"""

import math

import numpy as np
import pytest

import oracle
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


def solve(uot, p, iters=None, storage=0, det=False, dtype=torch.float32, tol=0.0, ld=None,
          rule=0, C=None):
    n, m = p.C.shape
    C = dev(p.C) if C is None else C
    store = torch.zeros((n, ld or m), dtype=dtype, device="cuda")
    plan = store[:, :m]
    opt = uot.options(uot.dtype_code(dtype), storage=storage, deterministic=det, rule=rule)
    uot.uot_init_kernel(C, plan, p.reg, opt)
    res = uot.uot_sinkhorn(plan, dev(p.a), dev(p.b), p.reg, p.reg_m,
                           p.iters if iters is None else iters, tol,
                           ws=uot.workspace(n, m, opt), opt=opt, check_status=False)
    cost = uot.uot_cost(plan, C).item()
    torch.cuda.synchronize()
    return plan, cost, res


@pytest.fixture(scope="module")
def large500():
    p = workloads.large_case(seed=0, n=2048, m=16384, iters=500)
    ref = oracle.sinkhorn(oracle.init_plan(p.C, p.reg), p.a, p.b, p.reg, p.reg_m, p.iters).plan
    return p, ref, oracle.transport_cost(ref, p.C)


@pytest.mark.slow
@pytest.mark.parametrize("storage", [0, 1], ids=["inplace", "kform"])
def test_large_workload_500_iterations_matches_oracle(uot, large500, storage):
    p, ref, ref_cost = large500
    plan, cost, res = solve(uot, p, storage=storage)
    assert res.iters_done == 500 and res.dev_status == 0
    assert rel_err(plan.double().cpu().numpy(), ref) <= FP32_TOL
    assert abs(cost - ref_cost) <= FP32_TOL * abs(ref_cost)


@pytest.mark.parametrize("n,m", [(1, 1), (3, 5), (33, 31), (1000, 127), (257, 4099),
                                 (300, 16384), (65, 16387), (40, 40000)])
def test_kform_storage_matches_oracle(uot, n, m):
    p = workloads.uniform2d(seed=n * 13 + m, n=n, m=m, reg=0.1, reg_m=0.7, iters=15)
    plan, cost, res = solve(uot, p, storage=1)
    ref = oracle.sinkhorn(oracle.init_plan(p.C, p.reg), p.a, p.b, p.reg, p.reg_m, p.iters)
    assert res.iters_done == p.iters and res.dev_status == ref.status == 0
    assert rel_err(plan.double().cpu().numpy(), ref.plan) <= FP32_TOL
    c_ref = oracle.transport_cost(ref.plan, p.C)
    assert abs(cost - c_ref) <= FP32_TOL * abs(c_ref)


@pytest.mark.parametrize("ld_extra", [1, 64])
def test_kform_storage_leading_dimension(uot, ld_extra):
    """ld > m (ld*4 % 16 != 0 takes the path without bulk copies); the
    padding is left untouched by the last sweep."""
    p = workloads.uniform2d(seed=5, n=300, m=777, reg=0.08, reg_m=1.5, iters=12)
    n, m = p.C.shape
    C = dev(p.C)
    store = torch.zeros((n, m + ld_extra), device="cuda")
    plan = store[:, :m]
    opt = uot.options(storage=1)
    uot.uot_init_kernel(C, plan, p.reg, opt)
    uot.uot_sinkhorn(plan, dev(p.a), dev(p.b), p.reg, p.reg_m, p.iters, opt=opt)
    ref = oracle.sinkhorn(oracle.init_plan(p.C, p.reg), p.a, p.b, p.reg, p.reg_m, p.iters)
    assert rel_err(plan.double().cpu().numpy(), ref.plan) <= FP32_TOL
    assert torch.count_nonzero(store[:, m:]).item() == 0


def test_kform_storage_stopping_rule(uot):
    p = workloads.uniform2d(seed=9, n=200, m=150, reg=0.3, reg_m=1.0, iters=3000)
    tol = 1e-6
    ref = oracle.sinkhorn(oracle.init_plan(p.C, p.reg), p.a, p.b, p.reg, p.reg_m, p.iters,
                          tol=tol)
    plan, _, res = solve(uot, p, storage=1, tol=tol)
    assert 2 <= ref.iters_done < 3000
    assert abs(res.iters_done - ref.iters_done) <= 2
    ref2 = oracle.sinkhorn(oracle.init_plan(p.C, p.reg), p.a, p.b, p.reg, p.reg_m,
                           res.iters_done)
    assert rel_err(plan.double().cpu().numpy(), ref2.plan) <= FP32_TOL
    assert res.err <= tol


def test_kform_storage_pot_rule(uot):
    """The scaling-vector rule needs the scalings, which kernel-form storage
    keeps: uot_sinkhorn accepts it there and follows the oracle's POT form."""
    p = workloads.uniform2d(seed=23, n=400, m=600, reg=0.1, reg_m=0.6, iters=40)
    plan, _, res = solve(uot, p, storage=1, rule=1)
    ref = oracle.sinkhorn_pot(oracle.init_plan(p.C, p.reg), p.a, p.b, p.reg, p.reg_m, p.iters)
    assert res.dev_status == 0
    assert rel_err(plan.double().cpu().numpy(), ref.plan) <= FP32_TOL
    with pytest.raises(uot.UotError) as ei:
        solve(uot, p, storage=0, rule=1)
    assert ei.value.status == uot.UOT_ERR_UNSUPPORTED


def test_kform_storage_bf16(uot):
    """BF16 buffer: K is the BF16 initial plan, rounded once; the result is
    rounded once more at the end, so the reduced-precision bar holds."""
    p = workloads.uniform2d(seed=24, n=1000, m=1500, reg=0.1, reg_m=1.0, iters=100)
    plan, cost, res = solve(uot, p, storage=1, dtype=torch.bfloat16)
    ref = oracle.sinkhorn(oracle.init_plan(p.C, p.reg), p.a, p.b, p.reg, p.reg_m, p.iters)
    assert res.dev_status == 0
    assert rel_err(plan.double().cpu().numpy(), ref.plan) <= LOW_TOL
    c_ref = oracle.transport_cost(ref.plan, p.C)
    assert abs(cost - c_ref) <= LOW_TOL * abs(c_ref)


@pytest.mark.parametrize("storage", [0, 1], ids=["inplace", "kform"])
@pytest.mark.parametrize("n,m", [(1500, 5000), (300, 20000), (777, 16384)])
def test_deterministic_runs_are_bit_identical(uot, storage, n, m):
    """Static rows and slot-ordered column sums: the same inputs give the
    same bits, for single-CTA rows and rows split over a cluster."""
    p = workloads.uniform2d(seed=n + m, n=n, m=m, reg=0.1, reg_m=0.8, iters=20)
    C = dev(p.C)
    a, _, r1 = solve(uot, p, storage=storage, det=True, C=C)
    b, _, r2 = solve(uot, p, storage=storage, det=True, C=C)
    assert r1.dev_status == r2.dev_status == 0
    assert torch.equal(a, b)
    ref = oracle.sinkhorn(oracle.init_plan(p.C, p.reg), p.a, p.b, p.reg, p.reg_m, p.iters)
    assert rel_err(a.double().cpu().numpy(), ref.plan) <= FP32_TOL


def test_deterministic_kernel_form_scalings_and_stop(uot):
    """uot_sinkhorn_kform in deterministic mode: U and V are bit-identical
    between runs, and the stopping rule stops both at the same iteration."""
    p = workloads.uniform2d(seed=25, n=900, m=3000, reg=0.3, reg_m=1.0, iters=3000)
    n, m = p.C.shape
    C, a, b = dev(p.C), dev(p.a), dev(p.b)
    K = torch.empty((n, m), device="cuda")
    opt = uot.options(deterministic=True)
    uot.uot_init_kernel(C, K, p.reg, opt)
    outs = []
    for _ in range(2):
        U, V, res = uot.uot_sinkhorn_kform(K, a, b, p.reg, p.reg_m, p.iters, 1e-6, opt=opt,
                                           ws=uot.workspace(n, m, opt))
        outs.append((U.clone(), V.clone(), res))
    (U1, V1, r1), (U2, V2, r2) = outs
    assert r1.iters_done == r2.iters_done < 3000 and r1.err == r2.err
    assert torch.equal(U1, U2) and torch.equal(V1, V2)
    ref = oracle.sinkhorn(oracle.init_plan(p.C, p.reg), p.a, p.b, p.reg, p.reg_m, r1.iters_done)
    plan = uot.uot_kform_plan(K, U1, V1).double().cpu().numpy()
    assert rel_err(plan, ref.plan) <= FP32_TOL


def test_deterministic_16bit_in_place(uot):
    p = workloads.uniform2d(seed=26, n=500, m=9000, reg=0.5, reg_m=1.0, iters=4)
    # masses n*m and 1.5*n*m keep the entries O(1), in FP16's normal range
    p.a = (p.a * np.float32(500 * 9000)).astype(np.float32)
    p.b = (p.b * np.float32(500 * 9000)).astype(np.float32)
    C = dev(p.C)
    x, _, _ = solve(uot, p, det=True, dtype=torch.float16, C=C)
    y, _, _ = solve(uot, p, det=True, dtype=torch.float16, C=C)
    assert torch.equal(x, y)
