"""The persistent schedule (every iteration in one cooperative launch, rows
held in shared memory across the GPU's CTAs) against the FP64 oracle and
against the one-launch-per-iteration schedule, through the C ABI.

Tolerances as everywhere: FP32 plan entries and cost within 1e-5 of the
oracle; 16-bit in-place plans within the rounding-count bound 1.25 (2T+1) u.
"""

import math

import numpy as np
import pytest

import oracle
from paper_2412_11079_gb300 import workloads

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

FP32_TOL = 1e-5
PASSES, PERSISTENT = 1, 2
# launches of one solve: the workspace reset (kernel-form storage also sets
# U, V and the gauge: two more) and the one persistent launch
LAUNCHES = {0: 2, 1: 4}


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


def solve(uot, p, schedule=PERSISTENT, storage=0, dtype=torch.float32, tol=0.0, max_ctas=0,
          iters=None, check_status=True):
    n, m = p.C.shape
    C = dev(p.C)
    plan = torch.empty((n, m), dtype=dtype, device="cuda")
    opt = uot.options(uot.dtype_code(dtype), storage=storage, schedule=schedule,
                      max_ctas=max_ctas)
    uot.uot_init_kernel(C, plan, p.reg, opt)
    before = uot.uot_launch_count()
    res = uot.uot_sinkhorn(plan, dev(p.a), dev(p.b), p.reg, p.reg_m,
                           p.iters if iters is None else iters, tol, opt=opt,
                           check_status=check_status)
    launches = uot.uot_launch_count() - before
    cost = uot.uot_cost(plan, C).item()
    torch.cuda.synchronize()
    return plan.double().cpu().numpy(), cost, res, launches


def oracle_of(p, iters=None, tol=0.0):
    res = oracle.sinkhorn(oracle.init_plan(p.C, p.reg), p.a, p.b, p.reg, p.reg_m,
                          p.iters if iters is None else iters, tol=tol)
    return res, oracle.transport_cost(res.plan, p.C)


@pytest.mark.parametrize("storage", [0, 1], ids=["inplace", "kform"])
def test_small_workload(uot, storage):
    """N=M=1024, 2-D uniform points, reg 0.05, reg_m 1.0, 100 iterations:
    the set-up launches and one persistent launch."""
    p = workloads.small_case(seed=0)
    got, cost, res, launches = solve(uot, p, storage=storage)
    ref, ref_cost = oracle_of(p)
    assert launches == LAUNCHES[storage] and res.iters_done == 100 and res.dev_status == 0
    assert rel_err(got, ref.plan) <= FP32_TOL
    assert abs(cost - ref_cost) <= FP32_TOL * abs(ref_cost)


@pytest.mark.parametrize("n,m", [(1, 1), (1, 3000), (3000, 1), (151, 153), (152, 64),
                                 (153, 1000), (700, 2048), (2048, 2048), (5, 20000)])
@pytest.mark.parametrize("storage", [0, 1], ids=["inplace", "kform"])
def test_shapes(uot, n, m, storage):
    """Ragged row blocks (fewer rows than CTAs, one more row than a multiple
    of the grid), a single row or column, up to the largest plans held."""
    p = workloads.uniform2d(seed=n * 101 + m, n=n, m=m, reg=0.1, reg_m=0.7, iters=12)
    got, cost, res, launches = solve(uot, p, storage=storage)
    ref, ref_cost = oracle_of(p)
    assert launches == LAUNCHES[storage] and res.dev_status == 0
    assert rel_err(got, ref.plan) <= FP32_TOL
    assert abs(cost - ref_cost) <= FP32_TOL * abs(ref_cost)


def test_kernel_form_entry_point_scalings(uot):
    """uot_sinkhorn_kform on the persistent schedule: K untouched, U and V
    the oracle's cumulative factors up to one power of two."""
    p = workloads.uniform2d(seed=40, n=500, m=700, reg=0.1, reg_m=0.7, iters=30)
    n, m = p.C.shape
    C = dev(p.C)
    K = torch.empty((n, m), device="cuda")
    opt = uot.options(schedule=PERSISTENT)
    uot.uot_init_kernel(C, K, p.reg, opt)
    K0 = K.clone()
    U, V, res = uot.uot_sinkhorn_kform(K, dev(p.a), dev(p.b), p.reg, p.reg_m, p.iters, opt=opt)
    torch.cuda.synchronize()
    assert torch.equal(K, K0) and res.iters_done == p.iters
    ref = oracle.sinkhorn(oracle.init_plan(p.C, p.reg), p.a, p.b, p.reg, p.reg_m, p.iters,
                          record=True)
    Ur, Vr = oracle.kernel_form_scalings(ref)
    U = U.double().cpu().numpy()
    V = V.double().cpu().numpy()
    g = 2.0 ** np.round(np.log2(np.median(U / Ur)))
    np.testing.assert_allclose(U, Ur * g, rtol=FP32_TOL)
    np.testing.assert_allclose(V, Vr / g, rtol=FP32_TOL)


@pytest.mark.parametrize("storage", [0, 1], ids=["inplace", "kform"])
def test_stopping_rule(uot, storage):
    p = workloads.uniform2d(seed=9, n=600, m=450, reg=0.3, reg_m=1.0, iters=3000)
    tol = 1e-6
    ref, _ = oracle_of(p, tol=tol)
    got, _, res, _ = solve(uot, p, storage=storage, tol=tol)
    assert 2 <= ref.iters_done < 3000
    assert abs(res.iters_done - ref.iters_done) <= 2 and res.err <= tol
    ref2, _ = oracle_of(p, iters=res.iters_done)
    assert rel_err(got, ref2.plan) <= FP32_TOL


@pytest.mark.parametrize("dtype,u", [(torch.bfloat16, 2.0 ** -8), (torch.float16, 2.0 ** -11)])
def test_16bit_in_place_rounding_bound(uot, dtype, u):
    T = 4
    n, m = 129, 1000
    p = workloads.uniform2d(seed=41, n=n, m=m, reg=0.5, reg_m=1.0, iters=T)
    p.a = (p.a * np.float32(n * m)).astype(np.float32)
    p.b = (p.b * np.float32(n * m)).astype(np.float32)
    got, cost, res, launches = solve(uot, p, dtype=dtype)
    ref, ref_cost = oracle_of(p)
    bound = 1.25 * (2 * T + 1) * u + 1e-5
    assert launches == 2
    assert rel_err(got, ref.plan) <= bound
    assert abs(cost - ref_cost) <= bound * abs(ref_cost)


def test_pot_rule_kernel_form_storage(uot):
    p = workloads.uniform2d(seed=42, n=300, m=500, reg=0.1, reg_m=0.6, iters=40)
    n, m = p.C.shape
    C = dev(p.C)
    plan = torch.empty((n, m), device="cuda")
    opt = uot.options(storage=1, schedule=PERSISTENT, rule=uot.UOT_RULE_POT)
    uot.uot_init_kernel(C, plan, p.reg, opt)
    uot.uot_sinkhorn(plan, dev(p.a), dev(p.b), p.reg, p.reg_m, p.iters, opt=opt)
    ref = oracle.sinkhorn_pot(oracle.init_plan(p.C, p.reg), p.a, p.b, p.reg, p.reg_m, p.iters)
    assert rel_err(plan.double().cpu().numpy(), ref.plan) <= FP32_TOL


def test_fewer_ctas_and_degenerate_rows(uot):
    """max_ctas = 7: each CTA holds 100 rows; a zero row and zero targets
    follow the degenerate readings and report ZERO_SUM."""
    p = workloads.uniform2d(seed=43, n=700, m=300, reg=0.1, reg_m=1.0, iters=10)
    p.a[3] = 0.0
    p.b[7] = 0.0
    P0 = oracle.init_plan(p.C, p.reg)
    P0[10, :] = 0.0
    n, m = p.C.shape
    plan = dev(P0.astype(np.float32))
    opt = uot.options(schedule=PERSISTENT, max_ctas=7)
    res = uot.uot_sinkhorn(plan, dev(p.a), dev(p.b), p.reg, p.reg_m, p.iters, opt=opt,
                           check_status=False)
    ref = oracle.sinkhorn(P0, p.a, p.b, p.reg, p.reg_m, p.iters)
    got = plan.double().cpu().numpy()
    assert res.dev_status & uot.UOT_DEV_ZERO_SUM and ref.status & oracle.STATUS_ZERO_SUM
    assert np.all(got[3] == 0) and np.all(got[:, 7] == 0) and np.all(got[10] == 0)
    assert rel_err(got, ref.plan) <= FP32_TOL


def test_refused_where_it_does_not_fit(uot):
    """A plan larger than the CTAs' shared memory, or a forced fused
    configuration, cannot take the persistent schedule."""
    big = torch.empty((2048, 16384), device="cuda")
    a = torch.ones(2048, device="cuda")
    b = torch.ones(16384, device="cuda")
    with pytest.raises(uot.UotError) as ei:
        uot.uot_sinkhorn(big, a, b, 0.1, 1.0, 1, opt=uot.options(schedule=PERSISTENT))
    assert ei.value.status == uot.UOT_ERR_UNSUPPORTED
    small = torch.ones((10, 10), device="cuda")
    with pytest.raises(uot.UotError) as ei:
        uot.uot_sinkhorn(small, a[:10], b[:10], 0.1, 1.0, 1,
                         opt=uot.options(schedule=PERSISTENT, deterministic=True))
    assert ei.value.status == uot.UOT_ERR_UNSUPPORTED


def test_graph_capture_replays(uot):
    p = workloads.uniform2d(seed=44, n=256, m=512, reg=0.1, reg_m=1.0, iters=20)
    n, m = p.C.shape
    C, a, b = dev(p.C), dev(p.a), dev(p.b)
    plan = torch.empty((n, m), device="cuda")
    opt = uot.options(schedule=PERSISTENT)
    ws = uot.workspace(n, m, opt)
    s = torch.cuda.Stream()
    s.wait_stream(torch.cuda.current_stream())
    g = torch.cuda.CUDAGraph()
    with torch.cuda.stream(s):
        uot.uot_init_kernel(C, plan, p.reg, opt, stream=s)
        uot.uot_sinkhorn(plan, a, b, p.reg, p.reg_m, p.iters, ws=ws, opt=opt, stream=s,
                         sync=False)
        torch.cuda.synchronize()
        with torch.cuda.graph(g, stream=s):
            uot.uot_init_kernel(C, plan, p.reg, opt, stream=s)
            uot.uot_sinkhorn(plan, a, b, p.reg, p.reg_m, p.iters, ws=ws, opt=opt, stream=s,
                             sync=False)
    for _ in range(2):
        g.replay()
    torch.cuda.synchronize()
    ref, _ = oracle_of(p)
    assert rel_err(plan.double().cpu().numpy(), ref.plan) <= FP32_TOL
    assert uot.uot_read_result(ws, n, m).iters_done == p.iters


def test_same_as_passes_schedule(uot):
    """Both schedules round every entry the same way; the row and column
    sums are added in different orders (one warp per row here, the whole CTA
    per row in the fused pass), which moves the factors by a few units of
    2^-24 per iteration.  They agree within half the oracle tolerance after
    50 iterations (each is within it of the oracle on its own)."""
    p = workloads.uniform2d(seed=45, n=1024, m=1024, reg=0.05, reg_m=1.0, iters=50)
    x, _, _, _ = solve(uot, p, schedule=PERSISTENT)
    y, _, _, _ = solve(uot, p, schedule=PASSES)
    assert rel_err(x, y) <= FP32_TOL / 2
