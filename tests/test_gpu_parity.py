"""CUDA path (through the C ABI) vs the FP64 CPU oracle, element by element.

Tolerances: FP32 plans within 1e-5 relative per entry (entries below 1e-6 of
the largest entry are judged against that floor), cost within 1e-5 relative.
16-bit in-place plans: every iteration rounds each entry twice (after the
column factor and after the row factor) and P0 once, so an entry carries at
most (2T+1) roundings of relative size u (2^-8 BF16, 2^-11 FP16); the test
allows 1.25 (2T+1) u + 1e-5.
"""

import math

import numpy as np
import pytest

import oracle
from paper_2412_11079_gb300 import workloads

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

FP32_TOL = 1e-5


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
    ref = np.asarray(ref, np.float64)
    floor = 1e-6 * np.abs(ref).max()
    return float(np.max(np.abs(got - ref) / np.maximum(np.abs(ref), floor)))


def dev(x):
    return torch.from_numpy(np.ascontiguousarray(x)).cuda()


def run_gpu(uot, p, iters=None, dtype=torch.float32, algo=0, tile=0, cluster=0, ld=None,
            tol=0.0, check_every=1, P0=None, schedule=0):
    iters = p.iters if iters is None else iters
    n, m = p.C.shape
    C = dev(p.C)
    ld = ld or m
    store = torch.zeros((n, ld), dtype=dtype, device="cuda")
    plan = store[:, :m]
    opt = uot.options(uot.dtype_code(dtype), algo, check_every, tile, cluster, schedule=schedule)
    if P0 is None:
        uot.uot_init_kernel(C, plan, p.reg, opt)
    else:
        plan.copy_(dev(P0).to(dtype))
    res = uot.uot_sinkhorn(plan, dev(p.a), dev(p.b), p.reg, p.reg_m, iters, tol, opt=opt,
                           check_status=False)
    cost = uot.uot_cost(plan, C).item()
    torch.cuda.synchronize()
    return plan.double().cpu().numpy(), cost, res, store


def run_oracle(p, iters=None, tol=0.0, check_every=1, P0=None):
    iters = p.iters if iters is None else iters
    P0 = oracle.init_plan(p.C, p.reg) if P0 is None else P0
    res = oracle.sinkhorn(P0, p.a, p.b, p.reg, p.reg_m, iters, tol=tol, check_every=check_every)
    return res, oracle.transport_cost(res.plan, p.C)


@pytest.mark.parametrize("algo", [0, 1])
def test_small_case_matches_oracle(uot, algo):
    """N=M=1024, 2-D uniform points, reg 0.05, reg_m 1.0, 100 iterations."""
    p = workloads.small_case(seed=0)
    got, cost, res, _ = run_gpu(uot, p, algo=algo)
    ref, ref_cost = run_oracle(p)
    assert res.iters_done == 100 and res.dev_status == 0
    assert rel_err(got, ref.plan) <= FP32_TOL
    assert abs(cost - ref_cost) / abs(ref_cost) <= FP32_TOL


SHAPES = [(1, 1), (1, 7), (7, 1), (3, 5), (31, 33), (33, 31), (127, 1000), (1000, 127),
          (1000, 1025), (257, 4099), (65, 16387)]


@pytest.mark.parametrize("n,m", SHAPES)
@pytest.mark.parametrize("algo,schedule", [(0, 1), (0, 0), (1, 0)],
                         ids=["fused-passes", "fused-auto", "multipass"])
def test_shapes_match_oracle(uot, n, m, algo, schedule):
    """Fused one launch per iteration, fused with the automatic schedule
    (one persistent launch wherever the plan fits in shared memory), and
    the multi-pass baseline."""
    p = workloads.uniform2d(seed=n * 7919 + m, n=n, m=m, reg=0.1, reg_m=0.7, iters=15)
    got, cost, res, _ = run_gpu(uot, p, algo=algo, schedule=schedule)
    ref, ref_cost = run_oracle(p)
    assert res.dev_status == ref.status == 0
    assert rel_err(got, ref.plan) <= FP32_TOL
    assert abs(cost - ref_cost) <= FP32_TOL * abs(ref_cost)


@pytest.mark.parametrize("ld_extra", [1, 3, 4, 64])
def test_leading_dimension(uot, ld_extra):
    """ld > m; ld*4 % 16 != 0 takes the path without bulk copies."""
    p = workloads.uniform2d(seed=5, n=300, m=777, reg=0.08, reg_m=1.5, iters=12)
    got, _, res, store = run_gpu(uot, p, ld=777 + ld_extra)
    ref, _ = run_oracle(p)
    assert rel_err(got, ref.plan) <= FP32_TOL
    assert torch.count_nonzero(store[:, 777:]).item() == 0  # padding untouched


def fused_configs(uot, dtype_code):
    total, _ = uot.uot_fused_config(-1)
    out = []
    for k in range(total):
        _, c = uot.uot_fused_config(k)
        if c["dtype"] == dtype_code:
            out.append((k, c))
    return out


@pytest.mark.parametrize("m", [1000, 2999])
def test_every_fp32_config_and_cluster(uot, m):
    """Each FP32 fused configuration at the smallest cluster size that covers
    m, and one size larger (its last CTA then owns no columns)."""
    p = workloads.uniform2d(seed=m, n=150, m=m, reg=0.1, reg_m=0.9, iters=10)
    ref, _ = run_oracle(p)
    for k, c in fused_configs(uot, uot.UOT_F32):
        cs_min = -(-m // c["cols"])
        for cs in (cs_min, cs_min + 1):
            if cs > 8:
                continue
            got, _, res, _ = run_gpu(uot, p, tile=k + 1, cluster=cs)
            assert rel_err(got, ref.plan) <= FP32_TOL, (k, c, cs)


def test_forced_cluster_too_small_is_rejected(uot):
    p = workloads.uniform2d(seed=1, n=20, m=600, iters=2)
    k = [k for k, c in fused_configs(uot, uot.UOT_F32) if c["cols"] == 256][0]
    with pytest.raises(uot.UotError):
        run_gpu(uot, p, tile=k + 1, cluster=2)


@pytest.mark.parametrize("check_every", [1, 3])
@pytest.mark.parametrize("schedule", [1, 2], ids=["passes", "persistent"])
def test_stopping_rule(uot, check_every, schedule):
    p = workloads.uniform2d(seed=9, n=200, m=150, reg=0.3, reg_m=1.0, iters=3000)
    tol = 1e-6
    ref, _ = run_oracle(p, tol=tol, check_every=check_every)
    got, _, res, _ = run_gpu(uot, p, tol=tol, check_every=check_every, schedule=schedule)
    assert 2 <= ref.iters_done < 3000
    # FP32 row sums can move the stop by an iteration or two.
    assert abs(res.iters_done - ref.iters_done) <= 2 * check_every
    assert res.iters_done % check_every == 0
    ref2, _ = run_oracle(p, iters=res.iters_done)
    assert rel_err(got, ref2.plan) <= FP32_TOL
    assert res.err <= tol


def test_resume_equals_single_call(uot):
    p = workloads.uniform2d(seed=11, n=400, m=300, reg=0.1, reg_m=0.5, iters=40)
    once, _, _, _ = run_gpu(uot, p)
    half, _, _, _ = run_gpu(uot, p, iters=17)
    twice, _, _, _ = run_gpu(uot, p, iters=23, P0=half)
    assert rel_err(twice, once) <= FP32_TOL


def test_balanced_limit(uot):
    """reg_m = inf (fi = 1): column sums equal b after every iteration."""
    p = workloads.uniform2d(seed=12, n=500, m=260, reg=0.2, reg_m=math.inf, iters=25)
    got, _, _, _ = run_gpu(uot, p)
    ref, _ = run_oracle(p)
    assert rel_err(got, ref.plan) <= FP32_TOL
    np.testing.assert_allclose(got.sum(axis=0), p.b, rtol=1e-5)


def test_degenerate_targets_and_rows(uot):
    p = workloads.uniform2d(seed=13, n=40, m=50, reg=0.1, reg_m=1.0, iters=6)
    p.a[3] = 0.0
    p.b[7] = 0.0
    P0 = oracle.init_plan(p.C, p.reg)
    P0[10, :] = 0.0
    ref, _ = run_oracle(p, P0=P0)
    got, _, res, _ = run_gpu(uot, p, P0=P0.astype(np.float32))
    assert ref.status & oracle.STATUS_ZERO_SUM
    assert res.dev_status & uot.UOT_DEV_ZERO_SUM
    assert np.all(got[3] == 0) and np.all(got[:, 7] == 0) and np.all(got[10] == 0)
    assert rel_err(got, ref.plan) <= FP32_TOL


def test_zero_sum_reports_status(uot):
    p = workloads.uniform2d(seed=14, n=8, m=9, iters=2)
    P0 = np.zeros((8, 9), np.float32)
    n, m = P0.shape
    plan = dev(P0)
    with pytest.raises(uot.UotError) as ei:
        uot.uot_sinkhorn(plan, dev(p.a), dev(p.b), 0.1, 1.0, 2)
    assert ei.value.status == uot.UOT_ERR_ZERO_SUM


def test_init_kernel_matches_exp(uot):
    p = workloads.uniform2d(seed=15, n=333, m=517, reg=0.02)
    C = dev(p.C)
    plan = torch.empty_like(C)
    uot.uot_init_kernel(C, plan, p.reg)
    ref = np.exp(-p.C.astype(np.float64) / p.reg)
    got = plan.double().cpu().numpy()
    normal = ref > 1.2e-38
    # The exponent is carried as hi + residual, so only expf's own error and
    # the final rounding remain (a few ulp of 2^-24), even where C/reg ~ 95.
    assert np.max(np.abs(got[normal] - ref[normal]) / ref[normal]) < 6e-7
    assert np.max(np.abs(got[~normal] - ref[~normal])) < 3e-45


@pytest.mark.parametrize("dtype", ["bfloat16", "float16"])
def test_init_kernel_16bit(uot, dtype):
    p = workloads.uniform2d(seed=16, n=64, m=99, reg=0.5)
    dt = getattr(torch, dtype)
    C = dev(p.C)
    plan = torch.empty(C.shape, dtype=dt, device="cuda")
    uot.uot_init_kernel(C, plan, p.reg)
    ref = torch.exp(-C.double() / p.reg).to(dt)
    assert torch.equal(plan, ref) or (plan.double() - ref.double()).abs().max().item() <= \
        ref.double().abs().max().item() * 2 ** -8


def test_cost_kernel(uot):
    p = workloads.uniform2d(seed=17, n=700, m=911)
    rng = np.random.default_rng(0)
    P = rng.random((700, 911)).astype(np.float32)
    got = uot.uot_cost(dev(P), dev(p.C)).item()
    ref = oracle.transport_cost(P, p.C)
    assert abs(got - ref) <= 1e-12 * abs(ref)


@pytest.mark.parametrize("dtype,u", [("bfloat16", 2.0 ** -8), ("float16", 2.0 ** -11)])
@pytest.mark.parametrize("n,m", [(129, 1000), (64, 16385)])
def test_inplace_16bit_within_rounding_bound(uot, dtype, u, n, m):
    # Masses n*m and 1.5*n*m keep plan entries O(1), inside FP16's normal
    # range (entries near 1e-6 would be FP16 subnormals with a few bits).
    T = 4
    p = workloads.uniform2d(seed=18 + m, n=n, m=m, reg=0.5, reg_m=1.0, iters=T)
    p.a = (p.a * np.float32(n * m)).astype(np.float32)
    p.b = (p.b * np.float32(n * m)).astype(np.float32)
    got, cost, res, _ = run_gpu(uot, p, dtype=getattr(torch, dtype))
    ref, ref_cost = run_oracle(p)
    bound = 1.25 * (2 * T + 1) * u + 1e-5
    assert rel_err(got, ref.plan) <= bound
    assert abs(cost - ref_cost) / abs(ref_cost) <= bound


def test_graph_capture_replays_same_result(uot):
    p = workloads.uniform2d(seed=19, n=256, m=512, reg=0.1, reg_m=1.0, iters=20)
    n, m = p.C.shape
    C, a, b = dev(p.C), dev(p.a), dev(p.b)
    plan = torch.empty((n, m), device="cuda")
    ws = uot.workspace(n, m)
    s = torch.cuda.Stream()
    s.wait_stream(torch.cuda.current_stream())
    g = torch.cuda.CUDAGraph()
    with torch.cuda.stream(s):
        uot.uot_init_kernel(C, plan, p.reg, stream=s)
        uot.uot_sinkhorn(plan, a, b, p.reg, p.reg_m, p.iters, ws=ws, stream=s, sync=False)
        torch.cuda.synchronize()
        with torch.cuda.graph(g, stream=s):
            uot.uot_init_kernel(C, plan, p.reg, stream=s)
            uot.uot_sinkhorn(plan, a, b, p.reg, p.reg_m, p.iters, ws=ws, stream=s, sync=False)
    g.replay()
    torch.cuda.synchronize()
    ref, _ = run_oracle(p)
    assert rel_err(plan.double().cpu().numpy(), ref.plan) <= FP32_TOL
    assert uot.uot_read_result(ws, n, m).iters_done == p.iters


def test_launch_count(uot):
    p = workloads.uniform2d(seed=20, n=64, m=64, iters=9)
    n, m = p.C.shape
    plan = dev(oracle.init_plan(p.C, p.reg).astype(np.float32))
    before = uot.uot_launch_count()
    uot.uot_sinkhorn(plan, dev(p.a), dev(p.b), p.reg, p.reg_m, 9,
                     opt=uot.options(schedule=uot.UOT_SCHED_PASSES))
    assert uot.uot_launch_count() - before == 9 + 2  # reset + 9 passes + finish
    before = uot.uot_launch_count()
    uot.uot_sinkhorn(plan, dev(p.a), dev(p.b), p.reg, p.reg_m, 9)
    assert uot.uot_launch_count() - before == 2  # reset + one persistent launch


@pytest.mark.slow
def test_large_case_full_size(uot):
    """N=M=16384 FP32 (1 GiB plan), 64-D Gaussian clouds, reg 0.1, reg_m 0.5,
    in the launch configuration the benchmark times: (1) three iterations from
    P0 against the oracle element by element; (2) 499 + 1 iterations equal 500
    (the state between calls is the plan alone), in deterministic mode so
    that the two solves differ only by where the 499th column factor is
    applied; (3) the 500th iteration, from the GPU's own state, against one
    oracle iteration from that state.  The full 500 iterations from P0 are
    compared with the oracle at 2048 x 16384 (test_gpu_storage_det.py)."""
    p = workloads.large_case(seed=0, n=16384, m=16384)
    n, m = p.C.shape
    C, a, b = dev(p.C), dev(p.a), dev(p.b)
    plan = torch.empty((n, m), device="cuda")
    ws = uot.workspace(n, m)
    uot.uot_init_kernel(C, plan, p.reg)
    res = uot.uot_sinkhorn(plan, a, b, p.reg, p.reg_m, 3, ws=ws)
    got3 = plan.double().cpu().numpy()
    ref3 = oracle.sinkhorn(oracle.init_plan(p.C, p.reg), p.a, p.b, p.reg, p.reg_m, 3).plan
    assert res.dev_status == 0
    assert rel_err(got3, ref3) <= FP32_TOL
    del got3, ref3

    det = uot.options(deterministic=True)
    wsd = uot.workspace(n, m, det)
    uot.uot_init_kernel(C, plan, p.reg)
    uot.uot_sinkhorn(plan, a, b, p.reg, p.reg_m, 499, ws=wsd, opt=det)
    state = plan.clone()
    uot.uot_sinkhorn(plan, a, b, p.reg, p.reg_m, 1, ws=wsd, opt=det)
    last = plan.clone()
    uot.uot_init_kernel(C, plan, p.reg)
    full = uot.uot_sinkhorn(plan, a, b, p.reg, p.reg_m, 500, ws=wsd, opt=det)
    assert full.iters_done == 500 and full.dev_status == 0
    assert torch.isfinite(plan).all().item()
    d = ((plan.double() - last.double()).abs() /
         torch.clamp(last.double().abs(), min=1e-6 * last.abs().max().item())).max().item()
    assert d <= FP32_TOL
    S = state.double().cpu().numpy()
    one = oracle.sinkhorn(S, p.a, p.b, p.reg, p.reg_m, 1).plan
    assert rel_err(last.double().cpu().numpy(), one) <= FP32_TOL
