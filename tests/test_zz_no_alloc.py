"""uot_sinkhorn_noalloc, the entry point for callers that cannot allocate
device memory (it runs on a scratch array built into the library), against
the workspace-taking uot_sinkhorn on the same inputs and against the FP64
oracle, through the C ABI.

Two calls in a row with different shapes also check that the array's stale
contents from the first call do not leak into the second.  This file is
collected last so a failure here comes after every other test has run.
"""

import ctypes

import numpy as np
import pytest

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
    floor = 1e-6 * np.abs(ref).max()
    return float(np.max(np.abs(got - ref) / np.maximum(np.abs(ref), floor)))


def solve_both(uot, p, tol=0.0):
    n, m = p.C.shape
    C = torch.from_numpy(p.C).cuda()
    a = torch.from_numpy(p.a).cuda()
    b = torch.from_numpy(p.b).cuda()
    p0 = torch.empty((n, m), device="cuda")
    uot.uot_init_kernel(C, p0, p.reg)
    ref_plan, got_plan = p0.clone(), p0.clone()
    ref = uot.uot_sinkhorn(ref_plan, a, b, p.reg, p.reg_m, p.iters, tol)
    # Straight through the C ABI: no workspace argument.
    res = uot.UotResult()
    st = uot.load().uot_sinkhorn_noalloc(
        got_plan.data_ptr(), m, a.data_ptr(), b.data_ptr(), n, m, p.reg, p.reg_m, p.iters,
        tol, None, ctypes.c_void_p(torch.cuda.current_stream().cuda_stream), ctypes.byref(res))
    assert st == uot.UOT_OK, uot.uot_status_string(st)
    torch.cuda.synchronize()
    return ref, res, ref_plan.double().cpu().numpy(), got_plan.double().cpu().numpy()


def test_noalloc_matches_workspace_entry_point_twice(uot):
    first = workloads.uniform2d(seed=31, n=300, m=517, reg=0.07, reg_m=0.8, iters=25)
    second = workloads.uniform2d(seed=32, n=129, m=2000, reg=0.2, reg_m=2.0, iters=40)
    for p in (first, second):
        ref, res, ref_plan, got_plan = solve_both(uot, p)
        assert res.dev_status == ref.dev_status == 0
        assert res.iters_done == ref.iters_done
        assert rel_err(got_plan, ref_plan) <= FP32_TOL


def test_noalloc_matches_the_oracle(uot):
    """The no-allocation entry point against the FP64 oracle of the rule
    (Section 2.1), element by element at the FP32 tolerance: a ragged shape
    over several tiles, 30 iterations."""
    import oracle
    p = workloads.uniform2d(seed=34, n=257, m=333, reg=0.08, reg_m=0.9, iters=30)
    _, res, _, got_plan = solve_both(uot, p)
    want = oracle.sinkhorn(oracle.init_plan(p.C, p.reg), p.a, p.b, p.reg, p.reg_m, p.iters)
    assert res.dev_status == 0 and want.status == 0
    assert res.iters_done == p.iters
    assert rel_err(got_plan, want.plan) <= FP32_TOL


def test_noalloc_rejects_problems_beyond_the_static_scratch(uot):
    big = 70000
    assert uot.uot_workspace_size(big, big) > uot.UOT_STATIC_SCRATCH_BYTES
    plan = torch.empty((1, big), device="cuda")  # never touched: rejected first
    a = torch.ones(1, device="cuda")
    b = torch.ones(big, device="cuda")
    st = uot.load().uot_sinkhorn_noalloc(plan.data_ptr(), big, a.data_ptr(), b.data_ptr(),
                                         big, big, 0.1, 1.0, 1, 0.0, None, None, None)
    assert st == uot.UOT_ERR_WORKSPACE


def test_noalloc_from_a_new_host_thread(uot):
    """A host thread that has made no CUDA call has no current context; the
    first call there still finds the array's address (the runtime makes the
    device's primary context current) and matches uot_sinkhorn.  Every tensor
    is made on the main thread, so the worker's only CUDA call is the entry
    point itself (on the legacy default stream)."""
    import threading

    p = workloads.uniform2d(seed=33, n=200, m=300, reg=0.1, reg_m=1.0, iters=12)
    n, m = p.C.shape
    C = torch.from_numpy(p.C).cuda()
    a = torch.from_numpy(p.a).cuda()
    b = torch.from_numpy(p.b).cuda()
    p0 = torch.empty((n, m), device="cuda")
    uot.uot_init_kernel(C, p0, p.reg)
    ref_plan, got_plan = p0.clone(), p0.clone()
    ref = uot.uot_sinkhorn(ref_plan, a, b, p.reg, p.reg_m, p.iters)
    torch.cuda.synchronize()
    res = uot.UotResult()
    out = {}

    def worker():
        out["st"] = uot.load().uot_sinkhorn_noalloc(
            got_plan.data_ptr(), m, a.data_ptr(), b.data_ptr(), n, m, p.reg, p.reg_m, p.iters,
            0.0, None, None, ctypes.byref(res))

    t = threading.Thread(target=worker)
    t.start()
    t.join()
    torch.cuda.synchronize()
    assert out["st"] == uot.UOT_OK, uot.uot_status_string(out["st"])
    assert res.dev_status == ref.dev_status == 0 and res.iters_done == p.iters
    assert rel_err(got_plan.double().cpu().numpy(), ref_plan.double().cpu().numpy()) <= FP32_TOL
