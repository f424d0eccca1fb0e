"""Failure detection without a GPU fault: the library's bounded device waits
give up, report UOT_DEV_TIMEOUT through a status word the host reads, and
leave the context usable."""

import time

import numpy as np
import pytest

import oracle
from paper_2412_11079_gb300 import workloads

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def uot():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2412_11079_gb300 import build, uot as u
    build.build()
    u.load()
    return u


def test_waits_that_nothing_completes_time_out(uot):
    counter = torch.zeros(1, dtype=torch.int32, device="cuda")  # nothing ever sets it
    status = torch.zeros(2, dtype=torch.int32, device="cuda")
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    uot.uot_selftest_wait(counter, 1, False, 0.2, status)
    torch.cuda.synchronize()
    dt = time.perf_counter() - t0
    assert status.tolist() == [uot.UOT_DEV_TIMEOUT, uot.UOT_DEV_TIMEOUT]
    assert dt >= 0.35  # both waits ran to their limit


def test_waits_that_complete_report_nothing(uot):
    counter = torch.ones(1, dtype=torch.int32, device="cuda")
    status = torch.full((2,), -1, dtype=torch.int32, device="cuda")
    uot.uot_selftest_wait(counter, 1, True, 0.2, status)
    torch.cuda.synchronize()
    assert status.tolist() == [0, 0]


def test_context_usable_after_a_timeout(uot):
    counter = torch.zeros(1, dtype=torch.int32, device="cuda")
    status = torch.zeros(2, dtype=torch.int32, device="cuda")
    uot.uot_selftest_wait(counter, 1, False, 0.1, status)
    p = workloads.uniform2d(seed=31, n=120, m=90, reg=0.1, reg_m=0.7, iters=12)
    C = torch.from_numpy(p.C).cuda()
    plan, cost, res = uot.solve(C, torch.from_numpy(p.a).cuda(), torch.from_numpy(p.b).cuda(),
                                p.reg, p.reg_m, p.iters)
    torch.cuda.synchronize()
    assert status.tolist() == [uot.UOT_DEV_TIMEOUT, uot.UOT_DEV_TIMEOUT]
    ref = oracle.sinkhorn(oracle.init_plan(p.C, p.reg), p.a, p.b, p.reg, p.reg_m, p.iters).plan
    got = plan.double().cpu().numpy()
    floor = 1e-6 * np.abs(ref).max()
    assert float(np.max(np.abs(got - ref) / np.maximum(np.abs(ref), floor))) <= 1e-5
    assert res.dev_status == 0
