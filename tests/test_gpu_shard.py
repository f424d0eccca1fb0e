"""Row-sharded iteration (Section 5.5) through the C ABI: row blocks passed
separately, their column sums all-reduced between passes, against the FP64
oracle of the whole (unsharded) problem, at the FP32 tolerance 1e-5.

The two-process test runs two processes on the one GPU, each with its own
row block, reducing the column sums with a gloo all-reduce of host copies
(no kernel ever waits on another process: each process waits on its own
stream between calls).
"""

import os
import socket

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
    floor = 1e-6 * np.abs(ref).max()
    return float(np.max(np.abs(got - ref) / np.maximum(np.abs(ref), floor)))


@pytest.mark.parametrize("n,m,cuts", [(300, 517, [140]), (1000, 2048, [1, 500, 999]),
                                      (96, 16387, [48])])
def test_shards_in_one_process(uot, n, m, cuts):
    """Row blocks passed one after the other, their column sums added on the
    device between passes: the union of the blocks is the oracle's plan."""
    p = workloads.uniform2d(seed=n + m, n=n, m=m, reg=0.1, reg_m=0.7, iters=15)
    C = torch.from_numpy(p.C).cuda()
    plan = torch.empty((n, m), device="cuda")
    uot.uot_init_kernel(C, plan, p.reg)
    a = torch.from_numpy(p.a).cuda()
    b = torch.from_numpy(p.b).cuda()
    edges = [0] + cuts + [n]
    blocks = [(lo, hi) for lo, hi in zip(edges[:-1], edges[1:])]
    wss = [uot.workspace(hi - lo, m) for lo, hi in blocks]
    parts = [torch.empty(m, device="cuda") for _ in blocks]
    beta = torch.empty(m, device="cuda")
    for t in range(1, p.iters + 1):
        for (lo, hi), ws, part in zip(blocks, wss, parts):
            uot.uot_shard_pass(plan[lo:hi], a[lo:hi], p.reg, p.reg_m, t,
                               beta if t > 1 else None, part, ws)
        total = torch.stack(parts).sum(0)
        uot.uot_shard_factors(total, b, p.reg, p.reg_m, beta)
    for lo, hi in blocks:
        uot.uot_shard_finish(plan[lo:hi], beta)
    torch.cuda.synchronize()
    ref = oracle.sinkhorn(oracle.init_plan(p.C, p.reg), p.a, p.b, p.reg, p.reg_m, p.iters)
    assert rel_err(plan.double().cpu().numpy(), ref.plan) <= FP32_TOL


def test_one_shard_is_the_whole_solve(uot):
    """A single block through the driver equals uot_sinkhorn's result."""
    from paper_2412_11079_gb300 import shard
    p = workloads.uniform2d(seed=7, n=400, m=600, reg=0.1, reg_m=1.0, iters=25)
    C = torch.from_numpy(p.C).cuda()
    a = torch.from_numpy(p.a).cuda()
    b = torch.from_numpy(p.b).cuda()
    x = torch.empty((400, 600), device="cuda")
    uot.uot_init_kernel(C, x, p.reg)
    st = shard.sinkhorn_rows(x, a, b, p.reg, p.reg_m, p.iters, lambda t: None)
    torch.cuda.synchronize()
    ref = oracle.sinkhorn(oracle.init_plan(p.C, p.reg), p.a, p.b, p.reg, p.reg_m, p.iters)
    assert st == 0
    assert rel_err(x.double().cpu().numpy(), ref.plan) <= FP32_TOL


def test_shard_degenerate_status(uot):
    """A zero row with a positive target: factor 1 and ZERO_SUM reported by
    the block that holds it."""
    from paper_2412_11079_gb300 import shard
    p = workloads.uniform2d(seed=8, n=60, m=70, reg=0.1, reg_m=1.0, iters=3)
    P0 = oracle.init_plan(p.C, p.reg)
    P0[5, :] = 0.0
    x = torch.from_numpy(P0.astype(np.float32)).cuda()
    st = shard.sinkhorn_rows(x, torch.from_numpy(p.a).cuda(), torch.from_numpy(p.b).cuda(),
                             p.reg, p.reg_m, p.iters, lambda t: None)
    ref = oracle.sinkhorn(P0, p.a, p.b, p.reg, p.reg_m, p.iters)
    assert st & uot.UOT_DEV_ZERO_SUM and ref.status & oracle.STATUS_ZERO_SUM
    assert rel_err(x.double().cpu().numpy(), ref.plan) <= FP32_TOL


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out_dir):
    import torch
    import torch.distributed as dist

    import oracle as orc
    from paper_2412_11079_gb300 import shard, uot as u, workloads as wl

    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    torch.cuda.set_device(0)
    u.load()
    p = wl.uniform2d(seed=3, n=500, m=700, reg=0.08, reg_m=0.9, iters=20)
    bounds = np.linspace(0, 500, world + 1).astype(int)
    lo, hi = int(bounds[rank]), int(bounds[rank + 1])
    C = torch.from_numpy(np.ascontiguousarray(p.C[lo:hi])).cuda()
    x = torch.empty((hi - lo, 700), device="cuda")
    u.uot_init_kernel(C, x, p.reg)

    def allreduce(t):
        h = t.cpu()  # synchronises this process's stream
        dist.all_reduce(h)
        t.copy_(h)

    st = shard.sinkhorn_rows(x, torch.from_numpy(p.a[lo:hi].copy()).cuda(),
                             torch.from_numpy(p.b).cuda(), p.reg, p.reg_m, p.iters, allreduce)
    ref = orc.sinkhorn(orc.init_plan(p.C, p.reg), p.a, p.b, p.reg, p.reg_m, p.iters).plan
    got = x.double().cpu().numpy()
    floor = 1e-6 * np.abs(ref).max()
    err = float(np.max(np.abs(got - ref[lo:hi]) / np.maximum(np.abs(ref[lo:hi]), floor)))
    with open(os.path.join(out_dir, f"rank{rank}.txt"), "w") as fh:
        fh.write(f"{err} {st}\n")
    dist.barrier()
    dist.destroy_process_group()


def test_two_processes_gloo_allreduce(uot, tmp_path):
    import torch.multiprocessing as mp
    world = 2
    mp.start_processes(_rank_main, args=(world, _free_port(), str(tmp_path)), nprocs=world,
                       join=True, start_method="spawn")
    for r in range(world):
        err, st = open(tmp_path / f"rank{r}.txt").read().split()
        assert int(st) == 0
        assert float(err) <= FP32_TOL, (r, err)
