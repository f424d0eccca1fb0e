"""Row-sharded Sinkhorn over 2 CPU ranks (gloo) with an all-reduce of the
column sums (Section 5.5) must equal the unsharded oracle to FP64 rounding."""

import os
import socket

import numpy as np
import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out):
    import sys
    sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
    import oracle
    from oracle import sharded

    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        rng = np.random.default_rng(42)
        N, M = 37, 23
        C = rng.random((N, M))
        a = rng.uniform(0.5, 1.5, N)
        b = rng.uniform(0.5, 1.5, M) * 1.3
        reg, reg_m, T = 0.2, 0.7, 40
        lo, hi = sharded.row_block(N, rank, world)

        def allreduce(x):
            t = torch.from_numpy(np.ascontiguousarray(x))
            dist.all_reduce(t)
            return t.numpy()

        P0 = oracle.init_plan(C, reg)
        P_loc, _ = sharded.sinkhorn_rows(P0[lo:hi], a[lo:hi], b, reg, reg_m, T, allreduce)
        ref = oracle.sinkhorn(P0, a, b, reg, reg_m, T).plan[lo:hi]
        err = float(np.max(np.abs(P_loc - ref) / np.abs(ref)))
        out[rank] = err
    finally:
        dist.destroy_process_group()


def test_row_sharded_matches_unsharded():
    world = 2
    ctx = mp.get_context("spawn")
    with ctx.Manager() as mgr:
        out = mgr.dict()
        port = _free_port()
        procs = [ctx.Process(target=_worker, args=(r, world, port, out)) for r in range(world)]
        for p in procs:
            p.start()
        for p in procs:
            p.join(120)
            assert p.exitcode == 0
        assert len(out) == world
        for r in range(world):
            assert out[r] < 1e-12


def test_row_block_partition():
    from oracle import sharded
    for n in (1, 2, 7, 37, 100):
        for w in (1, 2, 3, 8):
            blocks = [sharded.row_block(n, r, w) for r in range(w)]
            assert blocks[0][0] == 0 and blocks[-1][1] == n
            for (l0, h0), (l1, h1) in zip(blocks, blocks[1:]):
                assert h0 == l1
