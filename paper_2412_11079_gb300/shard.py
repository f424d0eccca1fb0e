"""Row-sharded solve (Section 5.5): each process holds a block of rows of the
plan, and the one exchange per iteration is an all-reduce (sum) of the
column-sum vector between the library's sharded passes.

``sinkhorn_rows(plan_rows, a_rows, b, reg, reg_m, iters, allreduce)`` runs
``iters`` iterations on the block with ``allreduce(tensor)`` reducing the
block's column sums in place across the processes (for example
``torch.distributed.all_reduce`` with NCCL on the device tensor, or a gloo
reduction of a host copy).  Every step of the iteration runs in the library's
kernels; this module only sequences the calls.
"""

from __future__ import annotations

from . import uot


def sinkhorn_rows(plan_rows, a_rows, b, reg: float, reg_m: float, iters: int, allreduce,
                  opt=None, stream=None):
    """Runs ``iters`` iterations of the Section 2.1 rule on the row block in
    place; returns the device status word of the block's passes."""
    torch = uot._torch()
    n, m = plan_rows.shape
    opt = opt or uot.options(uot.dtype_code(plan_rows.dtype))
    ws = uot.workspace(n, m, opt, plan_rows.device)
    colsum = torch.empty(m, dtype=torch.float32, device=plan_rows.device)
    beta = torch.empty(m, dtype=torch.float32, device=plan_rows.device)
    status = torch.zeros(1, dtype=torch.int32, device=plan_rows.device)
    for t in range(1, iters + 1):
        uot.uot_shard_pass(plan_rows, a_rows, reg, reg_m, t, beta if t > 1 else None, colsum,
                           ws, opt, stream)
        allreduce(colsum)
        uot.uot_shard_factors(colsum, b, reg, reg_m, beta, status, stream)
    if iters > 0:
        uot.uot_shard_finish(plan_rows, beta, stream)
    res = uot.uot_read_result(ws, n, m, opt, stream)
    return res.dev_status | int(status.item())
