"""Row-partitioned Sinkhorn-UOT with an all-reduce of the column sums.

TEST INFRASTRUCTURE ONLY.  Algorithm 1 gives each of T workers a contiguous
block of rows and a private column-sum array that is summed at the end of the
iteration; Section 5.5 replaces that final sum with ``MPI_Allreduce``.  This is
the same partition in FP64 with the all-reduce passed in as a callable, so a
world of CPU ranks (``torch.distributed`` with gloo) can run it.  Row sums and
row factors are local to a rank; the only exchange per iteration is the
all-reduce of the M-long column-sum vector.
"""

from __future__ import annotations

import numpy as np

from .uot import fi_exponent, scaling_factor


def row_block(n: int, rank: int, world: int):
    """Contiguous block of rows owned by ``rank`` (the first ``n % world`` ranks
    take one extra row)."""
    base, extra = divmod(n, world)
    lo = rank * base + min(rank, extra)
    hi = lo + base + (1 if rank < extra else 0)
    return lo, hi


def sinkhorn_rows(P_local, a_local, b, reg: float, reg_m: float, iters: int, allreduce):
    """Literal row-then-column rule on a block of rows; ``allreduce(x)`` must
    return the element-wise sum of ``x`` over all ranks."""
    fi = fi_exponent(reg, reg_m)
    P = np.array(P_local, dtype=np.float64, copy=True)
    a_local = np.asarray(a_local, np.float64)
    b = np.asarray(b, np.float64)
    status = 0
    for _ in range(iters):
        r = P.sum(axis=1)
        alpha, s1 = scaling_factor(a_local, r, fi)
        P *= alpha[:, None]
        c = allreduce(P.sum(axis=0))
        beta, s2 = scaling_factor(b, c, fi)
        P *= beta[None, :]
        status |= s1 | s2
    return P, status
