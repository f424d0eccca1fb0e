"""FP64 CPU oracle for the MAP-UOT Sinkhorn iteration.

TEST INFRASTRUCTURE ONLY.  Nothing in the product path may import, call or
link anything under ``oracle/``; only ``tests/``, ``__graft_entry__.smoke()``
and the ``cpu_baseline`` / ``--impl reference`` legs of ``bench.py`` use it.
The oracle shares no code, header, table or helper with the CUDA library in
``paper_2412_11079_gb300/csrc``.

Modules
-------
``uot``      the literal Sinkhorn-UOT rule of Section 2.1 in FP64 (plain numpy),
             the scaling-vector (POT) form of the unbalanced iteration, the
             transport cost, the FP64 adjoint of the unrolled iterations.
``convex``   brute-force entropic-OT solves (balanced: Newton on the smooth
             dual; unbalanced: Newton on the plan entries), used only to pin
             the oracle's fixed points on tiny problems.
``sharded``  the row-partitioned form of Algorithm 1 with an explicit
             all-reduce of the column sums (Section 5.5), used by the gloo tests.
"""

from .uot import (  # noqa: F401
    STATUS_NONFINITE,
    STATUS_ZERO_SUM,
    OracleResult,
    fi_exponent,
    init_plan,
    scaling_factor,
    row_step,
    col_step,
    sinkhorn,
    sinkhorn_pot,
    transport_cost,
    sinkhorn_grad,
    sinkhorn_grad_magnitude,
    sinkhorn_tensor3,
    kernel_form_scalings,
)
