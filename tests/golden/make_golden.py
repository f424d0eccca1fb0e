"""Writes the stored expected values under tests/golden/.

It calls only ``oracle/`` (here the brute-force convex solve, which is not a
Sinkhorn iteration).  Re-run with ``python tests/golden/make_golden.py``.

fixed_point_6x4.json: the limit of the row-then-column rule of Section 2.1 is
the balanced entropic-OT plan between the rescaled marginals
a k^(-1/fi) and b k^(1/fi - 1), k = (m_a/m_b)^(fi/(2-fi)); the plan stored here
is that convex problem solved by Newton's method on its dual.
"""

import json
import os
import sys

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

from oracle import convex  # noqa: E402


def fixed_point_6x4():
    rng = np.random.default_rng(20241211)
    C = np.round(rng.random((6, 4)), 6)
    a = np.round(rng.uniform(0.5, 1.5, 6), 6)
    b = np.round(rng.uniform(0.5, 1.5, 4), 6)
    reg, reg_m = 0.4, 0.9
    fi = reg_m / (reg_m + reg)
    p, q, k = convex.fixed_point_marginals(a, b, fi)
    plan = convex.entropic_ot_newton(C, p, q, reg)
    return {
        "what": "limit of the literal Sinkhorn-UOT rule (Section 2.1) = balanced "
                "entropic OT between rescaled marginals, solved on the dual",
        "C": C.tolist(), "a": a.tolist(), "b": b.tolist(),
        "reg": reg, "reg_m": reg_m, "k": k, "plan": plan.tolist(),
    }


if __name__ == "__main__":
    with open(os.path.join(HERE, "fixed_point_6x4.json"), "w") as fh:
        json.dump(fixed_point_6x4(), fh, indent=1)
    print("wrote", os.path.join(HERE, "fixed_point_6x4.json"))
