"""The rescaling factor (target/total)^fi as the library's kernels evaluate it
(FP32 division, then CUDA's fast power intrinsic), against FP64 pow.

The result is 2^e with e = fi log2(target/total).  The FP32 quotient is
rounded once (relative 2^-24, times fi in the result); the intrinsic's
logarithm and exponential each carry an error of a few units of 2^-23, and
the FP32 product fi * log2(x) is rounded relative to |e|, which enters the
result as an absolute error of the exponent (ln 2 times it, relative).  So
the test allows, per factor,
    |f - f*| / f* <= 2^-23 (4 + |e|)
over ratios in [1e-3, 1e3] and exponents fi in (0, 1] -- the range the
workloads reach (the largest |e| there is about 10).
"""

import math

import numpy as np
import pytest

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


@pytest.mark.parametrize("fi", [0.05, 0.3, 0.5, 0.8333333, 0.9090909, 0.9523810, 0.99, 1.0])
def test_factor_against_fp64_pow(uot, fi):
    rng = np.random.default_rng(int(fi * 1e6))
    count = 1 << 20
    ratio = np.exp(rng.uniform(math.log(1e-3), math.log(1e3), count))
    total = np.exp(rng.uniform(math.log(1e-9), math.log(1.0), count)).astype(np.float32)
    target = (ratio * total).astype(np.float32)
    f32 = float(np.float32(fi))
    got, st = uot.uot_selftest_factor(torch.from_numpy(target).cuda(),
                                      torch.from_numpy(total).cuda(), f32)
    got = got.double().cpu().numpy()
    x = target.astype(np.float64) / total.astype(np.float64)
    ref = x ** f32
    e = np.abs(f32 * np.log2(x))
    rel = np.abs(got - ref) / ref
    bound = 2.0 ** -23 * (4.0 + e)
    assert st == 0
    assert np.all(rel <= bound), (float(rel.max()), float((rel / bound).max()))


def test_factor_degenerate_readings(uot):
    """target 0 -> 0 (no status); total 0 < target -> 1 and ZERO_SUM; both 0
    -> 0; a non-finite total -> NONFINITE."""
    target = torch.tensor([0.0, 2.0, 0.0, 1.0], device="cuda")
    total = torch.tensor([3.0, 0.0, 0.0, math.inf], device="cuda")
    got, st = uot.uot_selftest_factor(target[:3], total[:3], 0.7)
    assert got.tolist() == [0.0, 1.0, 0.0]
    assert st == uot.UOT_DEV_ZERO_SUM
    _, st = uot.uot_selftest_factor(target[3:], total[3:], 0.7)
    assert st & uot.UOT_DEV_NONFINITE
