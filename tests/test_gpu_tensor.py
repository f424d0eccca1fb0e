"""Three-way form (uot_sinkhorn_tensor3, one sweep of the plan per
iteration) against the FP64 oracle of the same rule, element by element at
the FP32 tolerance 1e-5; 16-bit plans within the rounding-count bound of the
in-place matrix form (each entry is rounded twice per iteration and once at
the start: 1.25 (2T+1) u)."""

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
    floor = 1e-6 * np.abs(ref).max()
    return float(np.max(np.abs(got - ref) / np.maximum(np.abs(ref), floor)))


def run(uot, p, dtype=torch.float32, P0=None):
    n1, n2, n3 = p.C.shape
    C = torch.from_numpy(p.C).cuda()
    P = torch.empty((n1, n2, n3), dtype=dtype, device="cuda")
    if P0 is None:
        uot.uot_init_kernel(C.view(n1, n2 * n3), P.view(n1, n2 * n3), p.reg)
    else:
        P.copy_(torch.from_numpy(P0).to(dtype))
    res = uot.uot_sinkhorn_tensor3(P, *(torch.from_numpy(v).cuda() for v in (p.a, p.b, p.c)),
                                   p.reg, p.reg_m, p.iters,
                                   opt=uot.options(uot.dtype_code(dtype)), check_status=False)
    return P.double().cpu().numpy(), res


def oracle_of(p, P0=None):
    P0 = np.exp(-p.C.astype(np.float64) / p.reg) if P0 is None else P0
    return oracle.sinkhorn_tensor3(P0, p.a, p.b, p.c, p.reg, p.reg_m, p.iters)


@pytest.mark.parametrize("n1,n2,n3", [(1, 1, 1), (5, 4, 6), (1, 30, 40), (64, 32, 48),
                                      (300, 40, 50), (100, 128, 160), (3, 2, 9001)])
def test_tensor3_matches_oracle(uot, n1, n2, n3):
    """Ragged shapes; 160 x 128 = 20480 unfolded columns split over a
    cluster; a 9001-wide last mode."""
    p = workloads.tensor3(seed=n1 * 7 + n2 * 3 + n3, n1=n1, n2=n2, n3=n3, reg=0.2, reg_m=0.8,
                          iters=15)
    got, res = run(uot, p)
    assert res.dev_status == 0 and res.iters_done == p.iters
    assert rel_err(got, oracle_of(p)) <= FP32_TOL


def test_tensor3_balanced_marginals(uot):
    """fi = 1: after the last (mode-3) step the mode-3 sums equal c."""
    p = workloads.tensor3(seed=3, n1=80, n2=60, n3=70, reg=0.3, reg_m=math.inf, iters=20)
    got, res = run(uot, p)
    assert rel_err(got, oracle_of(p)) <= FP32_TOL
    np.testing.assert_allclose(got.sum(axis=(0, 1)), p.c, rtol=2e-5)


def test_tensor3_degenerate_targets(uot):
    p = workloads.tensor3(seed=4, n1=20, n2=15, n3=12, reg=0.2, reg_m=1.0, iters=5)
    p.a[2] = 0.0
    p.c[5] = 0.0
    got, res = run(uot, p)
    ref = oracle_of(p)
    assert np.all(got[2] == 0) and np.all(got[:, :, 5] == 0)
    assert rel_err(got, ref) <= FP32_TOL


@pytest.mark.parametrize("dtype,u", [(torch.bfloat16, 2.0 ** -8), (torch.float16, 2.0 ** -11)])
def test_tensor3_16bit_rounding_bound(uot, dtype, u):
    p = workloads.tensor3(seed=5, n1=40, n2=30, n3=20, reg=0.5, reg_m=1.0, iters=4)
    scale = np.float32(40 * 30 * 20)  # entries O(1), in FP16's normal range
    p.a, p.b, p.c = (v * scale for v in (p.a, p.b, p.c))
    got, res = run(uot, p, dtype=dtype)
    bound = 1.25 * (2 * p.iters + 1) * u + 1e-5
    assert rel_err(got, oracle_of(p)) <= bound
