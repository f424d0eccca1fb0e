"""Adjoint of the unrolled iteration (uot_sinkhorn_backward via the
autograd.Function) against FP64 finite differences, torch CPU FP64 autograd of
the plain unrolled loop, and the oracle's adjoint.

Inputs follow the differentiation workload: C = squared distances of 16-D
Gaussian clouds divided by max(C), a/b uniform(0.5, 1.5) normalised to 1.0 /
1.5, reg 0.05, reg_m 1.0, 200 iterations.

Tolerance, per element: each gradient entry is a sum of terms of both signs
(dC = P_T - dl / reg with dl collecting P_T C and every reverse step's
Q_t w and R_t z; da and db collect the row and column adjoints of every
step), so where they cancel the entry is far smaller than its terms and its
relative error is not bounded by the arithmetic.  FP32 rounding errors scale
with the terms' magnitudes instead, which the oracle computes by running the
same reverse recurrence on absolute values (sinkhorn_grad_magnitude).  The
GPU runs one FP32 forward (errors of the scalings about 1e-6 relative after
hundreds of iterations) and 2T reverse sweeps, each adding terms rounded to
u = 2^-24 of their size: |g - g*| <= (2T + 1) u mag per entry, 2.4e-5 mag at
T = 200 before reduction growth.  The test allows GRAD_TOL = 1e-4 of the
magnitude (floor 1e-6 of the largest), per entry.
"""

import numpy as np
import pytest

import oracle
from paper_2412_11079_gb300 import workloads

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

GRAD_TOL = 1e-4


@pytest.fixture(scope="module")
def ag():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2412_11079_gb300 import build, uot, autograd
    build.build()
    uot.load()
    return autograd


def case(n, iters=200, seed=0):
    p = workloads.gauss_normalised(seed, n, n, 16, 0.05, 1.0, iters, 1.0, 1.5, "uniform")
    return p


def gpu_grads(ag, p):
    C = torch.from_numpy(p.C).cuda().requires_grad_(True)
    a = torch.from_numpy(p.a).cuda().requires_grad_(True)
    b = torch.from_numpy(p.b).cuda().requires_grad_(True)
    L = ag.sinkhorn_cost(C, a, b, p.reg, p.reg_m, p.iters)
    L.backward()
    torch.cuda.synchronize()
    return (L.item(), C.grad.double().cpu().numpy(), a.grad.double().cpu().numpy(),
            b.grad.double().cpu().numpy())


def close(g, ref, mag, tol=GRAD_TOL):
    """Per entry: |g - ref| <= tol * max(mag, 1e-6 max(mag))."""
    err = np.max(np.abs(g - ref) / np.maximum(mag, 1e-6 * np.max(mag)))
    assert err <= tol, err


def magnitudes(p, iters=None, scale=1.0):
    m = oracle.sinkhorn_grad_magnitude(p.C, p.a, p.b, p.reg, p.reg_m,
                                       p.iters if iters is None else iters)
    return tuple(scale * x for x in m)


def test_grad_vs_finite_differences_16(ag):
    p = case(16)
    val, dC, da, db = gpu_grads(ag, p)
    C64, a64, b64 = p.C.astype(np.float64), p.a.astype(np.float64), p.b.astype(np.float64)

    def L(C_, a_, b_):
        P = oracle.sinkhorn(oracle.init_plan(C_, p.reg), a_, b_, p.reg, p.reg_m, p.iters).plan
        return oracle.transport_cost(P, C_)

    assert abs(val - L(C64, a64, b64)) <= 1e-5 * abs(L(C64, a64, b64))
    h = 1e-6
    fdC = np.zeros_like(C64)
    for i in range(16):
        for j in range(16):
            Cp, Cm = C64.copy(), C64.copy()
            Cp[i, j] += h
            Cm[i, j] -= h
            fdC[i, j] = (L(Cp, a64, b64) - L(Cm, a64, b64)) / (2 * h)
    fda = np.array([(L(C64, a64 + h * e, b64) - L(C64, a64 - h * e, b64)) / (2 * h)
                    for e in np.eye(16)])
    fdb = np.array([(L(C64, a64, b64 + h * e) - L(C64, a64, b64 - h * e)) / (2 * h)
                    for e in np.eye(16)])
    mC, ma, mb = magnitudes(p)
    close(dC, fdC, mC)
    close(da, fda, ma)
    close(db, fdb, mb)


def test_grad_vs_torch_fp64_autograd_256(ag):
    p = case(256)
    val, dC, da, db = gpu_grads(ag, p)
    fi = oracle.fi_exponent(p.reg, p.reg_m)
    Ct = torch.tensor(p.C, dtype=torch.float64, requires_grad=True)
    at = torch.tensor(p.a, dtype=torch.float64, requires_grad=True)
    bt = torch.tensor(p.b, dtype=torch.float64, requires_grad=True)
    P = torch.exp(-Ct / p.reg)
    for _ in range(p.iters):
        P = P * ((at / P.sum(1)) ** fi)[:, None]
        P = P * ((bt / P.sum(0)) ** fi)[None, :]
    loss = (P * Ct).sum()
    loss.backward()
    assert abs(val - loss.item()) <= 1e-5 * abs(loss.item())
    mC, ma, mb = magnitudes(p)
    close(dC, Ct.grad.numpy(), mC)
    close(da, at.grad.numpy(), ma)
    close(db, bt.grad.numpy(), mb)


@pytest.mark.slow
def test_grad_vs_oracle_adjoint_512(ag):
    p = case(512)
    val, dC, da, db = gpu_grads(ag, p)
    ref_val, rdC, rda, rdb = oracle.sinkhorn_grad(p.C, p.a, p.b, p.reg, p.reg_m, p.iters)
    assert abs(val - ref_val) <= 1e-5 * abs(ref_val)
    mC, ma, mb = magnitudes(p)
    close(dC, rdC, mC)
    close(da, rda, ma)
    close(db, rdb, mb)


def test_grad_full_size_few_iterations(ag):
    """N=M=2048 (the workload's size), 10 iterations, against the oracle."""
    p = case(2048, iters=10)
    val, dC, da, db = gpu_grads(ag, p)
    ref_val, rdC, rda, rdb = oracle.sinkhorn_grad(p.C, p.a, p.b, p.reg, p.reg_m, p.iters)
    assert abs(val - ref_val) <= 1e-5 * abs(ref_val)
    mC, ma, mb = magnitudes(p)
    close(dC, rdC, mC)
    close(da, rda, ma)
    close(db, rdb, mb)


@pytest.mark.slow
def test_grad_workload_configuration_200_iterations(ag):
    """One problem of the timed configuration: N=M=2048, all 200 unrolled
    iterations, forward and adjoint, against the oracle's FP64 adjoint."""
    p = case(2048, iters=200, seed=7)
    val, dC, da, db = gpu_grads(ag, p)
    ref_val, rdC, rda, rdb = oracle.sinkhorn_grad(p.C, p.a, p.b, p.reg, p.reg_m, p.iters)
    assert abs(val - ref_val) <= 1e-5 * abs(ref_val)
    mC, ma, mb = magnitudes(p)
    close(dC, rdC, mC)
    close(da, rda, ma)
    close(db, rdb, mb)


def test_grad_ragged_shape_and_grad_out(ag):
    """Rectangular, M not a multiple of 4, upstream gradient 2.5."""
    p = workloads.gauss_normalised(3, 37, 51, 16, 0.1, 0.7, 30, 1.0, 1.5, "uniform")
    C = torch.from_numpy(p.C).cuda().requires_grad_(True)
    a = torch.from_numpy(p.a).cuda().requires_grad_(True)
    b = torch.from_numpy(p.b).cuda().requires_grad_(True)
    (2.5 * ag.sinkhorn_cost(C, a, b, p.reg, p.reg_m, p.iters)).backward()
    ref_val, rdC, rda, rdb = oracle.sinkhorn_grad(p.C, p.a, p.b, p.reg, p.reg_m, p.iters)
    mC, ma, mb = magnitudes(p, scale=2.5)
    close(C.grad.double().cpu().numpy(), 2.5 * rdC, mC)
    close(a.grad.double().cpu().numpy(), 2.5 * rda, ma)
    close(b.grad.double().cpu().numpy(), 2.5 * rdb, mb)


def test_backward_takes_grad_out_on_the_device(ag):
    """The device scalar multiplies the host grad_out (0.5 * -3 here), with no
    host read of it; the result is the oracle's gradient times -1.5."""
    from paper_2412_11079_gb300 import uot
    p = workloads.gauss_normalised(4, 64, 96, 16, 0.1, 0.7, 20, 1.0, 1.5, "uniform")
    n, m = p.C.shape
    C = torch.from_numpy(p.C).cuda()
    a = torch.from_numpy(p.a).cuda()
    b = torch.from_numpy(p.b).cuda()
    K = torch.empty((n, m), device="cuda")
    uot.uot_init_kernel(C, K, p.reg)
    U, V, hist = uot.uot_sinkhorn_kform_save(K, a, b, p.reg, p.reg_m, p.iters)
    g = torch.tensor([-3.0], dtype=torch.float64, device="cuda")
    dC, da, db = uot.uot_sinkhorn_backward(K, C, a, b, p.reg, p.reg_m, p.iters, hist, 0.5,
                                           grad_out_dev=g)
    torch.cuda.synchronize()
    _, rdC, rda, rdb = oracle.sinkhorn_grad(p.C, p.a, p.b, p.reg, p.reg_m, p.iters)
    mC, ma, mb = magnitudes(p, scale=1.5)
    close(dC.double().cpu().numpy(), -1.5 * rdC, mC)
    close(da.double().cpu().numpy(), -1.5 * rda, ma)
    close(db.double().cpu().numpy(), -1.5 * rdb, mb)


def batched_case(seeds, n, m, iters, reg=0.1, reg_m=0.7):
    """Problems of one shape and parameters (a uniform batch), K with a padded
    leading dimension; the forward solves recorded per problem."""
    from paper_2412_11079_gb300 import uot
    probs = [workloads.gauss_normalised(s, n, m, 16, reg, reg_m, iters, 1.0, 1.5, "uniform")
             for s in seeds]
    B, ld = len(probs), (m + 3) // 4 * 4 + 4
    C = torch.stack([torch.from_numpy(p.C) for p in probs]).cuda()
    a = torch.stack([torch.from_numpy(p.a) for p in probs]).cuda()
    b = torch.stack([torch.from_numpy(p.b) for p in probs]).cuda()
    K = torch.empty((B, n, ld), device="cuda")[:, :, :m]
    hist = uot.grad_hist_batch(B, n, m, iters)
    for k, p in enumerate(probs):
        uot.uot_init_kernel(C[k], K[k], p.reg)
        uot.uot_sinkhorn_kform_save(K[k], a[k], b[k], p.reg, p.reg_m, iters, hist=hist[k])
    return probs, C, a, b, K, hist


def test_batched_adjoint_matches_oracle_per_problem(ag):
    """Three problems in one batched adjoint (one reverse launch per step for
    all three): M not a multiple of 4, padded K, per-problem device factors
    times the host grad_out; each problem against the oracle's gradient."""
    from paper_2412_11079_gb300 import uot
    probs, C, a, b, K, hist = batched_case([11, 12, 13], 300, 517, 25)
    g = torch.tensor([1.0, -2.0, 3.0], dtype=torch.float64, device="cuda")
    dC, da, db = uot.uot_sinkhorn_backward_batch(K, C, a, b, probs[0].reg, probs[0].reg_m, 25,
                                                 hist, 0.5, grad_out_dev=g)
    torch.cuda.synchronize()
    for k, p in enumerate(probs):
        f = 0.5 * float(g[k])
        _, rdC, rda, rdb = oracle.sinkhorn_grad(p.C, p.a, p.b, p.reg, p.reg_m, p.iters)
        mC, ma, mb = magnitudes(p, scale=abs(f))
        close(dC[k].double().cpu().numpy(), f * rdC, mC)
        close(da[k].double().cpu().numpy(), f * rda, ma)
        close(db[k].double().cpu().numpy(), f * rdb, mb)


def test_batched_adjoint_workload_geometry(ag):
    """32 problems of 2048^2, the differentiation workload's batch (19 CTAs
    per problem in a reverse launch, chunks of 64 rows and a ragged last
    block): the first and last problems against the oracle's adjoint at 6
    iterations, every problem against its own single-problem adjoint."""
    from paper_2412_11079_gb300 import uot
    iters = 6
    probs, C, a, b, K, hist = batched_case(list(range(100, 132)), 2048, 2048, iters, 0.05, 1.0)
    dC, da, db = uot.uot_sinkhorn_backward_batch(K, C, a, b, 0.05, 1.0, iters, hist)
    torch.cuda.synchronize()
    for k in (0, 31):
        p = probs[k]
        _, rdC, rda, rdb = oracle.sinkhorn_grad(p.C, p.a, p.b, p.reg, p.reg_m, p.iters)
        mC, ma, mb = magnitudes(p)
        close(dC[k].double().cpu().numpy(), rdC, mC)
        close(da[k].double().cpu().numpy(), rda, ma)
        close(db[k].double().cpu().numpy(), rdb, mb)
    for k in range(32):
        sC, sa, sb = uot.uot_sinkhorn_backward(K[k], C[k], a[k], b[k], 0.05, 1.0, iters, hist[k])
        torch.cuda.synchronize()
        # same arithmetic up to the order of the atomic column sums
        scale = float(sC.abs().max())
        assert float((dC[k] - sC).abs().max()) <= 1e-5 * scale
        assert float((da[k] - sa).abs().max()) <= 1e-5 * float(sa.abs().max())
        assert float((db[k] - sb).abs().max()) <= 1e-5 * float(sb.abs().max())
