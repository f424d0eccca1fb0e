"""Adjoint of the unrolled iteration (uot_sinkhorn_backward via the
autograd.Function) against FP64 finite differences, torch CPU FP64 autograd of
the plain unrolled loop, and the oracle's adjoint.

Inputs follow the differentiation workload: C = squared distances of 16-D
Gaussian clouds divided by max(C), a/b uniform(0.5, 1.5) normalised to 1.0 /
1.5, reg 0.05, reg_m 1.0, 200 iterations.  Tolerance: the GPU runs the
forward and 2T reverse sweeps in FP32, so each gradient is compared with
max|g - g*| <= 2e-4 max|g*| (the FP32 unit roundoff 6e-8 times the 2T+1 =
401 sweeps is 2.4e-5; the bound leaves room for the reductions' growth).
"""

import numpy as np
import pytest

import oracle
from paper_2412_11079_gb300 import workloads

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

GRAD_TOL = 2e-4


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


def close(g, ref, tol=GRAD_TOL):
    err = np.max(np.abs(g - ref)) / np.max(np.abs(ref))
    assert err <= tol, err


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
    close(dC, fdC)
    close(da, fda)
    close(db, fdb)


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
    close(dC, Ct.grad.numpy())
    close(da, at.grad.numpy())
    close(db, bt.grad.numpy())


@pytest.mark.slow
def test_grad_vs_oracle_adjoint_512(ag):
    p = case(512)
    val, dC, da, db = gpu_grads(ag, p)
    ref_val, rdC, rda, rdb = oracle.sinkhorn_grad(p.C, p.a, p.b, p.reg, p.reg_m, p.iters)
    assert abs(val - ref_val) <= 1e-5 * abs(ref_val)
    close(dC, rdC)
    close(da, rda)
    close(db, rdb)


def test_grad_full_size_few_iterations(ag):
    """N=M=2048 (the workload's size), 10 iterations, against the oracle."""
    p = case(2048, iters=10)
    val, dC, da, db = gpu_grads(ag, p)
    ref_val, rdC, rda, rdb = oracle.sinkhorn_grad(p.C, p.a, p.b, p.reg, p.reg_m, p.iters)
    assert abs(val - ref_val) <= 1e-5 * abs(ref_val)
    close(dC, rdC)
    close(da, rda)
    close(db, rdb)


def test_grad_ragged_shape_and_grad_out(ag):
    """Rectangular, M not a multiple of 4, upstream gradient 2.5."""
    p = workloads.gauss_normalised(3, 37, 51, 16, 0.1, 0.7, 30, 1.0, 1.5, "uniform")
    C = torch.from_numpy(p.C).cuda().requires_grad_(True)
    a = torch.from_numpy(p.a).cuda().requires_grad_(True)
    b = torch.from_numpy(p.b).cuda().requires_grad_(True)
    (2.5 * ag.sinkhorn_cost(C, a, b, p.reg, p.reg_m, p.iters)).backward()
    ref_val, rdC, rda, rdb = oracle.sinkhorn_grad(p.C, p.a, p.b, p.reg, p.reg_m, p.iters)
    close(C.grad.double().cpu().numpy(), 2.5 * rdC)
    close(a.grad.double().cpu().numpy(), 2.5 * rda)
    close(b.grad.double().cpu().numpy(), 2.5 * rdb)
