"""Seeded synthetic inputs for the UOT Sinkhorn workloads.

This module only draws inputs (point clouds, cost matrices, marginals and the
regularisation parameters); it holds none of the Sinkhorn arithmetic.  Both
the CUDA path and the CPU oracle receive the same FP32 arrays from here.

Workloads (the plan is N x M; ``a`` has length N, ``b`` length M):

* ``uniform2d``   -- points uniform in [0,1]^2, ``C`` = squared Euclidean
  distances, ``a``/``b`` uniform(0.5, 1.5) normalised to masses 1.0 / 1.5.
  At N=M=1024 with reg 0.05, reg_m 1.0 and 100 iterations this is the small
  single-problem case; at N=M=32768 with reg 0.1, reg_m 1.0 and 300
  iterations it is the reduced-precision case.
* ``gauss_normalised`` -- standard-Gaussian point clouds in D dimensions,
  ``C`` = squared distances divided by max(C), ``a``/``b`` Dirichlet(1) times
  masses 1.0 / 2.0 (the N=M=16384, D=64, reg 0.1, reg_m 0.5, 500-iteration
  large case).
* ``batch_uneven`` -- 512 problems with N and M log-uniform in [64, 4096],
  2-D uniform points, reg uniform in [0.02, 0.2], reg_m log-uniform in
  [0.1, 10], marginals as in ``uniform2d``.
* ``grad_batch`` -- problems of 16-D Gaussian points, C/max(C), marginals as in
  ``uniform2d``, reg 0.05, reg_m 1.0 (the differentiation case).
* ``tensor3`` -- three-way problems: points x_i, y_j, z_k uniform in [0,1]^2,
  C_ijk = |x_i - y_j|^2 + |y_j - z_k|^2 + |x_i - z_k|^2 (the sum of pairwise
  squared distances), mode targets uniform(0.5, 1.5) normalised to masses
  1.0, 1.5 and 1.2.
"""

from __future__ import annotations

import math
from dataclasses import dataclass

import numpy as np


@dataclass
class Problem:
    C: np.ndarray  # float32, (N, M), row-major
    a: np.ndarray  # float32, (N,)
    b: np.ndarray  # float32, (M,)
    reg: float
    reg_m: float
    iters: int
    name: str = ""

    def __post_init__(self):
        # The C ABI takes reg and reg_m as FP32: hand both sides the same
        # FP32-representable values.
        self.reg = float(np.float32(self.reg))
        self.reg_m = float(np.float32(self.reg_m))

    @property
    def shape(self):
        return self.C.shape


def sqdist(x: np.ndarray, y: np.ndarray) -> np.ndarray:
    """Squared Euclidean distances in FP64, clipped at 0."""
    x = np.asarray(x, np.float64)
    y = np.asarray(y, np.float64)
    d = (x * x).sum(1)[:, None] + (y * y).sum(1)[None, :] - 2.0 * (x @ y.T)
    np.maximum(d, 0.0, out=d)
    return d


def uniform_marginal(rng, n: int, mass: float) -> np.ndarray:
    w = rng.uniform(0.5, 1.5, size=n)
    return (w * (mass / w.sum())).astype(np.float32)


def dirichlet_marginal(rng, n: int, mass: float) -> np.ndarray:
    w = rng.dirichlet(np.ones(n))
    return (w * mass).astype(np.float32)


def uniform2d(seed: int = 0, n: int = 1024, m: int = 1024, reg: float = 0.05,
              reg_m: float = 1.0, iters: int = 100) -> Problem:
    rng = np.random.default_rng(seed)
    x = rng.random((n, 2))
    y = rng.random((m, 2))
    C = sqdist(x, y).astype(np.float32)
    a = uniform_marginal(rng, n, 1.0)
    b = uniform_marginal(rng, m, 1.5)
    return Problem(C, a, b, reg, reg_m, iters, f"uniform2d_{n}x{m}")


def gauss_normalised(seed: int = 0, n: int = 16384, m: int = 16384, dim: int = 64,
                     reg: float = 0.1, reg_m: float = 0.5, iters: int = 500,
                     mass_a: float = 1.0, mass_b: float = 2.0,
                     marginals: str = "dirichlet") -> Problem:
    rng = np.random.default_rng(seed)
    x = rng.standard_normal((n, dim))
    y = rng.standard_normal((m, dim))
    d = sqdist(x, y)
    d /= d.max()
    C = d.astype(np.float32)
    del d
    if marginals == "dirichlet":
        a = dirichlet_marginal(rng, n, mass_a)
        b = dirichlet_marginal(rng, m, mass_b)
    else:
        a = uniform_marginal(rng, n, mass_a)
        b = uniform_marginal(rng, m, mass_b)
    return Problem(C, a, b, reg, reg_m, iters, f"gauss{dim}_{n}x{m}")


def large_case(seed: int = 0, n: int = 16384, m: int = 16384, iters: int = 500) -> Problem:
    """N=M=16384 FP32 (1 GiB plan), 64-D Gaussian clouds, reg 0.1, reg_m 0.5."""
    return gauss_normalised(seed, n, m, 64, 0.1, 0.5, iters)


def small_case(seed: int = 0, n: int = 1024, m: int = 1024, iters: int = 100) -> Problem:
    """N=M=1024, 2-D uniform points, reg 0.05, reg_m 1.0, 100 iterations."""
    return uniform2d(seed, n, m, 0.05, 1.0, iters)


def uniform2d_device(seed: int, n: int, m: int, device, reg: float = 0.1, reg_m: float = 1.0,
                     iters: int = 300):
    """``uniform2d`` with the cost matrix formed on the GPU (torch, FP64 then
    FP32) for sizes where the host round trip dominates; same seeded points
    and marginals, C equal to the host version up to the last FP32 bit."""
    import torch
    rng = np.random.default_rng(seed)
    x = torch.from_numpy(rng.random((n, 2))).to(device)
    y = torch.from_numpy(rng.random((m, 2))).to(device)
    a = uniform_marginal(rng, n, 1.0)
    b = uniform_marginal(rng, m, 1.5)
    C = torch.cdist(x, y).square_().to(torch.float32)
    return C, torch.from_numpy(a).to(device), torch.from_numpy(b).to(device), \
        float(np.float32(reg)), float(np.float32(reg_m)), iters


def precision_case(seed: int = 0, n: int = 32768, m: int = 32768, iters: int = 300) -> Problem:
    """2-D uniform points, reg 0.1, reg_m 1.0, 300 iterations (N=M=32768 for
    timing; the accuracy check uses N=M=8192 of the same generator)."""
    return uniform2d(seed, n, m, 0.1, 1.0, iters)


def batch_uneven(seed: int = 0, count: int = 512, lo: int = 64, hi: int = 4096,
                 iters: int = 200) -> list:
    rng = np.random.default_rng(seed)
    out = []
    for k in range(count):
        n = int(round(math.exp(rng.uniform(math.log(lo), math.log(hi)))))
        m = int(round(math.exp(rng.uniform(math.log(lo), math.log(hi)))))
        reg = float(rng.uniform(0.02, 0.2))
        reg_m = float(math.exp(rng.uniform(math.log(0.1), math.log(10.0))))
        sub = int(rng.integers(0, 2**31 - 1))
        out.append(uniform2d(sub, n, m, reg, reg_m, iters))
        out[-1].name = f"batch{k}_{n}x{m}"
    return out


def grad_batch(seed: int = 0, count: int = 32, n: int = 2048, m: int = 2048,
               iters: int = 200) -> list:
    rng = np.random.default_rng(seed)
    out = []
    for k in range(count):
        sub = int(rng.integers(0, 2**31 - 1))
        p = gauss_normalised(sub, n, m, 16, 0.05, 1.0, iters, 1.0, 1.5, "uniform")
        p.name = f"grad{k}_{n}x{m}"
        out.append(p)
    return out


@dataclass
class Problem3:
    C: np.ndarray  # float32, (n1, n2, n3)
    a: np.ndarray
    b: np.ndarray
    c: np.ndarray
    reg: float
    reg_m: float
    iters: int

    def __post_init__(self):
        self.reg = float(np.float32(self.reg))
        self.reg_m = float(np.float32(self.reg_m))


def tensor3(seed: int = 0, n1: int = 64, n2: int = 48, n3: int = 40, reg: float = 0.1,
            reg_m: float = 1.0, iters: int = 20) -> Problem3:
    rng = np.random.default_rng(seed)
    x, y, z = rng.random((n1, 2)), rng.random((n2, 2)), rng.random((n3, 2))
    C = (sqdist(x, y)[:, :, None] + sqdist(y, z)[None, :, :] +
         sqdist(x, z)[:, None, :]).astype(np.float32)
    return Problem3(C, uniform_marginal(rng, n1, 1.0), uniform_marginal(rng, n2, 1.5),
                    uniform_marginal(rng, n3, 1.2), reg, reg_m, iters)


def tensor3_device(seed: int, n1: int, n2: int, n3: int, device, reg: float = 0.1,
                   reg_m: float = 1.0):
    """``tensor3`` with the cost tensor formed on the GPU (torch, FP64 then
    FP32) for sizes where the host round trip dominates; same seeded points
    and targets."""
    import torch
    rng = np.random.default_rng(seed)
    x, y, z = rng.random((n1, 2)), rng.random((n2, 2)), rng.random((n3, 2))
    a = uniform_marginal(rng, n1, 1.0)
    b = uniform_marginal(rng, n2, 1.5)
    c = uniform_marginal(rng, n3, 1.2)
    tx, ty, tz = (torch.from_numpy(v).to(device) for v in (x, y, z))
    C = (torch.cdist(tx, ty).square_()[:, :, None] + torch.cdist(ty, tz).square_()[None] +
         torch.cdist(tx, tz).square_()[:, None, :]).to(torch.float32)
    return (C, *(torch.from_numpy(v).to(device) for v in (a, b, c)),
            float(np.float32(reg)), float(np.float32(reg_m)))
