"""Differentiable transport cost: L = <P_T, C> of the unrolled Sinkhorn-UOT
iteration, with the hand-written adjoint of libuot as its backward.

The forward keeps K = exp(-C/reg) read-only (kernel form) and records only the
per-iteration scalings and sums; the backward recomputes plan tiles from K
and that history (uot_sinkhorn_backward).  Gradients flow to C, a and b.
"""

from __future__ import annotations

import torch

from . import uot


class UOTSinkhorn(torch.autograd.Function):
    @staticmethod
    def forward(ctx, C, a, b, reg: float, reg_m: float, iters: int):
        n, m = C.shape
        ld = (m + 3) // 4 * 4  # rows 16-byte aligned for the bulk copies
        Kst = torch.empty((n, ld), dtype=torch.float32, device=C.device)
        K = Kst[:, :m]
        Cc = C.detach().contiguous()
        uot.uot_init_kernel(Cc, K, reg)
        ac, bc = a.detach().contiguous(), b.detach().contiguous()
        U, V, hist = uot.uot_sinkhorn_kform_save(K, ac, bc, reg, reg_m, iters)
        cost = uot.uot_kform_cost(K, U, V, Cc)
        ctx.save_for_backward(Cc, ac, bc, K, hist)
        ctx.params = (reg, reg_m, iters)
        return cost.reshape(())

    @staticmethod
    def backward(ctx, grad_out):
        C, a, b, K, hist = ctx.saved_tensors
        reg, reg_m, iters = ctx.params
        # The incoming gradient stays on the device (no host synchronisation,
        # so the backward can sit inside a captured step).
        g = grad_out.detach().to(torch.float64).reshape(1).contiguous()
        dC, da, db = uot.uot_sinkhorn_backward(K, C, a, b, reg, reg_m, iters, hist, 1.0,
                                               grad_out_dev=g)
        return dC.to(C.dtype), da, db, None, None, None


def sinkhorn_cost(C, a, b, reg: float, reg_m: float, iters: int):
    """<P_T, C> (FP64 scalar tensor) with gradients for C, a and b."""
    return UOTSinkhorn.apply(C, a, b, reg, reg_m, iters)
