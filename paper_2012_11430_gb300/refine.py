"""Least-squares refinement of Prony estimates (t_j, c_j) on the GPU.

`ExpSumFn` is a torch.autograd.Function over the library's exponential-sum kernels
(Eq. 1 of Section 1): forward f(k) = sum_j c_j exp(-2 pi i <t_j, k>) on an integer box,
backward the vector-Jacobian product for t (float64) and c (complex64).  Nothing is saved
for backward except the inputs: the exponentials are recomputed by the backward kernel.

`refine_adam` runs a torch optimizer on L = sum_k |f(k) - y_k|^2 through ExpSumFn;
`refine_lm` calls the library's on-device Levenberg-Marquardt steps (one CUDA graph).
Both are argument marshalling around libprony.so; there is no CPU fallback.
"""
from __future__ import annotations

import numpy as np
import torch

from .binding import Context


class ExpSumFn(torch.autograd.Function):
    """f = ExpSumFn.apply(t, c, ctx, lo, length): t (m, d) float64 CUDA, c (m,) complex64 CUDA,
    lo/length the box {lo_l .. lo_l + length_l - 1}; f is complex64, row-major over the box."""

    @staticmethod
    def forward(fctx, t, c, lib: Context, lo, length):
        t = t.detach().contiguous()
        c = c.detach().contiguous()
        f = torch.empty(int(np.prod(length)), dtype=torch.complex64, device=t.device)
        lib.expsum_fwd_dev(t, c, lo, length, f, torch.cuda.current_stream(t.device).cuda_stream)
        fctx.save_for_backward(t, c)
        fctx.lib, fctx.lo, fctx.length = lib, lo, length
        return f

    @staticmethod
    def backward(fctx, g):
        t, c = fctx.saved_tensors
        g = g.contiguous().to(torch.complex64)
        gt = torch.empty_like(t)
        gc = torch.empty_like(c)
        fctx.lib.expsum_bwd_dev(t, c, fctx.lo, fctx.length, g, gt, gc,
                                torch.cuda.current_stream(t.device).cuda_stream)
        return gt, gc, None, None, None


def expsum(t, c, lib: Context, lo, length):
    return ExpSumFn.apply(t, c, lib, lo, length)


def loss_fn(t, c, y, lib: Context, lo, length):
    r = expsum(t, c, lib, lo, length) - y
    return (r.real.square() + r.imag.square()).sum()


def refine_adam(t0, c0, y, lib: Context, lo, length, steps: int = 50, lr_t: float = 1e-5, lr_c: float = 1e-2):
    """Adam on L(t, c).  Returns (t, c, losses) with the loss before each step and after the last."""
    t = t0.detach().clone().requires_grad_(True)
    c = c0.detach().to(torch.complex64).clone().requires_grad_(True)
    opt = torch.optim.Adam([{"params": [t], "lr": lr_t}, {"params": [c], "lr": lr_c}])
    losses = []
    for _ in range(steps):
        opt.zero_grad(set_to_none=True)
        L = loss_fn(t, c, y, lib, lo, length)
        losses.append(L.detach())
        L.backward()
        opt.step()
    with torch.no_grad():
        losses.append(loss_fn(t, c, y, lib, lo, length))
    return t.detach(), c.detach(), torch.stack(losses)


def refine_lm(t0, c0, y, lib: Context, lo, length, steps: int = 50, lambda0: float = 1e-3):
    """Damped Gauss-Newton on L(t, c), every step on the device.  Returns (t, c, losses)."""
    t = t0.detach().to(torch.float64).clone().contiguous()
    c = c0.detach().to(torch.complex128).clone().contiguous()
    losses = torch.empty(steps + 1, dtype=torch.float64, device=t.device)
    lib.refine_lm_dev(t, c, lo, length, y.contiguous().to(torch.complex64), steps, lambda0, losses,
                      torch.cuda.current_stream(t.device).cuda_stream)
    return t, c, losses
