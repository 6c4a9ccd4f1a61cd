"""Differentiable DODE loss for PyTorch (argument marshalling only).

``DodeLoss.apply(q, theta, ctx)`` returns L(q, theta) = sum over the loaded days
of sum m (B_d(theta) q_d - x_d)^2 (Eq. (nnls) with the logit route choice of
Eq. (logit) at dispersion theta per minute).  The forward pass runs the fused
CUDA kernel's forward sweep only and saves nothing but its inputs; the
backward pass rebuilds the DAR on the fly and runs the forward and adjoint
sweeps again (``dode_loss_grad``), returning dL/dq = 2 B^T r and

    dL/dtheta = sum_{k,h} 2 q[h][od(k)] g_k[h] p_k[h] (sum_{k'} p_k'[h] C_k'[h] - C_k[h])

with g_k the route-level adjoint and C the route times.  All arithmetic runs in
libdode; torch only provides device memory and the stream.
"""
from __future__ import annotations

import torch

from .dode import Context


class DodeLoss(torch.autograd.Function):
    """L(q, theta) of the loaded days as a torch autograd function (see the module docstring)."""
    @staticmethod
    def forward(fctx, q: torch.Tensor, theta: torch.Tensor, ctx: Context) -> torch.Tensor:
        if not q.is_cuda:
            raise ValueError("q must be a CUDA tensor")
        qc = q.detach().to(torch.float32).contiguous()
        th = float(theta.detach().cpu().item()) if isinstance(theta, torch.Tensor) else float(theta)
        ctx.use_torch_stream()
        ctx.loss(qc, th)
        total, _ = ctx.last_totals()
        fctx.save_for_backward(qc)
        fctx.theta = th
        fctx.dctx = ctx
        fctx.theta_is_tensor = isinstance(theta, torch.Tensor)
        fctx.theta_dtype = theta.dtype if isinstance(theta, torch.Tensor) else torch.float64
        fctx.theta_device = theta.device if isinstance(theta, torch.Tensor) else torch.device("cpu")
        fctx.q_dtype = q.dtype
        return torch.tensor(total, dtype=torch.float64, device=q.device)

    @staticmethod
    def backward(fctx, grad_out: torch.Tensor):
        (qc,) = fctx.saved_tensors
        ctx: Context = fctx.dctx
        dq = torch.empty_like(qc)
        ctx.loss_grad(qc, fctx.theta, dq_out=dq)
        _, dth_total = ctx.last_totals(with_dtheta=True)
        # chain rule: the upstream gradient scales the library's dL/dq and dL/dtheta
        g = grad_out.to(torch.float64)
        grad_q = (dq.to(torch.float64) * g).to(fctx.q_dtype)
        grad_theta = None
        if fctx.theta_is_tensor:
            grad_theta = torch.tensor(float(g.item()) * dth_total, dtype=fctx.theta_dtype,
                                      device=fctx.theta_device)
        return grad_q, grad_theta, None


def dode_loss(q: torch.Tensor, theta, ctx: Context) -> torch.Tensor:
    """L(q, theta) over all loaded days, differentiable in q and theta."""
    if not isinstance(theta, torch.Tensor):
        theta = torch.tensor(float(theta), dtype=torch.float64)
    return DodeLoss.apply(q, theta, ctx)
