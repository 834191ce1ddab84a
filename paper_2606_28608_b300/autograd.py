"""Differentiable periodic potential (torch.autograd).

The lattice sum at the sources is linear in the charges, Phi = A q, and A is symmetric:
A_ij = G_p(y_i - y_j) (i != j) plus the regular self part and the zero-mean constant on the
diagonal, all even in the separation.  For a loss L(Phi) with upstream gradient g = dL/dPhi:

    dL/dq = A g                              (one evaluation with charges g)
    dL/dy = g * grad Phi[q] + q * grad Phi[g]   (the evaluation's own gradient output)

so the backward pass is the library's adjoint entry point (pdmk_eval_adjoint), which runs
the same CUDA evaluation with charges q and with charges g and combines them on the device.
Gradients that flow into the returned field (a loss on forces) would need second derivatives
of the kernel; they are rejected.
"""
from __future__ import annotations

import torch

from . import Plan


class _PeriodicPotential(torch.autograd.Function):
    @staticmethod
    def forward(ctx, y, q, plan_args):
        L, eps, precision, kw = plan_args
        plan = Plan(L, eps, precision=precision, **kw)
        plan.set_sources(y.detach(), q.detach())
        n, d = y.shape
        pot = torch.empty(n, dtype=torch.float64, device=y.device)
        grad = torch.empty((n, d), dtype=torch.float64, device=y.device)
        plan.eval_device(pot, grad)
        ctx.plan = plan
        ctx.mark_non_differentiable(grad)
        return pot, grad

    @staticmethod
    def backward(ctx, g_pot, g_grad):
        if g_grad is not None and bool(torch.any(g_grad != 0)):
            raise RuntimeError("gradients through the returned field need second derivatives "
                               "of the periodic kernel, which this library does not provide")
        plan = ctx.plan
        # pdmk_eval_adjoint: dq = A g and dy = g grad Phi[q] + q grad Phi[g], on the device
        dq, dy = plan.eval_adjoint(g_pot.contiguous().to(torch.float64),
                                   want_q=ctx.needs_input_grad[1], want_y=ctx.needs_input_grad[0])
        plan.close()
        ctx.plan = None
        return dy, dq, None


def periodic_potential(L, y, q, eps: float = 1e-6, precision: str = "fp64", **kw):
    """Periodic potential and its gradient at the sources y (n x d, CUDA, float64) for charges
    q (n,), differentiable in y and q through the potential output."""
    return _PeriodicPotential.apply(y, q, (L, eps, precision, kw))
