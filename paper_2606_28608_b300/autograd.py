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

Plans are reused: a plan (its FP64 tables, Fourier grid and transform plans, device buffers)
depends only on the lattice, eps and options, so calls with new positions take a free plan
of the same parameters from a pool and only rebuild its tree (pdmk_set_sources).  A plan
stays with its forward call until the backward pass has used it (or, without a graph, until
the evaluation is enqueued), then returns to the pool.
"""
from __future__ import annotations

import threading

import numpy as np
import torch

from . import Plan


class _PlanPool:
    """Free plans per (lattice, eps, precision, options, device)."""

    def __init__(self):
        self._free = {}
        self._lock = threading.Lock()

    @staticmethod
    def key(L, eps, precision, kw, device):
        L = np.ascontiguousarray(np.asarray(L, dtype=np.float64))
        return (L.shape[0], L.tobytes(), float(eps), precision, tuple(sorted(kw.items())), str(device))

    def take(self, key, L, eps, precision, kw):
        with self._lock:
            lst = self._free.get(key)
            if lst:
                return lst.pop()
        return Plan(L, eps, precision=precision, **kw)

    def give(self, key, plan):
        with self._lock:
            self._free.setdefault(key, []).append(plan)

    def size(self):
        with self._lock:
            return sum(len(v) for v in self._free.values())


POOL = _PlanPool()


class _PeriodicPotential(torch.autograd.Function):
    @staticmethod
    def forward(ctx, y, q, plan_args):
        L, eps, precision, kw = plan_args
        key = POOL.key(L, eps, precision, kw, y.device)
        plan = POOL.take(key, L, eps, precision, kw)
        plan.set_sources(y.detach(), q.detach())
        n, d = y.shape
        pot = torch.empty(n, dtype=torch.float64, device=y.device)
        grad = torch.empty((n, d), dtype=torch.float64, device=y.device)
        plan.eval_device(pot, grad)
        ctx.mark_non_differentiable(grad)
        if any(ctx.needs_input_grad[:2]):  # a backward pass may come (grad mode and inputs)
            ctx.plan, ctx.key = plan, key
        else:
            POOL.give(key, plan)  # no backward will come: the plan is free again
            ctx.plan = None
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
        POOL.give(ctx.key, plan)
        ctx.plan = None
        return dy, dq, None


def periodic_potential(L, y, q, eps: float = 1e-6, precision: str = "fp64", **kw):
    """Periodic potential and its gradient at the sources y (n x d, CUDA, float64) for charges
    q (n,), differentiable in y and q through the potential output."""
    return _PeriodicPotential.apply(y, q, (L, eps, precision, kw))


class PeriodicPotential(torch.nn.Module):
    """The lattice sum as a module for repeated calls (e.g. a molecular-dynamics loop): fixed
    lattice, eps and options; positions and charges per call."""

    def __init__(self, L, eps: float = 1e-6, precision: str = "mixed", **kw):
        super().__init__()
        self.L = np.ascontiguousarray(np.asarray(L, dtype=np.float64))
        self.eps, self.precision, self.kw = float(eps), precision, dict(kw)

    def forward(self, y, q):
        return periodic_potential(self.L, y, q, eps=self.eps, precision=self.precision, **self.kw)
