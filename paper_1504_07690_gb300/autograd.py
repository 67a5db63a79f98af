"""torch.autograd.Function over the KPM line of a stencil operator.

KPMDensity.apply(diag, plan, W, t, sigma) returns the DGC/KPM estimate
phi(t_i) = sum_{l<=M} mu_l(t_i) Tr X_l / n_tot (Alg. 2) at the points t for the
operator whose diagonal is `diag` (a potential being optimised; the couplings
and the interval (a, b) are the plan's).  The forward pass runs the moment
recurrence in libssm.so; the backward pass runs its hand-written adjoint
(ssm_kpm_adjoint, then ssm_moments_adjoint, which recomputes the recurrence
from checkpoints).  A loss built from phi at any points, including
Tr f(A) = sum_i w_i phi(x_i) with (x, w) from ssm_trace_weights, is
differentiable in `diag`.  This module only marshals arguments.

The plan must be created with the adjoint option (options=2) and holds the
checkpoints of the last forward pass only: run each backward before the
next forward on the same plan (a mismatch raises).
"""
from __future__ import annotations

import torch

from . import api


class KPMDensity(torch.autograd.Function):
    @staticmethod
    def forward(ctx, diag, plan, W, t, sigma):
        api.ssm_plan_set_diag(plan, diag)
        api.ssm_moments(plan, W)
        plan._generation = getattr(plan, "_generation", 0) + 1
        _, kpm, _ = api.ssm_dos(plan, t, sigma, want_ss=False, want_kpm=True, want_rank=False)
        ctx.plan = plan
        ctx.sigma = float(sigma)
        ctx.generation = plan._generation
        ctx.save_for_backward(t)
        return kpm

    @staticmethod
    def backward(ctx, grad):
        (t,) = ctx.saved_tensors
        plan = ctx.plan
        if getattr(plan, "_generation", 0) != ctx.generation:
            raise RuntimeError("KPMDensity: the plan ran another forward pass before this backward pass")
        g = api.ssm_kpm_adjoint(plan, t, ctx.sigma, grad.contiguous())
        dd, _ = api.ssm_moments_adjoint(plan, g)
        return dd, None, None, None, None
