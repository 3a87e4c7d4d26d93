"""Differentiable advection: torch.autograd.Function over the tracker's RK2 path.

``advect(pos0, field, tracker, dt, steps)`` returns X_T after ``steps`` RK2
steps of Eq. (tracers) in ``field``.  Its backward pass is the library's
hand-written discrete adjoint (tracker_adjoint): the particle-to-grid
transpose of the interpolation for d/dfield and the kernel-derivative
Jacobian recurrence for d/dX_0, with the forward trajectory recomputed from
checkpoints every ``ckpt_every`` steps.  All arithmetic runs in the CUDA
library; this file only marshals tensors.
"""
from __future__ import annotations

import torch


class TrackerAdvect(torch.autograd.Function):
    @staticmethod
    def forward(ctx, pos0, field, tracker, dt, steps, ckpt_every):
        f = field.detach().contiguous()
        tracker.set_field(f)
        posT = pos0.detach().clone().contiguous()
        tracker.advance(posT, dt, steps)
        ctx.tracker, ctx.dt, ctx.steps, ctx.ckpt = tracker, float(dt), int(steps), int(ckpt_every)
        ctx.field_shape, ctx.field_dtype = tuple(field.shape), field.dtype
        # the field this graph was advanced in: another advect() or set_field on
        # the same tracker before backward replaces the tracker's copy
        ctx.field, ctx.field_generation = f, tracker.field_generation
        ctx.save_for_backward(pos0)
        return posT

    @staticmethod
    def backward(ctx, grad_posT):
        (pos0,) = ctx.saved_tensors
        if ctx.tracker.field_generation != ctx.field_generation:
            ctx.tracker.set_field(ctx.field)
            ctx.field_generation = ctx.tracker.field_generation
        gfield = None
        if ctx.needs_input_grad[1]:
            gfield = torch.zeros(ctx.field_shape, dtype=torch.float64, device=pos0.device)
        gpos0, _ = ctx.tracker.adjoint(pos0.detach().contiguous(), grad_posT.detach().double().contiguous(),
                                       ctx.dt, ctx.steps, ctx.ckpt, grad_field=gfield)
        gpos0 = gpos0 if ctx.needs_input_grad[0] else None
        if gfield is not None:
            gfield = gfield.to(ctx.field_dtype)
        return gpos0, gfield, None, None, None, None


def advect(pos0, field, tracker, dt, steps, ckpt_every=5):
    """X_T from X_0 (pos0[3][np], float64) through ``steps`` RK2 steps; differentiable in pos0 and field."""
    return TrackerAdvect.apply(pos0, field, tracker, dt, steps, ckpt_every)
