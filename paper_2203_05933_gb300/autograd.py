"""Differentiable volume potential: a torch.autograd.Function over libvp.

Forward is vp_eval (smooth-rule FMM + correction apply). Backward is
vp_eval_adjoint: the transposed FMM (charges g at the targets) plus the
transposed correction for dL/df, and the differentiated local expansions,
multipole evaluations and direct sums for dL/dt (target positions), with the
correction matrix held fixed (its weights are set-up data). Expansions are
recomputed in backward from the saved densities rather than stored per
right-hand side. Every step runs in libvp's CUDA kernels.

The plan fixes the geometry; `targets` is passed only so that autograd can
attach a gradient to the positions the plan was built on (it must hold those
positions; the values are not read).
"""

from __future__ import annotations

import torch

from . import vp


class VolumePotentialFunction(torch.autograd.Function):
    @staticmethod
    def forward(ctx, f: torch.Tensor, targets: torch.Tensor, plan: vp.Plan):
        squeeze = f.dim() == 1
        f2 = (f.reshape(1, -1) if squeeze else f).contiguous()
        out = plan.eval(f2)
        ctx.plan = plan
        ctx.squeeze = squeeze
        ctx.save_for_backward(f2)
        return out[0] if squeeze else out

    @staticmethod
    def backward(ctx, grad_out: torch.Tensor):
        (f2,) = ctx.saved_tensors
        need_f = ctx.needs_input_grad[0]
        need_t = ctx.needs_input_grad[1]
        g = (grad_out.reshape(1, -1) if ctx.squeeze else grad_out).contiguous()
        gf = gt = None
        if need_f or need_t:
            gf, gt = ctx.plan.adjoint(g, grad_f=need_f, f=f2 if need_t else None, grad_tgt=need_t)
        if gf is not None and ctx.squeeze:
            gf = gf[0]
        return gf, gt, None


def volume_potential(plan: vp.Plan, f: torch.Tensor, targets: torch.Tensor | None = None) -> torch.Tensor:
    """V[f] at the plan's targets; differentiable in f and, if `targets` is given
    (a tensor holding the plan's target positions), in the target positions."""
    if targets is None:
        targets = torch.zeros((plan.n_tgt, 2), dtype=torch.float64, device=f.device)
    return VolumePotentialFunction.apply(f, targets, plan)
