"""torch.autograd wrapper of the film-solve gradient (argument marshalling only: the forward
solve, the loss and the reverse sweep run in the C library, `mf_film_solve_gradient`)."""
from __future__ import annotations

import torch

from . import native


class FilmSolveLoss(torch.autograd.Function):
    """loss = 1/2 dx dy sum (h_z(T) - target)^2 of a frozen-step film solve (cold-started outside
    iterations of a fixed count) as a function of the per-cell jc map and the h_e knot values.

    apply(jc, knots, problem, g0, target, steps, iters): jc a device float64 tensor of the grid
    (the problem must have been created with a jc map), knots the knot values (float64), steps
    [(t, h), ...].  The forward sets both into the problem and computes the loss and its
    gradient in one call; the backward scales the stored gradient."""

    @staticmethod
    def forward(ctx, jc, knots, problem, g0, target, steps, iters):
        dev = getattr(problem, "device", jc.device)
        problem.mf_set_jc_map(jc.detach().to(device=dev, dtype=torch.float64).contiguous())
        problem.mf_set_knot_values(knots.detach().cpu().tolist())
        loss, jcbar, kbar = problem.mf_film_solve_gradient(g0, target, steps, iters, knots.numel())
        ctx.save_for_backward(jcbar.view_as(jc), torch.tensor(kbar, dtype=knots.dtype,
                                                              device=knots.device))
        return torch.tensor(loss, dtype=torch.float64, device=jc.device)

    @staticmethod
    def backward(ctx, grad):
        jcbar, kbar = ctx.saved_tensors
        return grad * jcbar, grad.to(kbar.device) * kbar, None, None, None, None, None


def film_solve_loss(jc, knots, problem: native.Problem, g0, target, steps, iters: int):
    return FilmSolveLoss.apply(jc, knots, problem, g0, target, steps, iters)
