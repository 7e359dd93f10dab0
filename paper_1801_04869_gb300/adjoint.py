"""torch.autograd wrapper of the film-solve gradient (argument marshalling only: the forward
solve, the loss and the reverse sweep run in the C library, `mf_film_solve_gradient`)."""
from __future__ import annotations

import torch

from . import native


class FilmSolveLoss(torch.autograd.Function):
    """loss = 1/2 dx dy sum (h_z(T) - target)^2 of a film solve with frozen decisions (the given
    steps, all accepted, and the given outside-iteration counts, 3 per step, with the warm start
    carried from call to call) as a function of the per-cell jc map and the h_e knot values.

    apply(jc, knots, problem, g0, target, steps, iters, ckpt_every): jc a float64 tensor of the
    grid on any device (the problem must have been created with a jc map), knots the knot values
    (float64), steps [(t, h), ...], iters 3 counts per step.  The forward sets both parameters into
    the problem and computes the loss and its gradient in one call (the gradient is kept for
    backward; film_solve_loss runs the forward alone when no gradient is recorded).  The backward
    scales the kept gradient; the gradients come back on the devices of jc and knots."""

    @staticmethod
    def forward(ctx, jc, knots, problem, g0, target, steps, iters, ckpt_every):
        dev = getattr(problem, "device", jc.device)
        problem.mf_set_jc_map(jc.detach().to(device=dev, dtype=torch.float64).contiguous())
        problem.mf_set_knot_values(knots.detach().cpu().tolist())
        loss, jcbar, kbar, _ = problem.mf_film_solve_gradient(g0, target, steps, iters, ckpt_every,
                                                              grad=True)
        ctx.save_for_backward(jcbar.view_as(jc).to(jc.device),
                              torch.tensor(kbar, dtype=knots.dtype, device=knots.device))
        return torch.tensor(loss, dtype=torch.float64, device=jc.device)

    @staticmethod
    def backward(ctx, grad):
        jcbar, kbar = ctx.saved_tensors
        return (grad.to(jcbar.device) * jcbar, grad.to(kbar.device) * kbar,
                None, None, None, None, None, None)


def film_solve_loss(jc, knots, problem: native.Problem, g0, target, steps, iters,
                    ckpt_every: int = 20):
    """The loss as a differentiable function of jc and knots; without a gradient to record
    (torch.no_grad(), or neither parameter requires one) only the forward solve runs."""
    if torch.is_grad_enabled() and (jc.requires_grad or knots.requires_grad):
        return FilmSolveLoss.apply(jc, knots, problem, g0, target, steps, iters, ckpt_every)
    dev = getattr(problem, "device", jc.device)
    problem.mf_set_jc_map(jc.detach().to(device=dev, dtype=torch.float64).contiguous())
    problem.mf_set_knot_values(knots.detach().cpu().tolist())
    loss = problem.mf_film_solve_gradient(g0, target, steps, iters, ckpt_every, grad=False)[0]
    return torch.tensor(loss, dtype=torch.float64, device=jc.device)
