"""torch.autograd.Function over the CUDA rollout and its reverse sweep.

Sec. III-B: the simulator's forward pass rolls each particle's plan out and
gradients of a loss on the states are back-propagated through the whole
trajectory.  Here the forward is stamp_rollout_fwd (it keeps the checkpoint
tape) and the backward is stamp_rollout_adjoint, so a cost computed by the
library can sit inside any PyTorch graph:

    cost = rollout_cost(theta, problem, seed=s, iteration=it)   # (N,)
    (w * cost).sum().backward()                                 # theta.grad

Argument marshalling only: both passes run in libstamp.so's kernels.  The
problem keeps one tape; when another forward has run on it since this one,
the backward first replays this forward (same seed and iteration, so the same
trajectory) before the reverse sweep.
"""
from __future__ import annotations

import itertools

import torch

from . import stamp as S

_generation = itertools.count(1)


class RolloutCost(torch.autograd.Function):
    """cost_i = C(theta_i): relaxed forward rollout; gradient by the reverse sweep."""

    @staticmethod
    def forward(ctx, theta: torch.Tensor, problem: "S.Problem", seed: int, iteration: int):
        if theta.dtype != torch.float32 or not theta.is_cuda:
            raise TypeError("theta must be a float32 CUDA tensor")
        theta = theta.contiguous()
        N = theta.shape[0]
        cost = torch.empty(N, device=theta.device, dtype=torch.float32)
        problem.rollout_fwd(theta, N, seed, iteration, 0, cost)
        gen = next(_generation)
        problem._tape_owner = gen
        ctx.problem, ctx.seed, ctx.iteration, ctx.gen = problem, seed, iteration, gen
        ctx.save_for_backward(theta)
        return cost

    @staticmethod
    def backward(ctx, grad_cost: torch.Tensor):
        (theta,) = ctx.saved_tensors
        prob, N = ctx.problem, theta.shape[0]
        if getattr(prob, "_tape_owner", None) != ctx.gen:
            # the tape belongs to a later forward: replay this one
            scratch = torch.empty(N, device=theta.device, dtype=torch.float32)
            prob.rollout_fwd(theta, N, ctx.seed, ctx.iteration, 0, scratch)
            prob._tape_owner = ctx.gen
        grad_logp = torch.empty_like(theta)
        prob.rollout_adjoint(theta, N, ctx.seed, ctx.iteration, grad_logp)
        # grad_logp = -dC/dtheta per particle
        return -grad_logp * grad_cost.to(torch.float32).unsqueeze(1), None, None, None


def rollout_cost(theta: torch.Tensor, problem: "S.Problem", seed: int = 0,
                 iteration: int = -1) -> torch.Tensor:
    """Differentiable per-particle goal cost C(theta) (iteration < 0: no Gumbel noise)."""
    return RolloutCost.apply(theta, problem, seed, iteration)
