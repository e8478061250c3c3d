"""One set of particles split over several ranks (one GPU each).

Algorithm 1's iteration rolls out every particle, back-propagates its cost
and moves it by the Stein direction of Eq. svgd, whose sum runs over all
particles j.  The rollout, its reverse sweep and particle i's update need
only particle i and the gathered particles, so a set of N particles splits
into contiguous shards, one per rank:

  1. each rank rolls out its rows (their Gumbel draws indexed by the rows'
     global particle numbers) and runs the reverse sweep: grad log rho of
     its rows;
  2. one exchange: an all-gather of theta and of grad log rho (N x D floats
     each; NCCL between GPUs, gloo on host-only runs);
  3. each rank computes the median bandwidth from all N particles (the same
     value on every rank: no further exchange), then the Stein direction
     and the Adam step of its own rows.

The shards together compute bit for bit what one process computes for all
N.  The arithmetic is the compute object's: `LibraryShard` runs it in the
CUDA library; the tests plug in the FP64 oracle to check this host logic
with CPU ranks.
"""
from __future__ import annotations

import torch


def partition(N: int, world: int, rank: int) -> tuple[int, int]:
    """Contiguous balanced shard of rank: (first row, rows); the first
    N % world ranks hold one row more."""
    base, extra = divmod(N, world)
    rows = base + (1 if rank < extra else 0)
    row0 = rank * base + min(rank, extra)
    return row0, rows


def all_gather_rows(x_rows: torch.Tensor, N: int, world: int, group=None) -> torch.Tensor:
    """All ranks' rows, in rank order, as one N x D tensor.  Shards differ by
    at most one row; each is padded to the largest for the collective."""
    if world == 1:
        return x_rows.contiguous()
    pad = -(-N // world)
    buf = torch.zeros((pad,) + tuple(x_rows.shape[1:]), dtype=x_rows.dtype, device=x_rows.device)
    buf[: x_rows.shape[0]] = x_rows
    parts = [torch.empty_like(buf) for _ in range(world)]
    torch.distributed.all_gather(parts, buf, group=group)
    return torch.cat([parts[r][: partition(N, world, r)[1]] for r in range(world)]).contiguous()


class ShardedSolver:
    """Algorithm 1's iterations over one rank's shard.

    compute: an object with
      grad(theta_rows, it) -> grad log rho of the rows (iteration it's noise)
      step_rows(theta_all, grad_all, theta_rows, m, v, step, lr, sgd_phase)
        -> updates theta_rows, m, v in place (this shard's rows).
    """

    def __init__(self, compute, N: int, world: int = 1, rank: int = 0, group=None):
        self.compute, self.N, self.world, self.rank, self.group = compute, N, world, rank, group
        self.row0, self.rows = partition(N, world, rank)

    def iteration(self, theta_rows, m, v, it: int, lr: float, sgd_phase: bool = False):
        g_rows = self.compute.grad(theta_rows, it)
        theta_all = all_gather_rows(theta_rows, self.N, self.world, self.group)
        grad_all = all_gather_rows(g_rows, self.N, self.world, self.group)
        self.compute.step_rows(theta_all, grad_all, theta_rows, m, v, it + 1, lr, sgd_phase)

    def run(self, theta_rows, m, v, svgd_iters: int, sgd_iters: int, lr: float):
        for it in range(svgd_iters + sgd_iters):
            self.iteration(theta_rows, m, v, it, lr, it >= svgd_iters)
        return theta_rows


class LibraryShard:
    """The compute of one GPU's shard: the library's rollout, reverse sweep
    and row-range Stein step on a problem sized for all N particles (the
    N x N distances of the bandwidth are computed on every rank)."""

    def __init__(self, P: dict, init, goal, N: int, row0: int, rows: int, seed: int,
                 stream: int | None = None):
        from paper_2310_01775_gb300 import stamp as S
        self.prob = S.Problem(P, init, goal, N, stream)
        self.prob.set_particle_offset(row0)
        self.N, self.row0, self.rows, self.seed = N, row0, rows, seed
        self.cost = torch.empty(rows, device="cuda")

    def grad(self, theta_rows, it):
        g = torch.empty_like(theta_rows)
        self.prob.rollout_fwd(theta_rows, self.rows, self.seed, it, 0, self.cost)
        self.prob.rollout_adjoint(theta_rows, self.rows, self.seed, it, g)
        return g

    def step_rows(self, theta_all, grad_all, theta_rows, m, v, step, lr, sgd_phase):
        self.prob.svgd_step_rows(theta_all, grad_all, self.N, self.row0, self.rows, theta_rows, m,
                                 v, step, lr, int(sgd_phase))

    def close(self):
        self.prob.close()
