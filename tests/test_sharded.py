"""Particle shards of one Stein iteration on CPU ranks (two and three gloo processes).

The sharded driver (paper_2310_01775_gb300/sharded.py) splits N particles
into contiguous shards, all-gathers theta and grad log rho once per
iteration, and leaves each rank the bandwidth of all N and the update of
its own rows.  Here the arithmetic is the FP64 oracle's, so the test checks
the host logic -- partition, Gumbel draws by global particle number, the
padded all-gather and its reassembly, per-rank Adam state -- against the
oracle's own unsharded Algorithm 1, bit for bit.
"""
import os
import socket
import sys

import numpy as np
import pytest
import torch
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
SVGD, SGD, LR = 3, 1, 1e-2


class OracleShard:
    """The compute of one shard with the oracle's functions (FP64, CPU)."""

    def __init__(self, P, init, goal, N, row0, rows, seed):
        self.P, self.init, self.goal = P, init, goal
        self.N, self.row0, self.rows, self.seed = N, row0, rows, seed

    def grad(self, theta_rows, it):
        from oracle import stamp_oracle as O
        M = 4 * self.P["n_blocks"]
        gum = O.gumbel_noise(self.seed, it, self.N, self.P["H"], M)[self.row0:self.row0 + self.rows]
        _, g = O.rollout_grad(theta_rows.numpy(), self.P, self.init, self.goal, gum)
        return torch.from_numpy(g)

    def step_rows(self, theta_all, grad_all, theta_rows, m, v, step, lr, sgd_phase):
        from oracle import stamp_oracle as O
        th, g = theta_all.numpy(), grad_all.numpy()
        sl = slice(self.row0, self.row0 + self.rows)
        phi = g[sl] if sgd_phase else O.stein_direction(th, g, O.median_bandwidth(th))[sl]
        t, mm, vv = O.adam_update(theta_rows.numpy(), m.numpy(), v.numpy(), -phi, step, lr)
        theta_rows.copy_(torch.from_numpy(t))
        m.copy_(torch.from_numpy(mm))
        v.copy_(torch.from_numpy(vv))


def _problem():
    from paper_2310_01775_gb300 import workloads as W
    P = W.params("pusher1_h2")
    init, goal = W.scene(P, 3)
    return P, init, goal


def _run(world, rank, N, seed, group=None):
    from oracle import stamp_oracle as O
    from paper_2310_01775_gb300 import sharded as SH
    P, init, goal = _problem()
    row0, rows = SH.partition(N, world, rank)
    D = O.dims(P)[2]
    th = torch.from_numpy(O.init_theta(seed, N, D)[row0:row0 + rows].copy())
    m, v = torch.zeros_like(th), torch.zeros_like(th)
    solver = SH.ShardedSolver(OracleShard(P, init, goal, N, row0, rows, seed), N, world, rank, group)
    solver.run(th, m, v, SVGD, SGD, LR)
    return SH.all_gather_rows(th, N, world, group).numpy()


def _rank(rank, world, port, N, seed, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    sys.path.insert(0, ROOT)
    torch.set_num_threads(1)
    torch.distributed.init_process_group("gloo", rank=rank, world_size=world)
    th = _run(world, rank, N, seed)
    out.put((rank, th))
    torch.distributed.destroy_process_group()


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def test_partition_is_contiguous_and_balanced():
    sys.path.insert(0, ROOT)
    from paper_2310_01775_gb300 import sharded as SH
    for N in (1, 2, 7, 33, 2048):
        for world in (1, 2, 3, 8):
            parts = [SH.partition(N, world, r) for r in range(world)]
            assert parts[0][0] == 0 and sum(r for _, r in parts) == N
            assert all(a + b == c for (a, b), (c, _) in zip(parts, parts[1:]))
            assert max(r for _, r in parts) - min(r for _, r in parts) <= 1


@pytest.mark.parametrize("world, N", [(2, 33), (3, 34)])   # ragged: 17 + 16, 12 + 11 + 11 rows
def test_gloo_shards_equal_the_unsharded_solve_bit_for_bit(world, N):
    from oracle import stamp_oracle as O
    seed = 5
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, world, port, N, seed, q)) for r in range(world)]
    for p in procs:
        p.start()
    got = dict(q.get(timeout=600) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for r in range(1, world):
        assert np.array_equal(got[0], got[r])        # every rank holds the gathered set
    P, init, goal = _problem()
    ref = O.solve(P, init, goal, N, SVGD, SGD, seed, LR, k=0)["theta"]
    assert np.array_equal(got[0], ref)
    assert np.array_equal(_run(1, 0, N, seed), ref)   # one rank through the same driver
