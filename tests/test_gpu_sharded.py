"""Particle shards through the library on one GPU: two shards of one set,
each with its own problem (rows offset into the set), exchange theta and
grad log rho by concatenation (what the all-gather delivers) and update
their own rows; together they must reproduce stamp_solve on the whole set
bit for bit.  The shards run one after the other: nothing waits on another
shard's kernels."""
import numpy as np
import pytest
import torch

from oracle import stamp_oracle as O
from paper_2310_01775_gb300 import workloads as W

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("name,over,N,svgd,sgd", [
    ("pusher1_h4", {}, 300, 4, 1),                    # one block, time-parallel sweep
    ("pusher3_h6", {"H": 2}, 203, 3, 1),              # three blocks, C = 25: segment replay
])
def test_two_shards_reproduce_the_whole_solve(name, over, N, svgd, sgd):
    from paper_2310_01775_gb300 import sharded as SH
    from paper_2310_01775_gb300 import stamp as S
    P = W.params(name, **over)
    init, goal = W.scene(P, 2)
    seed, lr = 11, P["lr"]
    stream = torch.cuda.current_stream().cuda_stream
    D = O.dims(P)[2]
    th0 = torch.tensor(O.init_theta(seed, N, D), dtype=torch.float32, device="cuda")

    whole = S.Problem(P, init, goal, N, stream)
    ref = torch.empty(N, D, device="cuda")
    whole.solve(N, svgd, sgd, seed, lr, th0, ref)
    whole.close()

    shards = [SH.LibraryShard(P, init, goal, N, *SH.partition(N, 2, r), seed, stream) for r in range(2)]
    th = [th0[s.row0:s.row0 + s.rows].clone() for s in shards]
    m = [torch.zeros_like(t) for t in th]
    v = [torch.zeros_like(t) for t in th]
    for it in range(svgd + sgd):
        g = [s.grad(t, it) for s, t in zip(shards, th)]
        th_all, g_all = torch.cat(th).contiguous(), torch.cat(g).contiguous()
        for s, t, mm, vv in zip(shards, th, m, v):
            s.step_rows(th_all, g_all, t, mm, vv, it + 1, lr, it >= svgd)
    for s in shards:
        s.prob.sync()
        s.close()
    assert torch.equal(torch.cat(th), ref)
