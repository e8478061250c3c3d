"""Whole-solve pin on the GPU: stamp_solve (Algorithm 1: 200 SVGD then 200
SGD iterations, N = 128) on the planted two-push problems of
tests/test_oracle_solve_modes.py must pass the same brute-force pin as the
FP64 oracle's solve: every mode held by a final particle's discrete plan,
the median hard cost below 0.7x the initial draws', the particles' mean
pairwise distance grown 2x or more, and the best particle on a mode below
cost 1e-2 (see tests/_modes.py).  The modes come from the oracle's brute
force; nothing expected comes from the CUDA path.
"""
import multiprocessing as mp

import numpy as np
import pytest
import torch

import _modes as MD

pytestmark = pytest.mark.gpu
SEEDS = (0, 1, 2, 3)


def _modes_job(seed):
    import torch
    torch.set_num_threads(4)
    P = MD.params()
    init, goal, _ = MD.planted(P, seed)
    return seed, MD.modes(P, init, goal)[0]


@pytest.fixture(scope="module")
def modes():
    with mp.get_context("spawn").Pool(len(SEEDS)) as pool:
        return dict(pool.map(_modes_job, SEEDS))


@pytest.mark.parametrize("seed", SEEDS)
def test_gpu_solve_covers_every_brute_force_mode(modes, seed):
    from paper_2310_01775_gb300 import stamp as S
    P = MD.params()
    init, goal, _ = MD.planted(P, seed)
    N = MD.N_PARTICLES
    prob = S.Problem(P, init, goal, N, torch.cuda.current_stream().cuda_stream)
    th = torch.zeros(N, prob.D, device="cuda")
    cost = torch.zeros(N, device="cuda")
    topk = np.zeros(3, dtype=np.int32)
    prob.solve(N, MD.ITERS, MD.SGD_ITERS, seed, P["lr"], None, th, cost, 3, topk, None)
    prob.close()
    fails, s = MD.pin(P, init, goal, seed, th.cpu().numpy().astype(np.float64),
                      cost.cpu().numpy().astype(np.float64), modes[seed])
    assert not fails, (fails, s)
