"""Whole-solve pin of the oracle's Algorithm 1 (oracle.solve) by brute force.

Two planted two-push problems (goal = end pose of a random hard plan, so a
zero-pose-error plan exists).  Brute force over the 16 side sequences x a
grid of offsets and distances per push (then an FP64 gradient polish near
the bar) gives the modes: side sequences that reach hard cost < 1e-2.  The
oracle's solve (N = 128 particles, 200 SVGD then 200 SGD iterations of
Algorithm 1) must hold every mode
among its final particles' discrete plans, move downhill (term A of
Eq. svgd), spread its particles (term B) and end with its best particle on a
mode below the bar (see tests/_modes.py).

Two mistakes planted in the oracle, each in a fresh process, must fail the
pin: the gradient's sign flipped (attraction uphill) and the repulsion term
dropped.  The physics is pusher1_h2's with the softer contact (k = 1e3,
c = 10); at the stiff constants (k = 1e4, c = 50) the same solve cannot be
told from the sign-flipped one (medians of the final hard costs 0.227 and
0.258 from 0.31, particle spread unchanged), because the reverse sweep
through the chattering contact gives no usable gradient.
"""
import multiprocessing as mp

import numpy as np
import pytest

SEEDS = (0, 1)


def _job(job):
    import torch
    from oracle import stamp_oracle as O
    import _modes as MD
    kind, seed, mutant = job
    P = MD.params()
    init, goal, plan = MD.planted(P, seed)
    if kind == "modes":
        torch.set_num_threads(2)
        c_plan, _ = O.rollout(plan, P, init, goal, None, hard=True)
        m, table = MD.modes(P, init, goal)
        return job, dict(modes=m, table=table, plan_cost=float(c_plan[0]),
                         plan_sides=tuple(int(x) for x in O.plan_codes(plan, P)[0]))
    torch.set_num_threads(1)
    if mutant == "sign":          # ascend the cost: grad log rho with the wrong sign
        step = O.svgd_step
        O.svgd_step = lambda th, g, m, v, s, lr, sgd_phase=False: step(
            th, -np.asarray(g), m, v, s, lr, sgd_phase)
    elif mutant == "norep":       # Eq. svgd without its repulsive term (B)
        def attract_only(theta, grad_logp, h, chunk=128, weights=None):
            th = np.asarray(theta, dtype=np.float64)
            d2 = ((th[:, None] - th[None]) ** 2).sum(-1)
            return np.exp(-d2 / h) @ np.asarray(grad_logp) / th.shape[0]
        O.stein_direction = attract_only
    r = O.solve(P, init, goal, MD.N_PARTICLES, MD.ITERS, MD.SGD_ITERS, seed, P["lr"])
    return job, dict(theta=r["theta"], cost=r["cost_hard"])


@pytest.fixture(scope="module")
def results():
    jobs = ([("modes", s, None) for s in SEEDS] + [("solve", s, None) for s in SEEDS]
            + [("solve", 0, "sign"), ("solve", 0, "norep")])
    # a fresh process per job: the planted mistakes patch the oracle module
    with mp.get_context("spawn").Pool(len(jobs), maxtasksperchild=1) as pool:
        return dict(pool.map(_job, jobs))


def test_brute_force_finds_the_planted_plan(results):
    for s in SEEDS:
        r = results[("modes", s, None)]
        assert r["plan_cost"] < 1e-3                 # only the push-length term remains
        assert r["plan_sides"] in r["modes"]
        assert len(r["table"]) == 16


@pytest.mark.parametrize("seed", SEEDS)
def test_oracle_solve_covers_every_brute_force_mode(results, seed):
    from oracle import stamp_oracle as O
    import _modes as MD
    P = MD.params()
    init, goal, _ = MD.planted(P, seed)
    r = results[("solve", seed, None)]
    fails, s = MD.pin(P, init, goal, seed, r["theta"], r["cost"],
                      results[("modes", seed, None)]["modes"])
    assert not fails, (fails, s)


@pytest.mark.parametrize("mutant,check", [("sign", "descent"), ("norep", "spread")])
def test_planted_mistakes_fail_the_pin(results, mutant, check):
    import _modes as MD
    P = MD.params()
    init, goal, _ = MD.planted(P, 0)
    r = results[("solve", 0, mutant)]
    fails, s = MD.pin(P, init, goal, 0, r["theta"], r["cost"], results[("modes", 0, None)]["modes"])
    assert check in fails, (fails, s)
