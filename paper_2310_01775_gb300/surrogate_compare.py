"""Surrogate-assisted against plain SVGD: wall time to a target hard cost.

Problems are planted so that a plan of zero pose error exists: the start
scene of the workload's scene generator, and as goal the poses a hard
(one-hot, noise-free) rollout of a random plan reaches.  Both arms run
Algorithm 1 through the C ABI with the same particle count, learning rate,
seed and early stop (every `check_every` iterations the particles are rolled
out hard on the simulator; the solve ends when the lowest cost is below the
target); the surrogate arm first trains the surrogate on simulator
transitions, then screens `n_candidates` uniform particles down to N and
runs its first iterations on the surrogate's gradients.  Argument
marshalling only: every step runs in libstamp.so.
"""
from __future__ import annotations

import time

import numpy as np
import torch

from . import stamp as S
from . import workloads as W


def planted_scene(P: dict, seed: int, stream) -> tuple[np.ndarray, np.ndarray]:
    """(init, goal): the scene generator's start poses and, as goal, the end
    poses of a hard rollout of the plan 3 * U(-1, 1)^D (seeded)."""
    init, _ = W.scene(P, seed)
    _, _, D = W.dims(P)
    plan = torch.tensor(3.0 * W.random_theta(1, D, 9000 + seed), device="cuda")
    prob = S.Problem(P, init, init, 1, stream)
    cost = torch.empty(1, device="cuda")
    final = torch.empty(1, 6 * P["n_blocks"], device="cuda")
    prob.rollout_fwd(plan, 1, 0, -1, 1, cost, final)
    prob.sync()
    prob.close()
    goal = final.cpu().numpy().reshape(P["n_blocks"], 6)[:, :3].astype(np.float64)
    return init, goal


def train_surrogate(P: dict, n_transitions: int, stream, max_rows: int, max_particles: int,
                    seed: int = 1, epochs: int = 16, batch: int = 4096, lr: float = 2e-3):
    """A surrogate trained on n GPU transitions; returns it and the seconds spent
    generating and training."""
    sur = S.Surrogate(P, max_rows, max_particles, stream)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    x = torch.empty(n_transitions, sur.in_dim, device="cuda")
    y = torch.empty(n_transitions, sur.out_dim, device="cuda")
    sur.transitions(n_transitions, seed, x, y)
    sur.init_params(seed + 1)
    losses = sur.train(x, y, n_transitions, epochs, batch, lr)
    torch.cuda.synchronize()
    secs = time.perf_counter() - t0
    del x, y
    return sur, secs, losses


def compare(P: dict, seeds, sur, *, N: int, n_candidates: int, surrogate_iters: int,
            sim_iters: int, sgd_iters: int = 0, plain_iters: int | None = None,
            plain_sgd_iters: int = 0, target: float = 1e-3, check_every: int = 10,
            lr: float = 1e-2, stream=None) -> dict:
    """Both arms on each planted problem; per seed: wall seconds, iterations
    run, lowest hard cost and whether the target was reached."""
    plain_iters = surrogate_iters + sim_iters if plain_iters is None else plain_iters
    _, _, D = W.dims(P)
    rows = []
    for seed in seeds:
        init, goal = planted_scene(P, seed, stream)
        prob = S.Problem(P, init, goal, N, stream)
        prob.set_target(target, check_every)
        theta = torch.empty(N, D, device="cuda")
        cost = torch.empty(N, device="cuda")
        row = {"seed": int(seed)}
        for arm in ("plain", "surrogate"):
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            if arm == "plain":
                prob.solve(N, plain_iters, plain_sgd_iters, seed, lr, None, theta, cost)
            else:
                prob.solve_surrogate(sur, n_candidates, N, surrogate_iters, sim_iters, seed, lr,
                                     theta, cost, sgd_iters=sgd_iters)
            secs = time.perf_counter() - t0
            it, best = prob.solve_info()
            row[arm] = {"seconds": round(secs, 4), "iterations": it, "best_cost": float(best),
                        "reached": bool(best < target)}
        prob.set_target(0.0, 0)
        prob.close()
        rows.append(row)
    return {
        "target": target, "N": N, "n_candidates": n_candidates,
        "surrogate_iters": surrogate_iters, "sim_iters": sim_iters, "sgd_iters": sgd_iters,
        "plain_iters": plain_iters, "plain_sgd_iters": plain_sgd_iters, "per_seed": rows,
    }
