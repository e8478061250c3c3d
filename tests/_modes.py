"""Brute-force modes of two-push, one-block problems, and the whole-solve pin
of Algorithm 1 built on them (test infrastructure only).

A planted problem's goal is the end pose of a hard, noise-free rollout of a
random plan, so a plan of cost ~0 exists.  Its *modes* are the discrete plans
Gamma = (side of push 1, side of push 2) that can reach hard cost below
MODE_COST: every one of the 16 side sequences is rolled out on a grid of
N_OFF contact offsets x N_DIST push distances per push (495,616 hard
rollouts), and a sequence whose best grid point is near the bar is polished
by FP64 gradient steps on its four continuous parameters.  The rollouts use
the oracle's own force and substep functions, one pusher at a time.

The pin (Sec. III-A-1, Eq. svgd; Sec. V-B's diversity of solutions):
  coverage  every mode is the discrete plan of at least one final particle;
  descent   the attraction term moves the particles downhill: the median
            hard cost of the final particles is below DESCENT x that of the
            initial U(-1, 1) draws;
  spread    the repulsion term keeps them apart: the cost is bounded while
            theta ranges over R^D (the uniform base of App. A.1 with u -> inf),
            so the Stein repulsion spreads the particles, and their mean
            pairwise distance grows by SPREAD x or more;
  best      after the SGD phase (Algorithm 1), the lowest final hard cost
            is below MODE_COST, on a mode.
"""
from __future__ import annotations

import math

import numpy as np
import torch

from oracle import stamp_oracle as O

SOFT = dict(k_contact=1e3, c_contact=10.0)
N_OFF, N_DIST = 11, 16
MODE_COST = 1e-2
POLISH_BELOW = 5e-2          # grid costs in [MODE_COST, POLISH_BELOW) are polished
DESCENT, SPREAD = 0.7, 2.0
N_PARTICLES, ITERS, SGD_ITERS = 128, 200, 200


def params():
    """pusher1_h2's physics with the softer contact (k = 1e3, c = 10): the
    stiff constants' reverse sweep is dominated by contact chaos (see the
    whole-solve test), which leaves Algorithm 1 without a usable gradient."""
    from paper_2310_01775_gb300 import workloads as W
    return W.params("pusher1_h2", **SOFT)


def planted(P, seed):
    """(init, goal, plan): goal = end pose of the hard rollout of a U(-1,1)^D plan."""
    from paper_2310_01775_gb300 import workloads as W
    init, _ = W.scene(P, seed)
    D = O.dims(P)[2]
    plan = W.random_theta(1, D, 9100 + seed).astype(np.float64)
    _, fin = O.rollout(plan, P, init, init, None, hard=True)
    return init, fin[0, :, :3].copy(), plan


def _push(q, v, side, off, dist, P):
    """One hard push (one real pusher of unit weight) of T substeps from (q, v)."""
    sx, sy, ux, uy = O.pusher_geometry(q, off, dist, P)
    col = torch.as_tensor(side).long()[:, None]
    sx, sy, ux, uy = (t.gather(1, col) for t in (sx, sy, ux, uy))
    w = torch.ones_like(sx)
    step = dist[:, None] / P["T"]
    for j in range(P["T"]):
        q, v = O.substep(q, v, (sx + (j + 1) * step * ux, sy + (j + 1) * step * uy,
                                ux * step / P["dt"], uy * step / P["dt"], w), P)
    return q, v


def _pose_cost(q, goal, P):
    g = torch.as_tensor(goal, dtype=torch.float64)
    e = q - g[None]
    return (e[..., 0] ** 2 + e[..., 1] ** 2 + P["w_yaw"] * O.wrap(e[..., 2]) ** 2).sum(1)


def grid(P):
    """Every (side, offset, distance) of one push: offsets evenly over 90% of
    the offset range, distances at the midpoints of N_DIST equal bins."""
    offs = np.linspace(-0.9, 0.9, N_OFF) * P["offset_max"]
    dists = (np.arange(N_DIST) + 0.5) * (P["dist_max"] / N_DIST)
    s, o, d = np.meshgrid(np.arange(4), offs, dists, indexing="ij")
    return s.ravel(), o.ravel(), d.ravel()


def enumerate_grid(P, init, goal, chunk=64):
    """Best grid point of every side sequence: {(s1, s2): (cost, (o1, d1, o2, d2))}."""
    S1, O1, D1 = grid(P)
    n = S1.size
    with torch.no_grad():
        q0 = torch.as_tensor(init, dtype=torch.float64)[None].expand(n, 1, 3).clone()
        q1, v1 = _push(q0, torch.zeros(n, 1, 3, dtype=torch.float64), S1,
                       torch.as_tensor(O1), torch.as_tensor(D1), P)
        best = {}
        for a in range(0, n, chunk):
            b = min(n, a + chunk)
            qa, va = q1[a:b].repeat_interleave(n, 0), v1[a:b].repeat_interleave(n, 0)
            s2, o2, d2 = np.tile(S1, b - a), np.tile(O1, b - a), np.tile(D1, b - a)
            qf, _ = _push(qa, va, s2, torch.as_tensor(o2), torch.as_tensor(d2), P)
            d1 = np.repeat(D1[a:b], n)
            c = (_pose_cost(qf, goal, P).numpy() + P["w_push"] * (d1 ** 2 + d2 ** 2))
            s1, o1 = np.repeat(S1[a:b], n), np.repeat(O1[a:b], n)
            for key in range(16):
                msk = (s1 * 4 + s2) == key
                i = int(np.argmin(np.where(msk, c, np.inf)))
                k = (key // 4, key % 4)
                if k not in best or c[i] < best[k][0]:
                    best[k] = (float(c[i]), (o1[i], d1[i], o2[i], d2[i]))
    return best


def plan_theta(P, sides, params):
    """A particle whose hard plan is `sides` with the given (offset, distance) per push."""
    M, Pn, D = O.dims(P)
    th = np.zeros(D)
    for k, s in enumerate(sides):
        off, dist = params[2 * k], params[2 * k + 1]
        th[k * Pn:k * Pn + M] = -2.0
        th[k * Pn + s] = 2.0
        th[k * Pn + M] = math.atanh(off / P["offset_max"])
        th[k * Pn + M + 1] = math.log(dist / (P["dist_max"] - dist))
    return th


def polish(P, init, goal, starts, steps=60, lr=0.05):
    """FP64 gradient polish (Adam on u, v of both pushes) of hard plans
    `starts` = [(sides, (o1, d1, o2, d2))]; returns the lowest cost of each."""
    th0 = torch.as_tensor(np.stack([plan_theta(P, s, p) for s, p in starts]))
    M, Pn, _ = O.dims(P)
    cont = [k * Pn + M + j for k in range(P["H"]) for j in range(2)]
    x = th0[:, cont].clone().requires_grad_(True)
    opt = torch.optim.Adam([x], lr=lr)
    best = np.full(len(starts), np.inf)
    for _ in range(steps + 1):
        th = th0.clone()
        th[:, cont] = x
        q, _, _, _, dist, _ = O.simulate(th, P, init, None, hard=True)
        c = O.cost(q, dist, goal, P)
        best = np.minimum(best, c.detach().numpy())
        opt.zero_grad()
        c.sum().backward()
        opt.step()
    return best


def modes(P, init, goal):
    """{sides: cost} of every side sequence that reaches hard cost < MODE_COST
    (grid, then polish of the sequences whose grid optimum is near the bar),
    and the full table of best costs."""
    best = enumerate_grid(P, init, goal)
    table = {k: v[0] for k, v in best.items()}
    near = [(k, v[1]) for k, v in best.items() if MODE_COST <= v[0] < POLISH_BELOW]
    if near:
        for (k, _), c in zip(near, polish(P, init, goal, near)):
            table[k] = min(table[k], float(c))
    return {k: c for k, c in table.items() if c < MODE_COST}, table


def mean_pairwise_distance(theta):
    return float(np.sqrt(O.pairwise_sq_dists(theta)).mean())


def pin(P, init, goal, seed, theta_final, cost_final, mode_set):
    """The four checks; returns (failures, summary)."""
    D = O.dims(P)[2]
    th0 = O.init_theta(seed, N_PARTICLES, D)
    c0, _ = O.rollout(th0, P, init, goal, None, hard=True)
    codes = [tuple(int(x) for x in r) for r in O.plan_codes(theta_final, P)]
    held = set(codes)
    ibest = int(np.argmin(cost_final))
    s = dict(modes=sorted(mode_set), missing=sorted(set(mode_set) - held),
             median0=float(np.median(c0)), median=float(np.median(cost_final)),
             spread0=mean_pairwise_distance(th0), spread=mean_pairwise_distance(theta_final),
             best=float(cost_final[ibest]), best_plan=codes[ibest])
    fails = []
    if s["missing"]:
        fails.append("coverage")
    if not s["median"] < DESCENT * s["median0"]:
        fails.append("descent")
    if not s["spread"] > SPREAD * s["spread0"]:
        fails.append("spread")
    if not (s["best"] < MODE_COST and s["best_plan"] in mode_set):
        fails.append("best")
    return fails, s
