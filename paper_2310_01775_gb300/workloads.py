"""Seeded synthetic workloads for the STAMP block-pushing path.

This module only draws numbers: scene poses, goal poses and random
parameter/gradient arrays for parity cases. It holds none of the method's
arithmetic (no simulation, relaxation, kernel or optimiser step), so both the
CUDA path and the FP64 oracle may be fed from it.

Physical constants follow the block-pushing setup of Sec. V-A-2 / App. D
(0.1 m square block of 1 kg pushed on one of its four sides); the paper leaves
the numbers to its simulator, so the values below are the workload's own
(friction 0.3, pusher disk radius 0.01 m, penalty contact k=1e4 with damping 50,
semi-implicit Euler with dt=0.01, Gumbel-softmax temperature 0.5, Adam lr 1e-2).
"""
from __future__ import annotations

import math

import numpy as np

# Physics and relaxation constants shared by every workload (SI units).
PHYSICS = dict(
    half_size=0.05,    # block half side [m] (0.1 m square)
    mass=1.0,          # block mass [kg]
    mu=0.3,            # ground Coulomb coefficient
    mu_c=0.3,          # pusher/block and block/block Coulomb coefficient
    g=9.81,            # gravity [m/s^2]
    pusher_r=0.01,     # pusher disk radius [m]
    k_contact=1e4,     # penalty stiffness [N/m]
    c_contact=50.0,    # penalty damping [N s/m]
    eps_v=0.05,        # ground-friction smoothing, linear [m/s]
    eps_w=1.0,         # ground-friction smoothing, angular [rad/s]
    eps_t=0.05,        # contact-friction smoothing, tangential [m/s]
    dt=0.01,           # integrator step [s]
    tau=0.5,           # Gumbel-softmax temperature
    w_yaw=0.1,         # cost weight of the squared wrapped yaw error
    w_push=1e-3,       # cost weight of the squared push distances
    offset_max=0.05,   # contact offset range [-offset_max, offset_max] [m]
    dist_max=0.3,      # push distance range [0, dist_max] [m]
)

# The workloads: block count, horizon H (actions), substeps T per action,
# checkpoint interval, particle count, SVGD iterations, Adam step size.
CONFIGS = {
    # 1 block, 2 pushes of 50 substeps, 32 particles, 200 iterations (D=12).
    "pusher1_h2": dict(n_blocks=1, H=2, T=50, ckpt_every=25, N=32,
                       svgd_iters=200, lr=1e-2),
    # 1 block, 4 pushes of 100 substeps, 1024 particles, 500 iterations (D=24).
    # Every substep is checkpointed (a 9.9 MB tape): the adjoint then replays
    # nothing, 1.6x faster than a checkpoint every 25 substeps on GB300.
    "pusher1_h4": dict(n_blocks=1, H=4, T=100, ckpt_every=1, N=1024,
                       svgd_iters=500, lr=1e-2),
    # 3 blocks with block-block contact, 6 pushes of 100 substeps, a
    # checkpoint every 25 substeps, 2048 particles (D=84).
    "pusher3_h6": dict(n_blocks=3, H=6, T=100, ckpt_every=25, N=2048,
                       svgd_iters=500, lr=1e-2),
}


def params(name: str, **over) -> dict:
    """Full parameter dict (physics + workload) for a named workload."""
    p = dict(PHYSICS)
    p.update(CONFIGS[name])
    p.update(over)
    return p


def dims(p: dict) -> tuple[int, int, int]:
    """(M choices per action, P parameters per action, D particle dimension)."""
    m = 4 * p["n_blocks"]
    return m, m + 2, p["H"] * (m + 2)


def scene(p: dict, seed: int) -> tuple[np.ndarray, np.ndarray]:
    """Initial and goal poses (n_blocks x 3: x, y, yaw), float64.

    One block: it starts at the origin with yaw 0; the goal position is
    uniform in the 0.5 m disc around it (radius 0.5*sqrt(U)) and the goal
    yaw uniform in [-pi/2, pi/2].  Several blocks: centres rejection-sampled
    in [-0.5, 0.5]^2 with pairwise centre distance above 0.16 m (more than
    two circumscribed radii of a 0.1 m square), yaw uniform in
    [-pi/2, pi/2]; goals are drawn the same way.
    """
    rng = np.random.default_rng(np.random.SeedSequence([seed, 0x5CE4E]))
    nb = p["n_blocks"]
    if nb == 1:
        init = np.zeros((1, 3))
        r = 0.5 * math.sqrt(rng.uniform())
        a = rng.uniform(0.0, 2.0 * math.pi)
        goal = np.array([[r * math.cos(a), r * math.sin(a),
                          rng.uniform(-math.pi / 2, math.pi / 2)]])
        return init, goal

    def spread():
        while True:
            c = rng.uniform(-0.5, 0.5, size=(nb, 2))
            d = np.sqrt(((c[:, None, :] - c[None, :, :]) ** 2).sum(-1))
            if (d[np.triu_indices(nb, 1)] > 0.16).all():
                yaw = rng.uniform(-math.pi / 2, math.pi / 2, size=(nb, 1))
                return np.concatenate([c, yaw], axis=1)

    return spread(), spread()


def random_theta(n: int, d: int, seed: int, scale: float = 1.0) -> np.ndarray:
    """Parity-test particles: uniform in [-scale, scale]^d, float32."""
    rng = np.random.default_rng(np.random.SeedSequence([seed, 0x7E7A]))
    return rng.uniform(-scale, scale, size=(n, d)).astype(np.float32)


def random_normal(shape, seed: int, scale: float = 1.0) -> np.ndarray:
    """Parity-test arrays (gradients, Adam moments): N(0, scale^2), float32."""
    rng = np.random.default_rng(np.random.SeedSequence([seed, 0x6A55]))
    return (scale * rng.standard_normal(size=shape)).astype(np.float32)


def mlp_init(sizes, seed: int):
    """Initial MLP parameters [(W (out, in), b (out,))] per layer: uniform in
    [-1/sqrt(in), 1/sqrt(in)], float64 (cast as needed)."""
    rng = np.random.default_rng(np.random.SeedSequence([seed, 0x4D4C50]))
    out = []
    for i, o in zip(sizes[:-1], sizes[1:]):
        k = 1.0 / math.sqrt(i)
        out.append((rng.uniform(-k, k, size=(o, i)), rng.uniform(-k, k, size=o)))
    return out


def batch_instances(n: int = 256, seed: int = 0, T: int = 100) -> list[dict]:
    """Seeded uneven instances for batched serving: blocks uniform in 1..4,
    horizon uniform in 2..8, particles log-uniform in [64, 1024] (rounded
    down), scenes from `scene`; each instance has its own solve seed."""
    rng = np.random.default_rng(np.random.SeedSequence([seed, 0xBA7C4]))
    out = []
    for g in range(n):
        nb = int(rng.integers(1, 5))
        H = int(rng.integers(2, 9))
        N = int(math.exp(rng.uniform(math.log(64), math.log(1024))))
        p = dict(PHYSICS, n_blocks=nb, H=H, T=T)
        init, goal = scene(p, 7919 * seed + g)
        out.append({"n_blocks": nb, "H": H, "N": N, "seed": 100003 * seed + g,
                    "init": init, "goal": goal})
    return out
