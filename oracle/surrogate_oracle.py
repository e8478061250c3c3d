"""FP64 reference of the learned pose-dynamics surrogate and of its training data.

TEST INFRASTRUCTURE ONLY: tests and the benchmark's CPU baseline may run it;
the product path never imports it.

The planning cost, the relaxation and the Stein update are the paper's
(Eq. gamma_map, Eq. svgd, Sec. III-B).  The surrogate is a learned stand-in
for the simulator of one push: it maps the blocks' poses at the push start
and the push's relaxed parameters to the pose change after the push.

Features of push k (F = 8 n_b + 2 values):
    f = [x_b, y_b, cos phi_b, sin phi_b for each block b]
        ++ z~_k  (M relaxed choice weights)
        ++ [offset_k / offset_max, dist_k / dist_max]     (= tanh u_k, sigmoid v_k)
Pose recursion and cost:
    q_0 = the scene's start poses,   q_{k+1} = q_k + MLP(f(q_k, action k))
    C   = sum_b |p_b - g_b|^2 + w_yaw wrap(phi_b - phi_gb)^2 + w_push sum_k dist_k^2
(the simulator's cost on q_H), with MLP the network of oracle/mlp_oracle.py
written here in torch float64 so that reverse mode gives -dC/dtheta.

Training transitions (one push from a random scene; the pose samplers are
counter-based SplitMix64 draws, the same definitions the CUDA sampler uses):
    transition g lives in chunk c0 = g - g mod 4096 with local index i; the
    chunk key is cs = sm64(seed, c0).
    start poses: key sm64(cs, 2); attempt a = 0..31 draws
        u_{b,q} = U(sm64(key, (32 i + a) * 12 + 3 b + q))
        x_b = u_{b,0} - 1/2,  y_b = u_{b,1} - 1/2,  phi_b = (u_{b,2} - 1/2) * pi_f
    in float32 (pi_f = float32(3.14159265)); the first attempt whose block
    centres are all more than 0.16 m apart (dx*dx + dy*dy > 0.16*0.16, each
    product and the sum rounded to float32) is taken; if none is, attempt 31
    with x_b = -0.4 + 0.8 b / max(n_b - 1, 1).
    action: key sm64(cs, 3); u_j = U(sm64(key, i (P + 1) + j)) for j <= P
    (P = M + 2); theta_j = (u_j - 1/2) * 6 in float32 for j < P, and the M
    logits are further multiplied by u_P, so the choice weights range from
    nearly uniform to nearly one-hot (each product rounded to float32).
    push: the simulator's one-action rollout (H = 1) from the start poses at
    rest, Gumbel noise of seed cs, iteration 0; the target is the pose change
    q_final - q_start.
"""
from __future__ import annotations

import numpy as np
import torch

from . import stamp_oracle as O

CHUNK = 4096
STREAM_POSES, STREAM_ACTIONS = 2, 3
MAX_BLOCKS = 4          # pose draws are laid out for up to four blocks per attempt
ATTEMPTS = 32


def feature_dims(n_blocks: int) -> tuple[int, int]:
    """(F, 3 n_b): network input and output widths."""
    return 8 * n_blocks + 2, 3 * n_blocks


# ----------------------------------------------------------------------------
# Training transitions
# ----------------------------------------------------------------------------


def _chunks(seed: int, n: int):
    for c0 in range(0, n, CHUNK):
        yield c0, min(CHUNK, n - c0), int(O.sm64(np.uint64(seed), np.uint64(c0)))


def sample_start_poses(cs: int, m: int, nb: int) -> np.ndarray:
    """(m, nb, 3) float32 start poses of one chunk, as defined in the header."""
    key = O.sm64(np.uint64(cs), STREAM_POSES)
    f32 = np.float32
    pi_f, half, thr = f32(3.14159265), f32(0.5), f32(0.16) * f32(0.16)
    out = np.zeros((m, nb, 3), dtype=np.float32)
    for i in range(m):
        for att in range(ATTEMPTS):
            base = (i * ATTEMPTS + att) * 3 * MAX_BLOCKS
            ctr = base + np.arange(3 * nb, dtype=np.uint64)
            u = O.uniform23(O.sm64(key, ctr)).astype(np.float32).reshape(nb, 3)
            p = np.empty((nb, 3), dtype=np.float32)
            p[:, 0] = u[:, 0] - half
            p[:, 1] = u[:, 1] - half
            p[:, 2] = (u[:, 2] - half) * pi_f
            ok = True
            for a in range(nb):
                for b in range(a + 1, nb):
                    dx, dy = p[a, 0] - p[b, 0], p[a, 1] - p[b, 1]
                    ok &= bool(f32(dx * dx) + f32(dy * dy) > thr)
            if ok:
                break
        if not ok:
            den = f32(max(nb - 1, 1))
            for b in range(nb):
                p[b, 0] = f32(-0.4) + f32(0.8) * f32(b) / den
        out[i] = p
    return out


def sample_actions(cs: int, m: int, Pn: int) -> np.ndarray:
    """(m, Pn) float32 action parameters of one chunk, in [-3, 3]."""
    key = O.sm64(np.uint64(cs), STREAM_ACTIONS)
    ctr = np.arange(m * (Pn + 1), dtype=np.uint64).reshape(m, Pn + 1)
    u = O.uniform23(O.sm64(key, ctr)).astype(np.float32)
    th = (u[:, :Pn] - np.float32(0.5)) * np.float32(6.0)
    th[:, :Pn - 2] *= u[:, Pn:]
    return th


def transitions(seed: int, n: int, P: dict, dtype=torch.float64):
    """Features (n, F), targets (n, 3 nb), start poses and actions of the first
    n transitions of `seed` under the physics of P (its H is ignored)."""
    nb = P["n_blocks"]
    P1 = dict(P, H=1)
    M, Pn, _ = O.dims(P1)
    xs, ys, starts, thetas = [], [], [], []
    for c0, m, cs in _chunks(seed, n):
        q0 = sample_start_poses(cs, m, nb)
        th = sample_actions(cs, m, Pn)
        g = O.gumbel_noise(cs, 0, m, 1, M)
        tt = torch.as_tensor(th.astype(np.float64), dtype=dtype)
        with torch.no_grad():
            q, _, z, off, dist, _ = O.simulate(tt, P1, q0.astype(np.float64), g)
            qs = torch.as_tensor(q0.astype(np.float64), dtype=dtype)
            xs.append(features(qs, z[:, 0], off[:, 0], dist[:, 0], P).numpy())
            ys.append((q - qs).reshape(m, 3 * nb).numpy())
        starts.append(q0)
        thetas.append(th)
    return (np.concatenate(xs), np.concatenate(ys), np.concatenate(starts),
            np.concatenate(thetas))


# ----------------------------------------------------------------------------
# Surrogate rollout
# ----------------------------------------------------------------------------


def features(q, z, offset, dist, P):
    """f(q, z~, offset, dist) for one push: q (N, nb, 3), z (N, M), offset and dist (N,)."""
    N = q.shape[0]
    pose = torch.stack([q[..., 0], q[..., 1], torch.cos(q[..., 2]), torch.sin(q[..., 2])], -1)
    return torch.cat([pose.reshape(N, -1), z, (offset / P["offset_max"])[:, None],
                      (dist / P["dist_max"])[:, None]], -1)


def mlp(params, x):
    """The multilayer perceptron of oracle/mlp_oracle.py: SiLU hidden layers, linear head."""
    a = x
    for l, (W, b) in enumerate(params):
        Wt = torch.as_tensor(np.asarray(W, dtype=np.float64), dtype=x.dtype)
        bt = torch.as_tensor(np.asarray(b, dtype=np.float64), dtype=x.dtype)
        zl = a @ Wt.T + bt
        a = zl * torch.sigmoid(zl) if l < len(params) - 1 else zl
    return a


def surrogate_poses(params, theta, P, init_poses, gumbel=None):
    """Poses q_0..q_H (list of (N, nb, 3)) and the relaxed dist (N, H)."""
    N, nb = theta.shape[0], P["n_blocks"]
    z, offset, dist = O.relax(theta, P, gumbel)
    q = torch.as_tensor(np.asarray(init_poses, dtype=np.float64), dtype=theta.dtype)
    q = q.expand(N, nb, 3) if q.dim() == 3 else q[None].expand(N, nb, 3)
    qs = [q]
    for k in range(P["H"]):
        q = q + mlp(params, features(q, z[:, k], offset[:, k], dist[:, k], P)).reshape(N, nb, 3)
        qs.append(q)
    return qs, dist


def rollout(params, theta, P, init_poses, goal_poses, gumbel=None):
    """Surrogate cost C(theta) of every particle."""
    th = torch.as_tensor(np.asarray(theta, dtype=np.float64))
    with torch.no_grad():
        qs, dist = surrogate_poses(params, th, P, init_poses, gumbel)
        return O.cost(qs[-1], dist, goal_poses, P).numpy()


def rollout_grad(params, theta, P, init_poses, goal_poses, gumbel=None):
    """Surrogate cost and grad log rho = -dC/dtheta (reverse mode through the H
    chained network evaluations and the relaxation)."""
    th = torch.tensor(np.asarray(theta, dtype=np.float64), requires_grad=True)
    qs, dist = surrogate_poses(params, th, P, init_poses, gumbel)
    c = O.cost(qs[-1], dist, goal_poses, P)
    (g,) = torch.autograd.grad(c.sum(), th)
    return c.detach().numpy(), (-g).numpy()


def select_lowest(costs, N):
    """Indices of the N lowest costs, ties to the lower index (the screening rule)."""
    c = np.asarray(costs)
    return np.lexsort((np.arange(len(c)), c))[:N]
