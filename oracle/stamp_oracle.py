"""FP64 CPU oracle for one STAMP iteration over relaxed block-pushing plans.

TEST INFRASTRUCTURE ONLY.  Nothing in the product path imports this module;
only the tests, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` run it.  It shares no code with the CUDA library: it is written in
plain PyTorch CPU ops (float64 by default), one obviously-correct step after
another, and its plan-parameter gradient comes from ``torch.autograd`` (the
reverse-mode tape of Sec. III-B) rather than a hand-derived adjoint.

What it computes (paper passages in brackets):
  * relaxation  z~_k = softmax((a_k + gumbel_k)/tau), Gamma = argmax one-hot
    [Sec. IV-A, Eq. gamma_map]; offset = offset_max*tanh(u), distance =
    dist_max*sigmoid(v) keep the particle on R^D [App. A.1];
  * a planar rigid-body pushing simulator: kinematic disk pushers, spring
    (penalty) contacts with damping, smoothed Coulomb friction, semi-implicit
    Euler [Sec. III-B];
  * the goal cost C and log rho = -C [Eq. posterior_dist, neglog_likelihood];
  * the RBF Stein update with a median-heuristic bandwidth [Eq. svgd;
    App. C.3 for the median heuristic] with unit importance weights
    [Eq. dsvgd with w_j = 1], Adam on -phi, and the SGD phase of Algorithm 1;
  * the final hard evaluation (Gamma, no noise) and the distinct-plan top-k.

Readings where the paper is silent (it delegates physics to its simulator):
  * pusher c = (object o, side s), s in N,E,S,W with outward normals
    (0,1),(1,0),(0,-1),(-1,0) and tangent t = (-n_y, n_x) in the block frame;
    at action start it touches side s (gap 0) at tangential offset `offset`
    and then moves a distance `dist` along -n at constant speed over the T
    substeps; during substep j its centre is p_start + (j/T)*dist*u;
  * every virtual pusher acts on every block, weighted by z~_{k,c};
  * disk/box: signed distance of the pusher centre to the square; contact iff
    r - sd > 0 (strict); normal from the block to the pusher (outside: the
    normalised clamped offset, inside: the axis of the larger q, ties to x);
    contact point p - r*n; normal force max(0, k*delta - c*v_n); tangential
    smoothed Coulomb mu_c*f_n*v_t/sqrt(|v_t|^2 + eps_t^2);
  * box/box: every corner of one box tested against the other box, normal =
    outward face normal of the penetrated box (axis of the larger q, ties to
    x), equal and opposite forces applied at the corner point;
  * ground: F = -mu*m*g*v/sqrt(|v|^2+eps_v^2),
    torque = -mu*m*g*r_eff*omega/sqrt(omega^2+eps_w^2), r_eff the mean distance
    of a uniform square to its centre, (a/6)(sqrt2 + ln(1+sqrt2));
  * cost = sum_b |p_b - g_b|^2 + w_yaw*wrap(phi_b - phi_gb)^2
           + w_push*sum_k dist_k^2, wrap(e) = atan2(sin e, cos e);
  * bandwidth h = med / ln(N+1), med the element of rank floor((M-1)/2) of
    the ascending squared distances d2_ij, i<j (M = N(N-1)/2); h = 1 when
    N = 1 or h < 1e-12;
  * Gumbel noise from SplitMix64 (Steele, Lea & Flood, OOPSLA 2014) used as a
    counter-based generator; see ``sm64``.
Parity status: every function here is pinned by a test in tests/test_oracle_*.py.
``solve`` (Algorithm 1 over many iterations) is pinned by brute force
(tests/test_oracle_solve_modes.py): on planted two-push problems with the
softer contact, its final particles hold every side sequence that a grid
search plus gradient polish shows can reach cost < 1e-2, move downhill, keep
spreading, and end on such a mode; a sign error in the gradient and a dropped
repulsion term each fail that pin.  Per-particle values of long solves at the
stiff contact constants are chaotic and stay unpinned.
"""
from __future__ import annotations

import math

import numpy as np
import torch

# ----------------------------------------------------------------------------
# Counter-based random numbers: SplitMix64 (Steele, Lea & Flood 2014).
# The generator's state advances by the golden-ratio increment and each output
# is the state passed through the published finaliser.  Output number n+1 of a
# generator started at state `key` is therefore mix(key + (n+1)*GAMMA), which
# is what `sm64` returns; keys are derived by chaining it.
# ----------------------------------------------------------------------------
GAMMA = np.uint64(0x9E3779B97F4A7C15)
STREAM_GUMBEL = 0
STREAM_INIT = 1


def _mix(z):
    z = np.asarray(z, dtype=np.uint64)
    with np.errstate(over="ignore"):
        z = (z ^ (z >> np.uint64(30))) * np.uint64(0xBF58476D1CE4E5B9)
        z = (z ^ (z >> np.uint64(27))) * np.uint64(0x94D049BB133111EB)
    return z ^ (z >> np.uint64(31))


def sm64(key, ctr):
    """Output number ctr+1 of a SplitMix64 generator started at state `key`."""
    key = np.asarray(key, dtype=np.uint64)
    ctr = np.asarray(ctr, dtype=np.uint64)
    with np.errstate(over="ignore"):
        return _mix(key + (ctr + np.uint64(1)) * GAMMA)


def uniform23(x):
    """Top 23 bits of a 64-bit draw as a float in (0, 1): ((x>>41)+0.5)/2^23,
    a value that float32 represents exactly."""
    return ((np.asarray(x, dtype=np.uint64) >> np.uint64(41)).astype(np.float64) + 0.5) * 2.0 ** -23


def gumbel_noise(seed: int, it: int, n: int, H: int, M: int) -> np.ndarray:
    """Gumbel(0,1) draws g[i,k,c] = -ln(-ln U) for particle i, action k, choice c.

    U comes from draw number (i*H + k)*M + c of the key chain
    seed -> stream 0 -> iteration `it`.
    """
    key = sm64(sm64(np.uint64(seed), STREAM_GUMBEL), np.uint64(it))
    ctr = np.arange(n * H * M, dtype=np.uint64).reshape(n, H, M)
    u = uniform23(sm64(key, ctr))
    return -np.log(-np.log(u))


def init_theta(seed: int, n: int, d: int) -> np.ndarray:
    """Initial particles theta ~ U(-1,1)^d: the uniform base distribution p0
    of App. A.1.  Draw number i*d + j of the key chain seed -> stream 1."""
    key = sm64(np.uint64(seed), STREAM_INIT)
    ctr = np.arange(n * d, dtype=np.uint64).reshape(n, d)
    return 2.0 * uniform23(sm64(key, ctr)) - 1.0


# ----------------------------------------------------------------------------
# Problem geometry
# ----------------------------------------------------------------------------
# Sides N, E, S, W: outward normals in the block frame (Sec. V-A-2 orders the
# four sides north, east, south, west).
SIDE_NORMALS = np.array([[0.0, 1.0], [1.0, 0.0], [0.0, -1.0], [-1.0, 0.0]])


def dims(P):
    m = 4 * P["n_blocks"]
    return m, m + 2, P["H"] * (m + 2)


def inertia(P):
    """Moment of inertia of a uniform square of side a about its centre,
    m*(a^2 + a^2)/12."""
    a = 2.0 * P["half_size"]
    return P["mass"] * (a * a + a * a) / 12.0


def r_eff(P):
    """Mean distance from the centre of a uniform square of side a to its
    points, (a/6)(sqrt(2) + ln(1 + sqrt(2)))."""
    a = 2.0 * P["half_size"]
    return a / 6.0 * (math.sqrt(2.0) + math.log(1.0 + math.sqrt(2.0)))


def relax(theta, P, gumbel=None, hard=False):
    """Per-action relaxed choice weights, offsets and push distances.

    theta: (N, D) laid out per action k as [a_k (M logits), u_k, v_k].
    Returns z (N,H,M), offset (N,H), dist (N,H).
    Soft:  z~_k = softmax((a_k + gumbel_k)/tau)   [Eq. gamma_map, relaxed]
    Hard:  z_k = one-hot argmax(a_k + gumbel_k), ties to the lowest index
           [Eq. gamma_map, Gamma].
    """
    M, Pn, _ = dims(P)
    N = theta.shape[0]
    th = theta.reshape(N, P["H"], Pn)
    a = th[:, :, :M]
    if gumbel is not None:
        a = a + torch.as_tensor(gumbel, dtype=theta.dtype)
    if hard:
        z = torch.nn.functional.one_hot(torch.argmax(a, dim=-1), M).to(theta.dtype)
    else:
        z = torch.softmax(a / P["tau"], dim=-1)
    offset = P["offset_max"] * torch.tanh(th[:, :, M])
    dist = P["dist_max"] * torch.sigmoid(th[:, :, M + 1])
    return z, offset, dist


# ----------------------------------------------------------------------------
# Contact and friction forces (Sec. III-B: penalty contacts, semi-implicit Euler)
# ----------------------------------------------------------------------------
def _square_query(px, py, bx, by, cphi, sphi, hs):
    """Local coordinates of point p in the square's frame and q = |p_l| - hs."""
    dx, dy = px - bx, py - by
    lx = cphi * dx + sphi * dy
    ly = -sphi * dx + cphi * dy
    return lx, ly, lx.abs() - hs, ly.abs() - hs


def _sign(x):
    return torch.where(x >= 0, torch.ones_like(x), -torch.ones_like(x))


def square_sd_normal(px, py, bx, by, phi, hs):
    """Signed distance from point p to a square (centre b, yaw phi, half side
    hs) and the unit normal (world frame) pointing from the square towards p.

    Outside: sd = |max(q, 0)| with q = |p_l| - hs, normal along the clamped
    offset.  Inside or on the boundary: sd = max(q_x, q_y) <= 0, normal the
    face axis of the larger q (ties to x) with the sign of p_l (sign(0) = +1).
    """
    c, s = torch.cos(phi), torch.sin(phi)
    lx, ly, qx, qy = _square_query(px, py, bx, by, c, s, hs)
    sx, sy = _sign(lx), _sign(ly)
    outside = (qx > 0) | (qy > 0)
    mx, my = qx.clamp(min=0.0), qy.clamp(min=0.0)
    # length of the clamped offset; 1 where it is not used keeps the tape finite
    ln = torch.sqrt(torch.where(outside, mx * mx + my * my, torch.ones_like(mx)))
    sd = torch.where(outside, ln, torch.maximum(qx, qy))
    x_axis = qx >= qy
    nlx = torch.where(outside, sx * mx / ln, torch.where(x_axis, sx, torch.zeros_like(sx)))
    nly = torch.where(outside, sy * my / ln, torch.where(x_axis, torch.zeros_like(sy), sy))
    return sd, c * nlx - s * nly, s * nlx + c * nly


def _penalty_force(delta, nx, ny, wx, wy, P):
    """Penalty contact along normal n with relative velocity w.

    Returns f_n = max(0, k*delta - c*(w.n)) where delta > 0 (else 0), the
    smoothed Coulomb factor gt = mu_c*f_n/sqrt(|w_t|^2 + eps_t^2) and the
    tangential relative velocity w_t = w - (w.n) n."""
    vn = wx * nx + wy * ny
    fn = torch.where(delta > 0, (P["k_contact"] * delta - P["c_contact"] * vn).clamp(min=0.0),
                     torch.zeros_like(delta))
    tx, ty = wx - vn * nx, wy - vn * ny
    gt = P["mu_c"] * fn / torch.sqrt(tx * tx + ty * ty + P["eps_t"] ** 2)
    return fn, gt, tx, ty


def disk_box_force(px, py, vpx, vpy, bx, by, phi, vx, vy, om, P):
    """Force (Fx, Fy) and torque on a square block from a kinematic disk pusher.

    All arguments broadcast.  The pusher disk (radius r, centre p, velocity
    v_p) is in contact when delta = r - sd > 0.  With n the normal from the
    block to the pusher, x_c = p - r*n the contact point, w = v_p - (velocity
    of the block at x_c) and v_n = w.n: f_n = max(0, k*delta - c*v_n); the
    block receives -f_n*n plus mu_c*f_n*w_t/sqrt(|w_t|^2 + eps_t^2).
    """
    hs, r = P["half_size"], P["pusher_r"]
    sd, nx, ny = square_sd_normal(px, py, bx, by, phi, hs)
    delta = r - sd
    cx, cy = px - r * nx, py - r * ny
    rx, ry = cx - bx, cy - by
    wx = vpx - (vx - om * ry)
    wy = vpy - (vy + om * rx)
    fn, gt, tx, ty = _penalty_force(delta, nx, ny, wx, wy, P)
    fx = -fn * nx + gt * tx
    fy = -fn * ny + gt * ty
    return fx, fy, rx * fy - ry * fx


def corner_box_force(kx, ky, kvx, kvy, bx, by, phi, vx, vy, om, P):
    """Force on the body owning corner point k (position, velocity) from square B.

    The corner penetrates B when its signed distance sd to B is negative
    (delta = -sd > 0); the normal n is B's outward face normal (axis of the
    larger q, ties to x).  With w the corner's velocity relative to B's
    material point under it and v_n = w.n, the corner's body receives
    f_n*n - mu_c*f_n*w_t/sqrt(|w_t|^2 + eps_t^2), f_n = max(0, k*delta - c*v_n);
    B receives the opposite force at the same point.
    """
    hs = P["half_size"]
    sd, nx, ny = square_sd_normal(kx, ky, bx, by, phi, hs)
    delta = -sd
    rx, ry = kx - bx, ky - by
    wx = kvx - (vx - om * ry)
    wy = kvy - (vy + om * rx)
    fn, gt, tx, ty = _penalty_force(delta, nx, ny, wx, wy, P)
    return fn * nx - gt * tx, fn * ny - gt * ty


def ground_friction(vx, vy, om, P):
    """Smoothed Coulomb ground friction: force and torque on a sliding square."""
    w = P["mu"] * P["mass"] * P["g"]
    sv = torch.sqrt(vx * vx + vy * vy + P["eps_v"] ** 2)
    so = torch.sqrt(om * om + P["eps_w"] ** 2)
    return -w * vx / sv, -w * vy / sv, -w * r_eff(P) * om / so


CORNERS = np.array([[1.0, 1.0], [-1.0, 1.0], [-1.0, -1.0], [1.0, -1.0]])


def substep(q, v, pushers, P):
    """One semi-implicit Euler step of all blocks.

    q, v: (N, nb, 3) poses (x, y, phi) and velocities (vx, vy, omega).
    pushers: None or (px, py, vpx, vpy, w), each (N, M): centres, velocities
    and relaxed weights of the virtual pushers during this substep.
    """
    nb = q.shape[1]
    bx, by, phi = q[..., 0], q[..., 1], q[..., 2]
    vx, vy, om = v[..., 0], v[..., 1], v[..., 2]
    Fx, Fy, Tq = ground_friction(vx, vy, om, P)
    if pushers is not None:
        px, py, vpx, vpy, w = pushers
        fx, fy, tq = disk_box_force(px[:, :, None], py[:, :, None], vpx[:, :, None],
                                    vpy[:, :, None], bx[:, None, :], by[:, None, :],
                                    phi[:, None, :], vx[:, None, :], vy[:, None, :],
                                    om[:, None, :], P)
        Fx = Fx + (w[:, :, None] * fx).sum(1)
        Fy = Fy + (w[:, :, None] * fy).sum(1)
        Tq = Tq + (w[:, :, None] * tq).sum(1)
    hs = P["half_size"]
    Fx, Fy, Tq = list(Fx.unbind(1)), list(Fy.unbind(1)), list(Tq.unbind(1))
    for A in range(nb):
        for B in range(A + 1, nb):
            for own, oth in ((A, B), (B, A)):
                co, so_ = torch.cos(phi[:, own]), torch.sin(phi[:, own])
                for ex, ey in CORNERS:
                    lx_, ly_ = ex * hs, ey * hs
                    kx = bx[:, own] + co * lx_ - so_ * ly_
                    ky = by[:, own] + so_ * lx_ + co * ly_
                    rox, roy = kx - bx[:, own], ky - by[:, own]
                    kvx = vx[:, own] - om[:, own] * roy
                    kvy = vy[:, own] + om[:, own] * rox
                    fx, fy = corner_box_force(kx, ky, kvx, kvy, bx[:, oth], by[:, oth],
                                              phi[:, oth], vx[:, oth], vy[:, oth],
                                              om[:, oth], P)
                    rtx, rty = kx - bx[:, oth], ky - by[:, oth]
                    Fx[own] = Fx[own] + fx
                    Fy[own] = Fy[own] + fy
                    Tq[own] = Tq[own] + rox * fy - roy * fx
                    Fx[oth] = Fx[oth] - fx
                    Fy[oth] = Fy[oth] - fy
                    Tq[oth] = Tq[oth] - (rtx * fy - rty * fx)
    Fx, Fy, Tq = torch.stack(Fx, 1), torch.stack(Fy, 1), torch.stack(Tq, 1)
    dt, m = P["dt"], P["mass"]
    nvx = vx + dt * Fx / m
    nvy = vy + dt * Fy / m
    nom = om + dt * Tq / inertia(P)
    nq = torch.stack([bx + dt * nvx, by + dt * nvy, phi + dt * nom], -1)
    nv = torch.stack([nvx, nvy, nom], -1)
    return nq, nv


def pusher_geometry(q, offset_k, dist_k, P):
    """Start centres and per-substep displacement of the M virtual pushers.

    Pusher c = (object o = c//4, side s = c%4) starts touching side s of block
    o at tangential offset `offset_k` and moves dist_k along the inward normal
    -R(phi_o) n_s.  Returns (sx, sy, ux, uy), each (N, M): start centre and
    unit direction.
    """
    nb = q.shape[1]
    hs, r = P["half_size"], P["pusher_r"]
    n = torch.as_tensor(np.tile(SIDE_NORMALS, (nb, 1)), dtype=q.dtype)        # (M, 2)
    t = torch.stack([-n[:, 1], n[:, 0]], -1)
    obj = torch.as_tensor(np.repeat(np.arange(nb), 4))
    po = q[:, obj, :]                                                        # (N, M, 3)
    c, s = torch.cos(po[..., 2]), torch.sin(po[..., 2])
    lx = n[:, 0] * (hs + r) + t[:, 0] * offset_k[:, None]
    ly = n[:, 1] * (hs + r) + t[:, 1] * offset_k[:, None]
    sx = po[..., 0] + c * lx - s * ly
    sy = po[..., 1] + s * lx + c * ly
    ux = -(c * n[:, 0] - s * n[:, 1])
    uy = -(s * n[:, 0] + c * n[:, 1])
    return sx, sy, ux, uy


def simulate(theta, P, init_poses, gumbel=None, hard=False, record=False):
    """Roll all particles' relaxed plans through H*T substeps from rest at
    `init_poses` ((nb, 3) shared, or (N, nb, 3) per particle).

    Returns (q, v, z, offset, dist, traj) with traj (N, H*T+1, nb, 6) the state
    before every substep and after the last one when `record` is set.
    """
    N = theta.shape[0]
    dt_ = theta.dtype
    H, T = P["H"], P["T"]
    z, offset, dist = relax(theta, P, gumbel, hard)
    nb = P["n_blocks"]
    q0 = torch.as_tensor(np.asarray(init_poses, dtype=np.float64), dtype=dt_)
    # one start pose set for all particles (nb, 3), or one per particle (N, nb, 3)
    q = q0.expand(N, nb, 3) if q0.dim() == 3 else q0[None].expand(N, nb, 3)
    v = torch.zeros(N, nb, 3, dtype=dt_)
    traj = []
    for k in range(H):
        sx, sy, ux, uy = pusher_geometry(q, offset[:, k], dist[:, k], P)
        step = dist[:, k, None] / T                     # distance per substep
        for j in range(T):
            if record:
                traj.append(torch.cat([q, v], -1))
            pushers = (sx + (j + 1) * step * ux, sy + (j + 1) * step * uy,
                       ux * step / P["dt"], uy * step / P["dt"], z[:, k])
            q, v = substep(q, v, pushers, P)
    if record:
        traj.append(torch.cat([q, v], -1))
        traj = torch.stack(traj, 1)
    return q, v, z, offset, dist, (traj if record else None)


def wrap(e):
    return torch.atan2(torch.sin(e), torch.cos(e))


def cost(q, dist, goal_poses, P):
    """C = sum_b |p_b - g_b|^2 + w_yaw wrap(phi_b - phi_gb)^2 + w_push sum_k dist_k^2.

    -C is log p(O=1|theta) up to a constant [Eq. neglog_likelihood]."""
    g = torch.as_tensor(np.asarray(goal_poses, dtype=np.float64), dtype=q.dtype)
    e = q - g[None]
    return ((e[..., 0] ** 2 + e[..., 1] ** 2 + P["w_yaw"] * wrap(e[..., 2]) ** 2).sum(1)
            + P["w_push"] * (dist ** 2).sum(1))


def rollout(theta, P, init_poses, goal_poses, gumbel=None, hard=False, record=False,
            dtype=torch.float64):
    """Cost and final state (N, nb, 6) of each particle; no gradient."""
    th = torch.as_tensor(np.asarray(theta), dtype=dtype)
    with torch.no_grad():
        q, v, _, _, dist, traj = simulate(th, P, init_poses, gumbel, hard, record)
        c = cost(q, dist, goal_poses, P)
    out = (c.numpy(), torch.cat([q, v], -1).numpy())
    return out + ((traj.numpy(),) if record else ())


def rollout_grad(theta, P, init_poses, goal_poses, gumbel=None, dtype=torch.float64):
    """Cost and grad log rho = -dC/dtheta per particle (reverse mode, Sec. III-B)."""
    th = torch.tensor(np.asarray(theta), dtype=dtype, requires_grad=True)
    q, v, _, _, dist, _ = simulate(th, P, init_poses, gumbel, False, False)
    c = cost(q, dist, goal_poses, P)
    (g,) = torch.autograd.grad(c.sum(), th)
    return c.detach().numpy(), (-g).numpy()


# ----------------------------------------------------------------------------
# SVGD [Eq. svgd], bandwidth by the median heuristic, Adam, Algorithm 1
# ----------------------------------------------------------------------------
def pairwise_sq_dists(theta, chunk=256):
    """d2[i, j] = sum_d (theta[i,d] - theta[j,d])^2, written out directly."""
    th = np.asarray(theta, dtype=np.float64)
    n = th.shape[0]
    d2 = np.empty((n, n))
    for i0 in range(0, n, chunk):
        diff = th[i0:i0 + chunk, None, :] - th[None, :, :]
        d2[i0:i0 + chunk] = (diff * diff).sum(-1)
    return d2


def median_bandwidth(theta):
    """h = med / ln(N+1); med = lower median of {d2_ij : i < j}."""
    n = np.asarray(theta).shape[0]
    if n < 2:
        return 1.0
    d2 = pairwise_sq_dists(theta)
    vals = np.sort(d2[np.triu_indices(n, 1)])
    h = vals[(vals.size - 1) // 2] / math.log(n + 1.0)
    return h if h >= 1e-12 else 1.0


def stein_direction(theta, grad_logp, h, chunk=128, weights=None):
    """phi_i = sum_j (w_j / w) [ k_ji grad log p(theta_j) + grad_{theta_j} k_ji ]
    with k(a, b) = exp(-|a - b|^2 / h), so grad_{theta_j} k_ji =
    (2/h) (theta_i - theta_j) k_ji  [Eq. svgd, terms (A) and (B); Eq. dsvgd
    with its weights w_j, w = sum_j w_j].  weights=None: w_j = 1, so the
    factor is 1/N."""
    th = np.asarray(theta, dtype=np.float64)
    g = np.asarray(grad_logp, dtype=np.float64)
    n = th.shape[0]
    wn = (np.full(n, 1.0 / n) if weights is None
          else np.asarray(weights, dtype=np.float64) / np.sum(weights))
    phi = np.empty_like(th)
    for i0 in range(0, n, chunk):
        diff = th[i0:i0 + chunk, None, :] - th[None, :, :]        # theta_i - theta_j
        k = np.exp(-(diff * diff).sum(-1) / h) * wn[None, :]     # (c, N), weighted
        attract = k @ g
        repulse = (2.0 / h) * (k[:, :, None] * diff).sum(1)
        phi[i0:i0 + chunk] = attract + repulse
    return phi


def structured_parts(theta, P):
    """Per-action components of the structured kernel: the continuous push
    parameters c_k = (u_k, v_k) (N, H, 2) and the choice probabilities
    s_k = softmax(a_k) (N, H, M)."""
    M, Pn, _ = dims(P)
    th = torch.as_tensor(np.asarray(theta), dtype=torch.float64).reshape(-1, P["H"], Pn)
    return th[..., M:], torch.softmax(th[..., :M], dim=-1)


def structured_bandwidths(theta, P):
    """(h_c, h_z): the median heuristic of each component on its per-action
    mean squared distance, (1/H) sum_k |x_ik - x_jk|^2, lower median over
    i < j, divided by ln(N+1): the plain bandwidth of the concatenated
    component divided by H (so 1/H in the plain rule's degenerate cases)."""
    c, z = structured_parts(theta, P)
    n = c.shape[0]
    return tuple(median_bandwidth(x.reshape(n, -1).numpy()) / P["H"] for x in (c, z))


def structured_kernel(theta_a, theta_b, P, h_c, h_z):
    """App. D.3's additive kernel restated for this parameterisation:
    K(a, b) = (1/2H) sum_k [exp(-|c_k(a) - c_k(b)|^2 / h_c)
                            + exp(-|softmax(a_k) - softmax(b_k)|^2 / h_z)]
    (torch, differentiable; K(a, a) = 1)."""
    ca, za = structured_parts_t(theta_a, P)
    cb, zb = structured_parts_t(theta_b, P)
    kc = torch.exp(-((ca - cb) ** 2).sum(-1) / h_c)
    kz = torch.exp(-((za - zb) ** 2).sum(-1) / h_z)
    return (kc + kz).sum(-1) / (2 * P["H"])


def structured_parts_t(theta, P):
    M, Pn, _ = dims(P)
    th = theta.reshape(*theta.shape[:-1], P["H"], Pn)
    return th[..., M:], torch.softmax(th[..., :M], dim=-1)


def stein_direction_structured(theta, grad_logp, P, weights=None):
    """phi_i = sum_j (w_j / w) [K(theta_j, theta_i) grad log p(theta_j)
    + grad_{theta_j} K(theta_j, theta_i)] with the structured kernel [Eq. svgd /
    Eq. dsvgd, kernel of App. D.3]; the kernel gradient by reverse mode."""
    th = torch.as_tensor(np.asarray(theta), dtype=torch.float64)
    g = torch.as_tensor(np.asarray(grad_logp), dtype=torch.float64)
    n = th.shape[0]
    h_c, h_z = structured_bandwidths(th.numpy(), P)
    wn = (torch.full((n,), 1.0 / n, dtype=torch.float64) if weights is None
          else torch.as_tensor(np.asarray(weights, dtype=np.float64) / np.sum(weights)))
    tj = th.clone().requires_grad_(True)
    phi = torch.zeros_like(th)
    for i in range(n):
        k = structured_kernel(tj, th[i].expand_as(th), P, h_c, h_z)   # K(theta_j, theta_i), (n,)
        (gk,) = torch.autograd.grad((k * wn).sum(), tj)
        phi[i] = ((k.detach() * wn)[:, None] * g).sum(0) + gk.sum(0)
    return phi.numpy()


def dsvgd_weights(cost_relaxed, cost_hard):
    """Importance weights of Eq. dsvgd, w_j = p~*(Gamma~(theta_j)) / p*(Gamma(theta_j)),
    with p* proportional to exp(-C) [Eq. neglog_likelihood]: the relaxed plan's
    cost against the hard plan's (the same Gumbel draws), w_j = exp(C_j - C~_j).
    Returned divided by their sum (the update uses w_j / w only)."""
    d = np.asarray(cost_hard, dtype=np.float64) - np.asarray(cost_relaxed, dtype=np.float64)
    w = np.exp(d - d.max())
    return w / w.sum()


ADAM_B1, ADAM_B2, ADAM_EPS = 0.9, 0.999, 1e-8


def adam_update(theta, m, v, grad, step, lr):
    """One Adam step (Kingma & Ba 2015, bias-corrected) minimising along `grad`."""
    m = ADAM_B1 * m + (1 - ADAM_B1) * grad
    v = ADAM_B2 * v + (1 - ADAM_B2) * grad * grad
    mh = m / (1 - ADAM_B1 ** step)
    vh = v / (1 - ADAM_B2 ** step)
    return theta - lr * mh / (np.sqrt(vh) + ADAM_EPS), m, v


def svgd_step(theta, grad_logp, m, v, step, lr, sgd_phase=False):
    """Algorithm 1, one update: SVGD phase moves along the Stein direction phi,
    SGD phase along grad log rho; Adam on -direction.  Returns
    (theta, m, v, h, phi)."""
    th = np.asarray(theta, dtype=np.float64)
    if sgd_phase:
        h, phi = 1.0, np.asarray(grad_logp, dtype=np.float64)
    else:
        h = median_bandwidth(th)
        phi = stein_direction(th, grad_logp, h)
    th, m, v = adam_update(th, np.asarray(m, dtype=np.float64),
                           np.asarray(v, dtype=np.float64), -phi, step, lr)
    return th, m, v, h, phi


def plan_codes(theta, P):
    """Discrete plan Gamma(theta): argmax choice per action, ties lowest."""
    M, Pn, _ = dims(P)
    th = np.asarray(theta).reshape(-1, P["H"], Pn)[:, :, :M]
    return np.argmax(th, axis=-1)


def topk_plans(costs, codes, k):
    """Rank by (cost, index) and keep the first k distinct discrete plans.

    Returns the particle index of each kept plan, -1 padded."""
    order = np.lexsort((np.arange(len(costs)), costs))
    seen, out = [], []
    for i in order:
        key = tuple(codes[i])
        if key not in seen:
            seen.append(key)
            out.append(int(i))
            if len(out) == k:
                break
    return out + [-1] * (k - len(out))


def solve(P, init_poses, goal_poses, N, svgd_iters, sgd_iters, seed, lr, k=3,
          theta0=None, dtype=torch.float64):
    """STAMP, Algorithm 1: SVGD iterations then SGD iterations, then the hard
    evaluation of every particle and the distinct-plan top-k.

    Returns dict(theta, cost_hard, topk, min_cost per iteration, h per iteration).
    """
    M, _, D = dims(P)
    th = init_theta(seed, N, D) if theta0 is None else np.asarray(theta0, dtype=np.float64)
    m = np.zeros_like(th)
    v = np.zeros_like(th)
    mins, hs = [], []
    for it in range(svgd_iters + sgd_iters):
        gum = gumbel_noise(seed, it, N, P["H"], M)
        c, g = rollout_grad(th, P, init_poses, goal_poses, gum, dtype=dtype)
        mins.append(float(np.min(c)))
        th, m, v, h, _ = svgd_step(th, g, m, v, it + 1, lr, sgd_phase=it >= svgd_iters)
        hs.append(h)
    ch, _ = rollout(th, P, init_poses, goal_poses, None, hard=True, dtype=dtype)
    return dict(theta=th, cost_hard=ch, topk=topk_plans(ch, plan_codes(th, P), k),
                min_cost=np.array(mins), h=np.array(hs))
