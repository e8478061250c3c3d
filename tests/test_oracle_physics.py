"""Pins for the oracle's planar rigid-body pushing simulator (Sec. III-B).

Each pin is independent of the oracle's own formulas:
* smoothed Coulomb sliding/spinning stops at the closed-form distance/angle,
  with O(dt) convergence under dt-halving, and tends to v0^2/(2 mu g);
* the square signed distance agrees with the exact distance to its four
  edge segments;
* penalty contact forces are minus the gradient of the spring energy
  (k/2) delta^2 (finite differences of the brute-force distance), and the
  torque satisfies virtual work in the block's yaw;
* with frictionless ground, block-block contact conserves linear and angular
  momentum (equal and opposite forces at one point, semi-implicit Euler);
* pushers start touching their side and move along its inward normal;
* the autograd gradient of the cost matches central finite differences.
"""
import math

import numpy as np
import pytest
import torch

from oracle import stamp_oracle as O
from paper_2310_01775_gb300 import workloads as W


def _slide(P, v0, w0, dt, t_end):
    P = dict(P, dt=dt)
    q = torch.zeros(1, 1, 3, dtype=torch.float64)
    v = torch.tensor([[[v0, 0.0, w0]]], dtype=torch.float64)
    for _ in range(int(round(t_end / dt))):
        q, v = O.substep(q, v, None, P)
    return float(q[0, 0, 0]), float(q[0, 0, 2])


def _smoothed_stop(v0, eps, decel):
    """Distance covered under dv/dt = -decel * v / sqrt(v^2 + eps^2) from v0:
    the integral of sqrt(v^2+eps^2)/decel dv over [0, v0]."""
    s = math.sqrt(v0 * v0 + eps * eps)
    return (v0 / 2 * s + eps * eps / 2 * math.log((v0 + s) / eps)) / decel


def test_sliding_block_closed_form_and_dt_convergence():
    P = W.params("pusher1_h2")
    v0 = 1.0
    exact = _smoothed_stop(v0, P["eps_v"], P["mu"] * P["g"])
    d = [_slide(P, v0, 0.0, dt, 2.0)[0] for dt in (0.01, 0.005, 0.0025)]
    errs = [abs(x - exact) for x in d]
    # first order: halving dt halves the error, and Richardson extrapolation
    # (2 d(dt/2) - d(dt)) removes the leading term
    assert 1.7 < errs[0] / errs[1] < 2.3 and 1.7 < errs[1] / errs[2] < 2.3
    assert abs(2 * d[2] - d[1] - exact) < 1e-4 * exact


def test_sliding_block_tends_to_coulomb_stop():
    """As the smoothing vanishes the distance tends to v0^2 / (2 mu g)."""
    P = W.params("pusher1_h2", eps_v=1e-3)
    x, _ = _slide(P, 1.0, 0.0, 1e-4, 1.0)
    assert abs(x - 1.0 / (2 * P["mu"] * P["g"])) < 0.01 * x


def test_spinning_block_closed_form():
    P = W.params("pusher1_h2")
    w0 = 10.0
    decel = P["mu"] * P["mass"] * P["g"] * O.r_eff(P) / O.inertia(P)
    exact = _smoothed_stop(w0, P["eps_w"], decel)
    d = [_slide(P, 0.0, w0, dt, 1.0)[1] for dt in (0.004, 0.002, 0.001)]
    errs = [abs(x - exact) for x in d]
    assert 1.7 < errs[0] / errs[1] < 2.3 and 1.7 < errs[1] / errs[2] < 2.3
    assert abs(2 * d[2] - d[1] - exact) < 1e-4 * exact


def test_r_eff_is_mean_distance_of_square():
    """Monte-Carlo mean |x| over a uniform 0.1 m square."""
    P = W.params("pusher1_h2")
    a = 2 * P["half_size"]
    pts = np.random.default_rng(0).uniform(-a / 2, a / 2, size=(2_000_000, 2))
    assert abs(np.sqrt((pts ** 2).sum(1)).mean() - O.r_eff(P)) < 2e-5


def _seg_dist(p, a, b):
    ab = b - a
    t = np.clip(((p - a) * ab).sum(-1) / (ab * ab).sum(-1), 0, 1)
    c = a + t[..., None] * ab
    return np.sqrt(((p - c) ** 2).sum(-1))


def brute_sd(px, py, bx, by, phi, hs):
    """Exact signed distance via the four edge segments (negative inside)."""
    c, s = math.cos(phi), math.sin(phi)
    loc = np.array([[hs, hs], [-hs, hs], [-hs, -hs], [hs, -hs]])
    cor = np.stack([bx + c * loc[:, 0] - s * loc[:, 1], by + s * loc[:, 0] + c * loc[:, 1]], -1)
    p = np.array([px, py])
    d = min(_seg_dist(p, cor[i], cor[(i + 1) % 4]) for i in range(4))
    lx = c * (px - bx) + s * (py - by)
    ly = -s * (px - bx) + c * (py - by)
    inside = abs(lx) < hs and abs(ly) < hs
    return -d if inside else d


def test_signed_distance_matches_edge_segments():
    rng = np.random.default_rng(1)
    hs = 0.05
    for _ in range(400):
        bx, by, phi = rng.uniform(-0.3, 0.3), rng.uniform(-0.3, 0.3), rng.uniform(-3, 3)
        px, py = bx + rng.uniform(-0.12, 0.12), by + rng.uniform(-0.12, 0.12)
        t = lambda x: torch.tensor(x, dtype=torch.float64)
        sd, nx, ny = O.square_sd_normal(t(px), t(py), t(bx), t(by), t(phi), hs)
        assert abs(float(sd) - brute_sd(px, py, bx, by, phi, hs)) < 1e-12
        # the normal is the gradient of the brute-force distance
        e = 1e-7
        gx = (brute_sd(px + e, py, bx, by, phi, hs) - brute_sd(px - e, py, bx, by, phi, hs)) / (2 * e)
        gy = (brute_sd(px, py + e, bx, by, phi, hs) - brute_sd(px, py - e, bx, by, phi, hs)) / (2 * e)
        assert abs(float(nx) - gx) < 1e-5 and abs(float(ny) - gy) < 1e-5


def _energy(px, py, bx, by, phi, P):
    d = P["pusher_r"] - brute_sd(px, py, bx, by, phi, P["half_size"])
    return 0.5 * P["k_contact"] * max(d, 0.0) ** 2


def test_contact_force_is_spring_energy_gradient_and_virtual_work():
    P = W.params("pusher1_h2", c_contact=0.0, mu_c=0.0)
    rng = np.random.default_rng(2)
    t = lambda x: torch.tensor(x, dtype=torch.float64)
    z = t(0.0)
    e = 1e-7
    checked = 0
    for _ in range(300):
        bx, by, phi = rng.uniform(-0.2, 0.2), rng.uniform(-0.2, 0.2), rng.uniform(-3, 3)
        px, py = bx + rng.uniform(-0.065, 0.065), by + rng.uniform(-0.065, 0.065)
        if _energy(px, py, bx, by, phi, P) == 0.0:
            continue
        fx, fy, tq = O.disk_box_force(t(px), t(py), z, z, t(bx), t(by), t(phi), z, z, z, P)
        # block force = -dE/d(block position); torque = -dE/d(block yaw)
        dEx = (_energy(px, py, bx + e, by, phi, P) - _energy(px, py, bx - e, by, phi, P)) / (2 * e)
        dEy = (_energy(px, py, bx, by + e, phi, P) - _energy(px, py, bx, by - e, phi, P)) / (2 * e)
        dEp = (_energy(px, py, bx, by, phi + e, P) - _energy(px, py, bx, by, phi - e, P)) / (2 * e)
        scale = max(1.0, abs(float(fx)), abs(float(fy)))
        assert abs(float(fx) + dEx) < 1e-4 * scale
        assert abs(float(fy) + dEy) < 1e-4 * scale
        assert abs(float(tq) + dEp) < 1e-4 * scale
        checked += 1
    assert checked > 50


def _momenta(q, v, P):
    m, I = P["mass"], O.inertia(P)
    lin = m * v[..., :2].sum(1)
    ang = (I * v[..., 2] + m * (q[..., 0] * v[..., 1] - q[..., 1] * v[..., 0])).sum(1)
    return lin, ang


@pytest.mark.parametrize("nb", [2, 3])
def test_block_contact_conserves_momentum_without_ground_friction(nb):
    P = W.params("pusher3_h6", mu=0.0, n_blocks=nb)
    q = torch.tensor([[[0.0, 0.0, 0.1], [0.092, 0.03, 0.7], [-0.05, 0.093, -0.4]][:nb]],
                     dtype=torch.float64)
    v = torch.tensor([[[0.3, 0.1, 2.0], [-0.4, 0.05, -1.0], [0.1, -0.5, 3.0]][:nb]],
                     dtype=torch.float64)
    l0, a0 = _momenta(q, v, P)
    touched = False
    for _ in range(200):
        nq, nv = O.substep(q, v, None, P)
        touched |= not torch.allclose(nv - v, torch.zeros_like(v))
        q, v = nq, nv
    l1, a1 = _momenta(q, v, P)
    assert touched
    assert torch.allclose(l0, l1, rtol=0, atol=1e-12)
    assert torch.allclose(a0, a1, rtol=0, atol=1e-12)


def test_pusher_starts_touching_and_moves_inward():
    P = W.params("pusher3_h6")
    rng = np.random.default_rng(3)
    q = torch.tensor(rng.uniform(-0.4, 0.4, size=(5, 3, 3)))
    off = torch.tensor(rng.uniform(-0.05, 0.05, size=5))
    sx, sy, ux, uy = O.pusher_geometry(q, off, None, P)
    for i in range(5):
        for c in range(12):
            o, s = divmod(c, 4)
            bx, by, phi = (float(x) for x in q[i, o])
            assert abs(brute_sd(float(sx[i, c]), float(sy[i, c]), bx, by, phi, 0.05)
                       - P["pusher_r"]) < 1e-12
            # moving along u enters the block through side s
            ex = float(sx[i, c] + 0.02 * ux[i, c])
            ey = float(sy[i, c] + 0.02 * uy[i, c])
            assert abs(brute_sd(ex, ey, bx, by, phi, 0.05) - (P["pusher_r"] - 0.02)) < 1e-12
            n = O.SIDE_NORMALS[s]
            assert abs(float(ux[i, c]) + (math.cos(phi) * n[0] - math.sin(phi) * n[1])) < 1e-12


def test_cost_at_goal_is_push_penalty_only():
    P = W.params("pusher1_h2")
    goal = np.array([[0.2, -0.1, 3.0]])
    q = torch.tensor(goal + np.array([[0.0, 0.0, 2 * math.pi]]))[None]   # yaw differs by 2pi
    dist = torch.tensor([[0.1, 0.2]], dtype=torch.float64)
    assert abs(float(O.cost(q, dist, goal, P)[0]) - P["w_push"] * 0.05) < 1e-12
    q2 = torch.tensor(goal + np.array([[0.3, 0.4, 0.5]]))[None]
    assert abs(float(O.cost(q2, dist, goal, P)[0]) - (0.25 + P["w_yaw"] * 0.25 + P["w_push"] * 0.05)) < 1e-12


def test_autograd_gradient_matches_central_differences():
    """Sec. III-B: the reverse-mode gradient is the derivative of the rollout
    (checked on particles where two FD step sizes agree, i.e. away from
    contact-onset kinks)."""
    P = W.params("pusher1_h2")
    init, goal = W.scene(P, 0)
    M, _, D = O.dims(P)
    n = 6
    th = O.init_theta(21, n, D)
    gum = O.gumbel_noise(21, 0, n, P["H"], M)
    _, g = O.rollout_grad(th, P, init, goal, gum)

    def fd(h):
        out = np.zeros_like(th)
        for d in range(D):
            e = np.zeros_like(th)
            e[:, d] = h
            cp, _ = O.rollout(th + e, P, init, goal, gum)
            cm, _ = O.rollout(th - e, P, init, goal, gum)
            out[:, d] = -(cp - cm) / (2 * h)
        return out

    f1, f2 = fd(1e-5), fd(2e-6)
    smooth = np.abs(f1 - f2).max(1) < 1e-6 * np.maximum(np.abs(f1).max(1), 1e-8) * 10
    assert smooth.sum() >= 2
    for i in np.where(smooth)[0]:
        assert np.abs(g[i] - f1[i]).max() <= 1e-5 * np.abs(f1[i]).max()
