"""Pins for the structure the time-parallel reverse sweep relies on, checked
on the FP64 oracle's own simulator (oracle/stamp_oracle.py).

The sweep (csrc/adjoint_time.cu) rewrites the reverse pass of one
semi-implicit Euler substep of a block as
    av1 = (a_vx + dt a_x, a_vy + dt a_y, a_om + dt a_ph),
    a_before = (a_x, a_y, a_ph, av1) + M^T av1,
    M = diag(dt/m, dt/m, dt/I) dF/ds,
with F = (F_x, F_y, T) the block's total force and torque (ground friction
plus the relaxed-weighted pusher contacts) and s = (x, y, ph, vx, vy, om).
It also moves the pushers with the block's start position, which needs the
contact force to depend on the pusher and the block only through their
relative position and velocity.  These tests check both on the oracle:
the substep's reverse-mode derivative (torch autograd through
oracle.substep) against the rewrite with dF/ds taken from the oracle's force
functions alone, and the invariance of oracle.disk_box_force.  A substep
with explicit instead of semi-implicit Euler, a force assembled with a
wrong weight or sign, or a contact force depending on absolute positions
fails them.
"""
import numpy as np
import torch

from oracle import stamp_oracle as O
from paper_2310_01775_gb300 import workloads as W


def _pushers(rng, n, P):
    """Four virtual pushers per particle around a block at the origin, most
    of them pressing into it (centre just inside the touching distance)."""
    hs, r = P["half_size"], P["pusher_r"]
    n_side = O.SIDE_NORMALS
    reach = hs + r - rng.uniform(-0.002, 0.006, size=(n, 4))       # < hs + r: contact
    tang = rng.uniform(-0.04, 0.04, size=(n, 4))
    px = n_side[:, 0] * reach - n_side[:, 1] * tang
    py = n_side[:, 1] * reach + n_side[:, 0] * tang
    vpx = -n_side[:, 0] * rng.uniform(0.0, 0.4, size=(n, 4)) + rng.normal(0, 0.05, (n, 4))
    vpy = -n_side[:, 1] * rng.uniform(0.0, 0.4, size=(n, 4)) + rng.normal(0, 0.05, (n, 4))
    w = rng.dirichlet(np.ones(4), size=n)
    return [torch.tensor(x, dtype=torch.float64) for x in (px, py, vpx, vpy, w)]


def _state(rng, n):
    q = torch.tensor(np.stack([rng.normal(0, 0.003, n), rng.normal(0, 0.003, n),
                               rng.normal(0, 0.2, n)], -1)[:, None, :], dtype=torch.float64)
    v = torch.tensor(np.stack([rng.normal(0, 0.2, n), rng.normal(0, 0.2, n),
                               rng.normal(0, 1.0, n)], -1)[:, None, :], dtype=torch.float64)
    return q, v


def _total_force(s, pushers, P):
    """(F_x, F_y, T) on the block for states s (n, 6), from the oracle's
    force functions: ground friction plus the weighted pusher contacts."""
    px, py, vpx, vpy, w = pushers
    bx, by, ph, vx, vy, om = s.unbind(1)
    Fx, Fy, Tq = O.ground_friction(vx, vy, om, P)
    fx, fy, tq = O.disk_box_force(px, py, vpx, vpy, bx[:, None], by[:, None], ph[:, None],
                                  vx[:, None], vy[:, None], om[:, None], P)
    return torch.stack([Fx + (w * fx).sum(1), Fy + (w * fy).sum(1), Tq + (w * tq).sum(1)], 1)


def test_substep_adjoint_is_the_linear_recurrence():
    P = W.params("pusher1_h4")
    rng = np.random.default_rng(3)
    n = 64
    pushers = _pushers(rng, n, P)
    q, v = _state(rng, n)
    s = torch.cat([q[:, 0], v[:, 0]], 1).requires_grad_(True)
    # reverse mode through the oracle's substep
    nq, nv = O.substep(s[:, None, :3], s[:, None, 3:], pushers, P)
    out = torch.cat([nq[:, 0], nv[:, 0]], 1)
    a = torch.tensor(rng.normal(size=(n, 6)), dtype=torch.float64)
    (want,) = torch.autograd.grad((out * a).sum(), s)
    # the rewrite: dF/ds per particle from the force functions alone
    F = _total_force(s, pushers, P)
    J = torch.stack([torch.autograd.grad(F[:, m].sum(), s, retain_graph=True)[0]
                     for m in range(3)], 1)                                   # (n, 3, 6)
    dt = P["dt"]
    cm = torch.tensor([dt / P["mass"], dt / P["mass"], dt / O.inertia(P)], dtype=torch.float64)
    M = cm[None, :, None] * J
    av1 = a[:, 3:] + dt * a[:, :3]
    got = torch.cat([a[:, :3], av1], 1) + torch.einsum("nms,nm->ns", M, av1)
    assert torch.allclose(got, want, rtol=1e-12, atol=1e-12 * want.abs().max())
    # the cases are not degenerate: contacts press and the Jacobian is large
    assert (J[:, :2, :2].abs().amax((1, 2)) > 100.0).float().mean() > 0.5


def test_contact_force_moves_with_pusher_and_block():
    """Translating pusher and block together, or giving both the same
    velocity, leaves the contact force and torque unchanged:
    d/dp = -d/db and d/dv_p = -d/dv_b."""
    P = W.params("pusher1_h4")
    rng = np.random.default_rng(5)
    n = 32
    px, py, vpx, vpy, _ = _pushers(rng, n, P)
    q, v = _state(rng, n)
    args = [px[:, 0], py[:, 0], vpx[:, 0], vpy[:, 0], q[:, 0, 0], q[:, 0, 1], q[:, 0, 2],
            v[:, 0, 0], v[:, 0, 1], v[:, 0, 2]]
    args = [x.clone().requires_grad_(True) for x in args]
    f = O.disk_box_force(*args, P)
    for out in f:
        g = torch.autograd.grad(out.sum(), args, retain_graph=True)
        gpx, gpy, gvpx, gvpy, gbx, gby, _, gvx, gvy, _ = g
        scale = max(float(torch.stack([x.abs().max() for x in (gpx, gpy, gvpx, gvpy)]).max()), 1e-12)
        for gp, gb in ((gpx, gbx), (gpy, gby), (gvpx, gvx), (gvpy, gvy)):
            assert torch.allclose(gp, -gb, rtol=1e-12, atol=1e-12 * scale)
    assert (f[0].abs() > 1e-3).float().mean() > 0.5   # most pushers press
