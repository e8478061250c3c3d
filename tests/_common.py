"""Shared helpers of the GPU parity tests (test infrastructure only)."""
import numpy as np
import torch

from oracle import stamp_oracle as O

TRAJ_TOL, GRAD_TOL = 1e-4, 1e-3   # the parity bar (relative, max-norm per particle)


def rel_err(a, b):
    """max|a-b| / max(max|b|, 1e-8), per leading index (one row per particle)."""
    a = np.asarray(a, dtype=np.float64).reshape(len(a), -1)
    b = np.asarray(b, dtype=np.float64).reshape(len(b), -1)
    return np.abs(a - b).max(1) / np.maximum(np.abs(b).max(1), 1e-8)


class Reference:
    """FP64 oracle results plus the float32 floor of each particle.

    The configured contact dynamics (stiffness 1e4, damping 50, dt 0.01, a
    1/600 kg m^2 block) sit near the stability edge of explicit integration,
    so some particles amplify rounding chaotically.  The oracle rerun in
    float32 measures that floor per particle; a particle is *conditioned*
    when its float32 floor is below a tenth of the bar (trajectory and
    gradient): only there is a float32 implementation with another rounding
    order expected to meet the bar.
    """

    def __init__(self, theta, P, init, goal, gumbel, C=1, need_grad=True, hard=False):
        th = np.asarray(theta, dtype=np.float64)
        self.cost, _, t64 = O.rollout(th, P, init, goal, gumbel, hard=hard, record=True)
        _, _, t32 = O.rollout(th, P, init, goal, gumbel, hard=hard, record=True,
                             dtype=torch.float32)
        self.traj = t64[:, ::C]
        self.final = t64[:, -1]
        self.floor_traj = rel_err(t32[:, ::C], self.traj)
        self.ok = rel_err(t32, t64) < TRAJ_TOL / 10
        self.grad = self.floor_grad = None
        if need_grad:
            _, self.grad = O.rollout_grad(th, P, init, goal, gumbel)
            _, g32 = O.rollout_grad(th, P, init, goal, gumbel, dtype=torch.float32)
            self.floor_grad = rel_err(g32, self.grad)
            self.ok &= self.floor_grad < GRAD_TOL / 10

    def check(self, tape, final, cost, grad=None, min_frac=0.3, min_count=3):
        """Bar on conditioned particles (at least min_count of them and a
        min_frac share); on all particles the GPU's error distribution must
        match the float32 floor's."""
        ok = self.ok
        need = min(min_count, len(ok)) if min_frac > 0 else 0
        assert ok.sum() >= need and ok.mean() >= min_frac, \
            f"only {ok.sum()} of {len(ok)} particles conditioned"
        et = rel_err(tape, self.traj)
        assert et[ok].max(initial=0) < TRAJ_TOL, et[ok].max(initial=0)
        assert rel_err(final, self.final)[ok].max(initial=0) < TRAJ_TOL
        if cost is not None:
            ec = np.abs(cost - self.cost) / np.maximum(np.abs(self.cost), 1e-8)
            assert ec[ok].max(initial=0) < TRAJ_TOL
        assert np.median(et) <= 3 * np.median(self.floor_traj) + 1e-6
        if grad is not None:
            eg = rel_err(grad, self.grad)
            assert eg[ok].max(initial=0) < GRAD_TOL, eg[ok].max(initial=0)
            assert np.median(eg) <= 3 * np.median(self.floor_grad) + 1e-6
        return ok
