"""The torch.autograd.Function over the rollout (forward = stamp_rollout_fwd,
backward = stamp_rollout_adjoint) against FP64 central finite differences of
the oracle (h = 1e-5, within 1e-2 relative) and the oracle's reverse-mode tape
(within 1e-3 relative, on particles well-conditioned at float32 rounding);
the checkpoint interval does not change the gradient."""
import numpy as np
import pytest
import torch

from oracle import stamp_oracle as O
from paper_2310_01775_gb300 import workloads as W

from _common import Reference, rel_err

pytestmark = pytest.mark.gpu
SOFT = dict(k_contact=1e3, c_contact=10.0)


def f32(P):
    return {k: (float(np.float32(v)) if isinstance(v, float) else v) for k, v in P.items()}


def setup(N, seed, **over):
    P = f32(W.params("pusher1_h2", **over))
    init, goal = W.scene(P, seed)
    init = init.astype(np.float32).astype(np.float64)
    goal = goal.astype(np.float32).astype(np.float64)
    M, _, D = O.dims(P)
    theta = O.init_theta(seed, N, D).astype(np.float32)
    return P, init, goal, M, D, theta


def gpu_grad(P, init, goal, theta, w, seed, it):
    from paper_2310_01775_gb300 import stamp as S
    from paper_2310_01775_gb300.autograd import rollout_cost
    N = theta.shape[0]
    prob = S.Problem(P, init, goal, N, torch.cuda.current_stream().cuda_stream)
    th = torch.tensor(theta, device="cuda", requires_grad=True)
    cost = rollout_cost(th, prob, seed, it)
    (torch.tensor(w, device="cuda", dtype=torch.float32) * cost).sum().backward()
    g = th.grad.cpu().numpy()
    prob.close()
    return cost.detach().cpu().numpy(), g


def test_gradient_matches_fp64_central_differences():
    seed, it, N = 3, 2, 6
    P, init, goal, M, D, theta = setup(N, seed, **SOFT)
    w = np.random.default_rng(0).uniform(0.5, 1.5, size=N)
    _, g = gpu_grad(P, init, goal, theta, w, seed, it)
    gum = O.gumbel_noise(seed, it, N, P["H"], M)
    h = 1e-5
    fd = np.zeros_like(g, dtype=np.float64)
    th = theta.astype(np.float64)
    for d in range(D):
        e = np.zeros_like(th)
        e[:, d] = h
        cp, _ = O.rollout(th + e, P, init, goal, gum)
        cm, _ = O.rollout(th - e, P, init, goal, gum)
        fd[:, d] = w * (cp - cm) / (2 * h)
    assert rel_err(g, fd).max() < 1e-2, rel_err(g, fd)


@pytest.mark.parametrize("over,min_frac", [(SOFT, 0.9), ({}, 0.3)])
def test_gradient_matches_oracle_tape(over, min_frac):
    seed, it, N = 8, 5, 40
    P, init, goal, M, D, theta = setup(N, seed, ckpt_every=1, **over)
    w = np.ones(N)
    cost, g = gpu_grad(P, init, goal, theta, w, seed, it)
    gum = O.gumbel_noise(seed, it, N, P["H"], M)
    ref = Reference(theta, P, init, goal, gum)
    ok = ref.ok
    assert ok.mean() >= min_frac
    assert rel_err(g[ok], -ref.grad[ok]).max() < 1e-3
    assert (np.abs(cost - ref.cost) / ref.cost)[ok].max() < 1e-4


def test_backward_replays_an_overwritten_tape():
    from paper_2310_01775_gb300 import stamp as S
    from paper_2310_01775_gb300.autograd import rollout_cost
    seed, N = 4, 16
    P, init, goal, M, D, theta = setup(N, seed, **SOFT)
    prob = S.Problem(P, init, goal, N, torch.cuda.current_stream().cuda_stream)
    a = torch.tensor(theta, device="cuda", requires_grad=True)
    b = torch.tensor(theta[::-1].copy(), device="cuda", requires_grad=True)
    ca = rollout_cost(a, prob, seed, 0)
    cb = rollout_cost(b, prob, seed, 1)          # overwrites the tape
    ca.sum().backward()                          # must replay a's forward
    cb.sum().backward()
    ga, gb = a.grad.clone(), b.grad.clone()
    a2 = torch.tensor(theta, device="cuda", requires_grad=True)
    rollout_cost(a2, prob, seed, 0).sum().backward()
    assert torch.equal(ga, a2.grad)
    b2 = torch.tensor(theta[::-1].copy(), device="cuda", requires_grad=True)
    rollout_cost(b2, prob, seed, 1).sum().backward()
    assert torch.equal(gb, b2.grad)
    prob.close()


def test_checkpoint_interval_does_not_change_the_gradient():
    """Segment replay recomputes the states the forward stored (same lanes per
    particle; the compiler may contract the replayed arithmetic differently),
    so every interval gives the same gradient to float32 rounding."""
    from paper_2310_01775_gb300 import stamp as S
    seed, N = 6, 33
    grads = []
    for C in (1, 5, 25, 50):
        P, init, goal, M, D, theta = setup(N, seed, ckpt_every=C, **SOFT)
        prob = S.Problem(P, init, goal, N, torch.cuda.current_stream().cuda_stream)
        prob.set_lanes(4, 4)
        th = torch.tensor(theta, device="cuda")
        c = torch.empty(N, device="cuda")
        g = torch.empty(N, D, device="cuda")
        prob.rollout_fwd(th, N, seed, 2, 0, c)
        prob.rollout_adjoint(th, N, seed, 2, g)
        prob.sync()
        grads.append(g.cpu().numpy())
        prob.close()
    for g in grads[1:]:
        assert rel_err(g, grads[0]).max() < 1e-4
