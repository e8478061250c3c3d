"""Pins for the FP64 surrogate reference (oracle/surrogate_oracle.py).

The surrogate composes pinned parts (the relaxation, the cost, the MLP of
oracle/mlp_oracle.py); these tests pin the composition: a bias-only network
has a closed-form pose recursion, cost and gradient; one surrogate step equals
the independently pinned numpy MLP on hand-checked features; the reverse
sweep matches central differences; the transition samplers meet their
stated ranges, separation rule and moments; and a transition's target is the
simulator's pose change over one push.
"""
import math

import numpy as np
import torch

from oracle import mlp_oracle as MO
from oracle import stamp_oracle as O
from oracle import surrogate_oracle as SO
from paper_2310_01775_gb300 import workloads as W


def _net(nb, seed, hidden=16):
    F, OUT = SO.feature_dims(nb)
    return W.mlp_init([F, hidden, hidden, hidden, OUT], seed)


def test_features_of_a_known_pose():
    P = W.params("pusher1_h2")
    q = torch.tensor([[[0.1, -0.2, math.pi / 2]]], dtype=torch.float64)
    z = torch.tensor([[0.1, 0.2, 0.3, 0.4]], dtype=torch.float64)
    off = torch.tensor([0.5 * P["offset_max"]], dtype=torch.float64)
    dist = torch.tensor([0.25 * P["dist_max"]], dtype=torch.float64)
    f = SO.features(q, z, off, dist, P).numpy()[0]
    assert np.allclose(f, [0.1, -0.2, 0.0, 1.0, 0.1, 0.2, 0.3, 0.4, 0.5, 0.25], atol=1e-15)


def test_bias_only_network_closed_form():
    """All weights zero: every hidden activation is SiLU(0) = 0, so each push
    adds the head's bias b.  Then q_H = q_0 + H b, C is the cost of that pose
    plus the push term, and only the distance parameters get a gradient:
    dC/dv_k = 2 w_push dist_k * dist_max * s (1 - s), s = sigmoid(v_k)."""
    P = W.params("pusher3_h6")
    init, goal = W.scene(P, 4)
    F, OUT = SO.feature_dims(3)
    params = [(np.zeros((o, i)), np.zeros(o)) for i, o in [(F, 8), (8, 8), (8, 8), (8, OUT)]]
    b = np.linspace(-0.05, 0.07, OUT)
    params[-1] = (np.zeros((OUT, 8)), b)
    M, Pn, D = O.dims(P)
    theta = W.random_theta(5, D, 3).astype(np.float64)
    c, g = SO.rollout_grad(params, theta, P, init, goal)
    qH = np.asarray(init) + P["H"] * b.reshape(3, 3)
    e = qH - np.asarray(goal)
    yaw = np.arctan2(np.sin(e[:, 2]), np.cos(e[:, 2]))
    th = theta.reshape(5, P["H"], Pn)
    s = 1.0 / (1.0 + np.exp(-th[:, :, M + 1]))
    dist = P["dist_max"] * s
    want = (e[:, :2] ** 2).sum() + P["w_yaw"] * (yaw ** 2).sum() + P["w_push"] * (dist ** 2).sum(1)
    assert np.allclose(c, want, rtol=1e-13)
    g = g.reshape(5, P["H"], Pn)
    assert np.abs(g[:, :, :M + 1]).max() == 0.0
    assert np.allclose(g[:, :, M + 1], -2 * P["w_push"] * dist * P["dist_max"] * s * (1 - s), rtol=1e-12)


def test_one_step_equals_the_numpy_mlp():
    P = W.params("pusher1_h2", H=1)
    init, goal = W.scene(P, 0)
    params = _net(1, 9)
    M, Pn, D = O.dims(P)
    theta = W.random_theta(6, D, 11).astype(np.float64)
    gum = O.gumbel_noise(7, 2, 6, 1, M)
    qs, _ = SO.surrogate_poses(params, torch.tensor(theta), P, init, gum)
    # features written out by hand from the relaxation's definition
    a = theta[:, :M] + gum[:, 0]
    z = np.exp(a / P["tau"] - (a / P["tau"]).max(1, keepdims=True))
    z /= z.sum(1, keepdims=True)
    q0 = np.asarray(init)[0]
    f = np.concatenate([np.tile([q0[0], q0[1], np.cos(q0[2]), np.sin(q0[2])], (6, 1)), z,
                        np.tanh(theta[:, M:M + 1]), 1 / (1 + np.exp(-theta[:, M + 1:M + 2]))], 1)
    y, _ = MO.forward(params, f)
    assert np.allclose(qs[1].numpy().reshape(6, 3), q0 + y, rtol=1e-12, atol=1e-14)


def test_gradient_matches_central_differences():
    P = W.params("pusher3_h6", H=3)
    init, goal = W.scene(P, 1)
    params = _net(3, 5)
    M, Pn, D = O.dims(P)
    theta = W.random_theta(2, D, 21).astype(np.float64)
    gum = O.gumbel_noise(3, 5, 2, P["H"], M)
    _, g = SO.rollout_grad(params, theta, P, init, goal, gum)
    h = 1e-6
    for i in range(2):
        for d in range(0, D, 3):
            tp, tm = theta.copy(), theta.copy()
            tp[i, d] += h
            tm[i, d] -= h
            fd = (SO.rollout(params, tp, P, init, goal, gum)[i]
                  - SO.rollout(params, tm, P, init, goal, gum)[i]) / (2 * h)
            assert abs(-g[i, d] - fd) <= 1e-6 * max(1.0, abs(fd)), (i, d, -g[i, d], fd)


def test_start_pose_sampler_ranges_separation_and_moments():
    cs = int(O.sm64(np.uint64(17), np.uint64(0)))
    q = SO.sample_start_poses(cs, 3000, 3).astype(np.float64)
    assert np.abs(q[..., :2]).max() <= 0.5 and np.abs(q[..., 2]).max() <= math.pi / 2
    for a in range(3):
        for b in range(a + 1, 3):
            assert (np.hypot(q[:, a, 0] - q[:, b, 0], q[:, a, 1] - q[:, b, 1]) > 0.16).all()
    # one block: the first attempt is always taken, so the draws are uniform
    q1 = SO.sample_start_poses(cs, 4000, 1).astype(np.float64)[:, 0]
    se = math.sqrt(1 / 12 / 4000)
    assert abs(q1[:, 0].mean()) < 4 * se and abs(q1[:, 1].mean()) < 4 * se
    assert abs(q1[:, 0].var() - 1 / 12) < 0.01
    assert abs(q1[:, 2].var() - math.pi ** 2 / 12) < 0.1


def test_action_sampler_range_and_moments():
    """Offset and distance parameters U(-3, 3) (variance 3); logits U(-3, 3)
    times a per-row U(0, 1) scale: variance 3 E[w^2] = 1, and one row's
    logits share that scale."""
    th = SO.sample_actions(123, 5000, 6).astype(np.float64)
    assert th.shape == (5000, 6) and np.abs(th).max() <= 3.0
    assert abs(th.mean()) < 0.05
    assert abs(th[:, 4:].var() - 3.0) < 0.15 and abs(th[:, :4].var() - 1.0) < 0.06
    cs = 123
    key = O.sm64(np.uint64(cs), SO.STREAM_ACTIONS)
    w = O.uniform23(O.sm64(key, np.arange(5000, dtype=np.uint64) * 7 + 6))
    assert (np.abs(th[:, :4]).max(1) <= 3.0 * w + 1e-6).all()


def test_transition_targets_are_simulator_pose_changes():
    """The target of transition i is the pose after one relaxed push minus the
    start pose; the start pose is inside the features."""
    P = W.params("pusher1_h2")
    x, y, q0, th = SO.transitions(5, 6, P)
    cs = int(O.sm64(np.uint64(5), np.uint64(0)))
    P1 = dict(P, H=1)
    M = 4
    c, final = O.rollout(th.astype(np.float64), P1, q0.astype(np.float64), np.zeros((1, 3)),
                         O.gumbel_noise(cs, 0, 6, 1, M))
    assert np.allclose(y, final[:, :, :3].reshape(6, 3) - q0.reshape(6, 3), atol=1e-15)
    assert np.allclose(x[:, :2], q0[:, 0, :2])
    assert np.allclose(x[:, 2], np.cos(q0[:, 0, 2])) and np.allclose(x[:, 3], np.sin(q0[:, 0, 2]))
    assert np.allclose(x[:, 8], np.tanh(th[:, M])) and np.allclose(x[:, 9], 1 / (1 + np.exp(-th[:, M + 1])))
    # every side's virtual pusher starts touching the block: a push always moves it
    assert (np.abs(y[:, :2]).max(1) > 1e-4).all()


def test_select_lowest_breaks_ties_by_index():
    c = np.array([3.0, 1.0, 2.0, 1.0, 0.5], dtype=np.float32)
    assert list(SO.select_lowest(c, 3)) == [4, 1, 3]
