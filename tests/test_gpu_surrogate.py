"""The learned pose-dynamics surrogate on the GPU against the FP64 oracle
(oracle/surrogate_oracle.py), through the C ABI.

Bars.  Transition features: sampled poses bit-exact (same float32 operations
on both sides), derived features within 2e-6; simulated pose changes within
the trajectory bar 1e-4 on conditioned transitions (two float32 replays, one
from start poses moved by an ulp, within 1e-5 of FP64 over the whole push).  Surrogate cost and gradient: the network runs in bfloat16 (8
significant bits, unit roundoff 2^-9); a bias-only network removes the
bfloat16 products and must match the closed form to float32 rounding, while
a random network is held to a median relative error of 2e-2 (cost) and 3e-2
(gradient), about ten bfloat16 roundoffs, with no particle above 0.25.
Screening is index work: bit-exact against the selection rule applied to the
GPU's own float32 costs.
"""
import math

import numpy as np
import pytest
import torch

from oracle import stamp_oracle as O
from oracle import surrogate_oracle as SO
from paper_2310_01775_gb300 import workloads as W

pytestmark = pytest.mark.gpu


def _S():
    from paper_2310_01775_gb300 import stamp as S
    return S


def _stream():
    return torch.cuda.current_stream().cuda_stream


def _packed(params):
    return torch.tensor(np.concatenate([np.concatenate([Wl.ravel(), bl]) for Wl, bl in params]),
                        dtype=torch.float32, device="cuda")


def _random_net(nb, seed, head_scale=0.3):
    F, OUT = SO.feature_dims(nb)
    params = W.mlp_init([F, 256, 256, 256, OUT], seed)
    params[-1] = (params[-1][0] * head_scale, params[-1][1] * head_scale)
    return params


def test_transitions_match_the_oracle():
    S = _S()
    P = W.params("pusher3_h6")
    n, seed = 4096 + 300, 11                      # a full chunk and a ragged one
    sur = S.Surrogate(P, 8192, 256, _stream())
    F, OUT = sur.in_dim, sur.out_dim
    x = torch.empty(n, F, device="cuda")
    y = torch.empty(n, OUT, device="cuda")
    sur.transitions(n, seed, x, y)
    sur.sync()
    x, y = x.cpu().numpy(), y.cpu().numpy()
    xo, yo, q0, th = SO.transitions(seed, n, P)
    pose_cols = [4 * b + c for b in range(3) for c in (0, 1)]
    assert np.array_equal(x[:, pose_cols], q0[:, :, :2].reshape(n, 6))
    # cos/sin, softmax with Gumbel noise, tanh, sigmoid in float32 vs float64
    assert np.abs(x - xo).max() <= 2e-5, np.abs(x - xo).max(0)
    # the push itself: final pose start + delta against the FP64 and FP32 simulator
    P1 = dict(P, H=1)
    M = 12
    gum = np.concatenate([O.gumbel_noise(cs, 0, m, 1, M) for _, m, cs in SO._chunks(seed, n)])
    th64, q64 = th.astype(np.float64), q0.astype(np.float64)
    _, f64, t64 = O.rollout(th64, P1, q64, np.zeros((3, 3)), gum, record=True)
    want = f64[:, :, :3].reshape(n, 9)
    scale = np.abs(want).max(1)

    def traj_floor(init):
        """Largest pose deviation from FP64 over the whole push, of a float32 replay."""
        _, _, t = O.rollout(th64, P1, init, np.zeros((3, 3)), gum, record=True, dtype=torch.float32)
        return np.abs(t[..., :3] - t64[..., :3]).reshape(n, -1).max(1) / scale

    # conditioning: float32 replays stay within 1e-5 of FP64 over the whole push,
    # also from start poses moved by about one float32 ulp (fixed random signs);
    # squeezed blocks can diverge mid-push and re-converge at rest, so the end
    # pose alone does not show it
    sgn = np.where(np.random.default_rng(0).random(q64.shape) < 0.5, -1.0, 1.0)
    floor, probe = traj_floor(q64), traj_floor(q64 * (1 + sgn * 2.0 ** -23))
    got = q0.reshape(n, 9).astype(np.float64) + y
    err = np.abs(got - want).max(1) / scale
    ok = (floor < 1e-5) & (probe < 1e-5)
    stats = (f"conditioned {ok.mean():.3f}, max err there {err[ok].max(initial=0):.2e}, "
             f"median err {np.median(err):.2e}, median floor {np.median(floor):.2e}")
    assert ok.mean() > 0.5, stats
    assert err[ok].max() < 1e-4, stats
    assert np.median(err) <= 3 * np.median(floor) + 1e-6, stats


def test_bias_only_network_is_exact():
    """Zero weights: every push adds the head's float32 bias, so the cost and
    gradient follow the closed form of the oracle's pin to float32 rounding."""
    S = _S()
    P = W.params("pusher3_h6")
    init, goal = W.scene(P, 3)
    F, OUT = SO.feature_dims(3)
    params = [(np.zeros((o, i)), np.zeros(o)) for i, o in [(F, 256), (256, 256), (256, 256), (256, OUT)]]
    params[-1] = (np.zeros((OUT, 256)), np.linspace(-0.05, 0.07, OUT))
    N = 300
    prob = S.Problem(P, init, goal, N, _stream())
    sur = S.Surrogate(P, 1024, N, _stream())
    sur.set_params(_packed(params))
    theta = torch.tensor(W.random_theta(N, prob.D, 5), device="cuda")
    cost = torch.empty(N, device="cuda")
    grad = torch.full((N, prob.D), float("nan"), device="cuda")
    sur.rollout(prob, theta, N, 7, 2, cost, grad)
    sur.sync()
    M = 12
    gum = O.gumbel_noise(7, 2, N, P["H"], M)
    c_o, g_o = SO.rollout_grad(params, theta.cpu().numpy().astype(np.float64), P, init, goal, gum)
    c = cost.cpu().numpy()
    assert np.abs(c - c_o).max() <= 1e-5 * np.abs(c_o).max()
    g = grad.cpu().numpy()
    assert np.isfinite(g).all()
    assert np.abs(g - g_o).max() <= 1e-5 * np.abs(g_o).max()
    prob.close()
    sur.close()


@pytest.mark.parametrize("name,N", [("pusher3_h6", 300), ("pusher1_h4", 129)])
def test_surrogate_rollout_and_gradient_match_the_oracle(name, N):
    S = _S()
    P = W.params(name)
    nb = P["n_blocks"]
    init, goal = W.scene(P, 1)
    params = _random_net(nb, 21)
    prob = S.Problem(P, init, goal, N, _stream())
    sur = S.Surrogate(P, 1024, N, _stream())
    sur.set_params(_packed(params))
    theta = torch.tensor(W.random_theta(N, prob.D, 8), device="cuda")
    cost = torch.empty(N, device="cuda")
    grad = torch.empty(N, prob.D, device="cuda")
    sur.rollout(prob, theta, N, 3, 9, cost, grad)
    cost_nograd = torch.empty(N, device="cuda")
    sur.rollout(prob, theta, N, 3, 9, cost_nograd)
    sur.sync()
    gum = O.gumbel_noise(3, 9, N, P["H"], 4 * nb)
    c_o, g_o = SO.rollout_grad(params, theta.cpu().numpy().astype(np.float64), P, init, goal, gum)
    c, g = cost.cpu().numpy().astype(np.float64), grad.cpu().numpy().astype(np.float64)
    assert np.array_equal(cost.cpu().numpy(), cost_nograd.cpu().numpy())
    ec = np.abs(c - c_o) / np.abs(c_o)
    eg = np.abs(g - g_o).max(1) / np.abs(g_o).max(1)
    stats = f"cost median {np.median(ec):.2e} max {ec.max():.2e}; grad median {np.median(eg):.2e} max {eg.max():.2e}"
    assert np.median(ec) <= 2e-2 and ec.max() <= 0.25, stats
    assert np.median(eg) <= 3e-2 and eg.max() <= 0.25, stats
    prob.close()
    sur.close()


def test_screening_keeps_the_lowest_surrogate_costs():
    S = _S()
    P = W.params("pusher3_h6")
    init, goal = W.scene(P, 2)
    n_cand, N = 20000, 500                        # three selection chunks, two passes
    prob = S.Problem(P, init, goal, N, _stream())
    sur = S.Surrogate(P, n_cand, N, _stream())
    sur.set_params(_packed(_random_net(3, 4)))
    cand = torch.tensor(O.init_theta(5, n_cand, prob.D).astype(np.float32), device="cuda")
    cost = torch.empty(n_cand, device="cuda")
    sur.rollout(prob, cand, n_cand, 0, -1, cost)
    out = torch.empty(N, prob.D, device="cuda")
    idx = torch.empty(N, dtype=torch.int32, device="cuda")
    sur.screen(prob, cand, n_cand, N, out, idx)
    sur.sync()
    want = SO.select_lowest(cost.cpu().numpy(), N)
    assert np.array_equal(idx.cpu().numpy(), want)
    assert torch.equal(out, cand[idx.long()])
    prob.close()
    sur.close()


@pytest.fixture(scope="module")
def trained():
    """A surrogate for the 3-block physics trained on 2^20 GPU transitions
    (4096 Adam steps of 4096 rows), sized for 131072-candidate screening."""
    from paper_2310_01775_gb300 import surrogate_compare as SC
    S = _S()
    P = W.params("pusher3_h6")
    sur, secs, losses = SC.train_surrogate(P, 1 << 20, _stream(), 131072, 2048)
    yield S, P, sur, losses
    sur.close()


def test_training_lowers_the_loss_and_predicts_held_out_pushes(trained):
    """Held-out transitions of another seed (blow-ups dropped as in training):
    every output keeps a large share of its variance explained (positions are
    the hard part: opposing virtual pushers nearly cancel, so the net motion
    of a squeezed block is a small difference)."""
    S, P, sur, losses = trained
    assert np.isfinite(losses).all()
    assert losses[-1] < 0.4 * losses[0], losses
    assert sur.last_kept() > 0.95 * (1 << 20)
    n = 8192
    x = torch.empty(n, sur.in_dim, device="cuda")
    y = torch.empty(n, sur.out_dim, device="cuda")
    sur.transitions(n, 99, x, y)                  # held-out seed
    net = S.MLP(sur.in_dim, sur.out_dim, n, 0, _stream())
    params = torch.empty(sur.n_params, device="cuda")
    sur.get_params(params)
    net.set_params(params)
    pred = torch.empty_like(y)
    net.forward(x, n, pred)
    net.sync()
    keep = (y[:, [0, 1, 3, 4, 6, 7]].abs().max(1).values <= 0.5) & \
           (y[:, [2, 5, 8]].abs().max(1).values <= math.pi)
    y, pred = y[keep], pred[keep]
    r2 = (1 - ((pred - y) ** 2).mean(0) / y.var(0)).cpu().numpy()
    assert r2[[0, 1, 3, 4, 6, 7]].min() > 0.55 and r2[[2, 5, 8]].min() > 0.85, r2
    net.close()


def test_trained_surrogate_screens_better_than_random_or_untrained(trained):
    """What the learned model gains at the start of a solve: of 16384 uniform
    candidates, the 256 it ranks best have a lower true (simulated, relaxed,
    noise-free) cost than the 256 a plain solve starts from, and than the 256
    an untrained network picks; on a uniform-goal and a planted scene."""
    from paper_2310_01775_gb300 import surrogate_compare as SC
    S, P, sur, _ = trained
    n_cand, N = 16384, 256
    fresh = S.Surrogate(P, n_cand, N, _stream())
    fresh.init_params(2)
    for init, goal in (W.scene(P, 7), SC.planted_scene(P, 3, _stream())):
        prob = S.Problem(P, init, goal, N, _stream())
        cand = torch.tensor(O.init_theta(7, n_cand, prob.D).astype(np.float32), device="cuda")

        def true_cost(th):
            c = torch.empty(N, device="cuda")
            prob.rollout_fwd(th, N, 0, -1, 0, c)
            prob.sync()
            return float(np.median(c.cpu().numpy()))

        picked = torch.empty(N, prob.D, device="cuda")
        sur.screen(prob, cand, n_cand, N, picked)
        sur.sync()
        c_trained, c_plain = true_cost(picked), true_cost(cand[:N].contiguous())
        fresh.screen(prob, cand, n_cand, N, picked)
        fresh.sync()
        c_untrained = true_cost(picked)
        assert c_trained < 0.8 * c_plain and c_trained < 0.85 * c_untrained, \
            (c_trained, c_plain, c_untrained)
        prob.close()
    fresh.close()


def test_surrogate_solve_beats_plain_svgd_on_planted_problems(trained):
    """What the learned model gains over the method without it: on planted
    3-block problems (N = 2048, 500 iterations each arm) the surrogate-assisted
    solve (131072 candidates screened, 300 surrogate + 200 simulator
    iterations) ends at a lower hard cost on most problems, in less time."""
    from paper_2310_01775_gb300 import surrogate_compare as SC
    S, P, sur, _ = trained
    res = SC.compare(P, (3, 4, 5), sur, N=2048, n_candidates=131072, surrogate_iters=300,
                     sim_iters=200, stream=_stream())
    rows = res["per_seed"]
    better = sum(r["surrogate"]["best_cost"] <= r["plain"]["best_cost"] for r in rows)
    t_sur = sum(r["surrogate"]["seconds"] for r in rows)
    t_plain = sum(r["plain"]["seconds"] for r in rows)
    assert better >= 2 and t_sur < 0.8 * t_plain, rows


def test_solve_surrogate_without_surrogate_work_is_the_plain_solve():
    S = _S()
    P = W.params("pusher1_h2")
    init, goal = W.scene(P, 0)
    N = 32
    prob = S.Problem(P, init, goal, N, _stream())
    sur = S.Surrogate(P, 64, N, _stream())
    a = torch.empty(N, prob.D, device="cuda")
    b = torch.empty(N, prob.D, device="cuda")
    prob.solve(N, 20, 6, 5, 1e-2, None, a)
    prob.solve_surrogate(sur, N, N, 0, 20, 5, 1e-2, b, sgd_iters=6)
    assert torch.equal(a, b)
    prob.close()
    sur.close()


def test_solve_surrogate_runs_all_phases_and_stops_at_the_target(trained):
    S, P, sur, _ = trained
    init, goal = W.scene(P, 5)
    N = 256
    prob = S.Problem(P, init, goal, N, _stream())
    th = torch.empty(N, prob.D, device="cuda")
    cost = torch.empty(N, device="cuda")
    topk = np.zeros(3, dtype=np.int32)
    stats = np.zeros(35, dtype=np.float32)
    prob.solve_surrogate(sur, 8192, N, 20, 10, 4, 1e-2, th, cost, 3, topk, stats, sgd_iters=5)
    it, best = prob.solve_info()
    c = cost.cpu().numpy()
    assert it == 35 and np.isfinite(stats).all() and np.isfinite(c).all()
    assert best == c.min()
    assert topk[0] == int(np.lexsort((np.arange(N), c))[0])
    # early stop: any cost is below a huge target at the first check
    prob.set_target(1e9, 5)
    prob.solve_surrogate(sur, 8192, N, 20, 10, 4, 1e-2, th, cost, 3, topk, None)
    assert prob.solve_info()[0] == 5
    prob.set_target(0.0, 0)
    prob.close()
