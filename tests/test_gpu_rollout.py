"""GPU rollout / adjoint parity against the FP64 oracle (through the C ABI).

Tolerances: trajectories and costs within 1e-4 relative and gradients within
1e-3 relative (max-norm per particle), on every particle whose rollout is
well-conditioned at float32 rounding (see tests/_common.conditioned); the
share of such particles is asserted too, so the bar cannot pass vacuously.
"""
import numpy as np
import pytest
import torch

from oracle import stamp_oracle as O
from paper_2310_01775_gb300 import workloads as W

from _common import Reference, rel_err

pytestmark = pytest.mark.gpu


def f32(P):
    """The problem as the library sees it: every constant rounded to float32."""
    return {k: (float(np.float32(v)) if isinstance(v, float) else v) for k, v in P.items()}


def setup(name, over, N, seed):
    P = f32(W.params(name, **over))
    init, goal = W.scene(P, seed)
    init = init.astype(np.float32).astype(np.float64)
    goal = goal.astype(np.float32).astype(np.float64)
    M, _, D = O.dims(P)
    theta = O.init_theta(seed, N, D).astype(np.float32)
    return P, init, goal, M, D, theta


def gpu_rollout(P, init, goal, theta, seed, it, lanes=None, hard=0, adj_mode=None):
    from paper_2310_01775_gb300 import stamp as S
    dev = torch.device("cuda:0")
    N, D = theta.shape
    prob = S.Problem(P, init, goal, N, torch.cuda.current_stream().cuda_stream)
    if lanes:
        prob.set_lanes(lanes, lanes)
    if adj_mode is not None:
        prob.set_adjoint_mode(adj_mode)
    th = torch.tensor(theta, device=dev)
    cost = torch.empty(N, device=dev)
    fin = torch.empty(N, prob.S, device=dev)
    grad = torch.empty(N, D, device=dev)
    tape = torch.empty(prob.n_ckpt + 1, N, prob.S, device=dev)
    prob.rollout_fwd(th, N, seed, it, hard, cost, fin)
    prob.read_tape(N, tape)
    if not hard:
        prob.rollout_adjoint(th, N, seed, it, grad)
    prob.sync()
    prob.close()
    nb = P["n_blocks"]
    tape = tape.cpu().numpy().transpose(1, 0, 2).reshape(N, -1, nb, 6)
    return cost.cpu().numpy(), fin.cpu().numpy(), tape, grad.cpu().numpy()


# Contact constants of the workloads (k=1e4, c=50) and a softer contact
# (k=1e3, c=10) under which every particle is well-conditioned, so the bar
# holds on all particles and over whole horizons.
SOFT = dict(k_contact=1e3, c_contact=10.0)
CASES = [
    # name, overrides, N, lanes, minimum share of conditioned particles
    ("pusher1_h2", dict(H=1, ckpt_every=1), 37, 1, 0.3),
    ("pusher1_h2", dict(H=1, ckpt_every=1), 37, 2, 0.3),
    ("pusher1_h2", dict(H=1, ckpt_every=1), 37, 4, 0.3),
    ("pusher1_h4", dict(H=1, ckpt_every=1), 64, 4, 0.3),
    ("pusher1_h2", dict(ckpt_every=1), 32, 4, 0.3),           # both actions, every substep
    ("pusher1_h2", dict(ckpt_every=25), 33, 4, 0.3),          # checkpoint replay
    ("pusher3_h6", dict(n_blocks=2, H=1, ckpt_every=1), 48, 8, 0.1),
    ("pusher3_h6", dict(n_blocks=2, H=1, ckpt_every=25), 48, 16, 0.1),
    ("pusher3_h6", dict(H=1, ckpt_every=1), 48, 16, 0.1),
    ("pusher3_h6", dict(H=1, ckpt_every=25), 48, 8, 0.1),
    ("pusher3_h6", dict(H=1, ckpt_every=20), 48, 32, 0.1),
    ("pusher3_h6", dict(n_blocks=4, H=1, ckpt_every=25), 32, 16, 0.05),
    ("pusher1_h2", dict(SOFT, ckpt_every=1), 40, 4, 1.0),
    ("pusher1_h4", dict(SOFT), 40, 4, 1.0),                    # 4 actions of 100 substeps
    ("pusher1_h4", dict(SOFT), 40, 1, 1.0),
    ("pusher3_h6", dict(SOFT, n_blocks=2, H=2), 24, 8, 0.6),
    ("pusher3_h6", dict(SOFT, H=2), 24, 16, 0.6),
]


@pytest.mark.parametrize("name,over,N,lanes,min_frac", CASES)
def test_rollout_and_adjoint_parity(name, over, N, lanes, min_frac):
    seed, it = 5, 3
    P, init, goal, M, D, theta = setup(name, over, N, seed)
    cost, fin, tape, grad = gpu_rollout(P, init, goal, theta, seed, it, lanes)
    gum = O.gumbel_noise(seed, it, N, P["H"], M)
    ref = Reference(theta, P, init, goal, gum, C=P["ckpt_every"])
    assert tape.shape == ref.traj.shape
    ref.check(tape, fin, cost, grad, min_frac=min_frac)
    assert np.isfinite(tape).all() and np.isfinite(grad).all()


def test_hard_rollout_parity():
    seed = 2
    P, init, goal, M, D, theta = setup("pusher1_h2", dict(ckpt_every=1), 40, seed)
    cost, fin, tape, _ = gpu_rollout(P, init, goal, theta, seed, -1, hard=1)
    ref = Reference(theta, P, init, goal, None, need_grad=False, hard=True)
    ref.check(tape, fin, cost)


@pytest.mark.parametrize("N", [1, 2, 31, 33])
def test_ragged_particle_counts(N):
    seed, it = 9, 0
    P, init, goal, M, D, theta = setup("pusher1_h2", dict(H=1, ckpt_every=1), N, seed)
    cost, fin, tape, grad = gpu_rollout(P, init, goal, theta, seed, it)
    gum = O.gumbel_noise(seed, it, N, P["H"], M)
    ref = Reference(theta, P, init, goal, gum)
    ref.check(tape, fin, cost, grad, min_frac=0.0)
    assert np.isfinite(grad).all()


def test_noise_free_and_deterministic():
    seed = 4
    P, init, goal, M, D, theta = setup("pusher1_h2", {}, 16, seed)
    a = gpu_rollout(P, init, goal, theta, seed, -1)
    b = gpu_rollout(P, init, goal, theta, seed, -1)
    for x, y in zip(a, b):
        assert np.array_equal(x, y)
    Reference(theta, P, init, goal, None, C=P["ckpt_every"]).check(a[2], a[1], a[0], a[3])


@pytest.mark.parametrize("name,sample,min_count", [("pusher1_h4", 16, 3), ("pusher3_h6", 512, 20)])
def test_full_size_sampled_particles(name, sample, min_count):
    """Full workload in the default launch configuration; the oracle checks a
    sample of particles one by one, over the first action (at least
    min_count of them conditioned) and, on a smaller sample, over the whole
    horizon."""
    P = f32(W.params(name))
    N, seed, it = P["N"], 11, 7
    init, goal = W.scene(P, seed)
    init = init.astype(np.float32).astype(np.float64)
    goal = goal.astype(np.float32).astype(np.float64)
    M, _, D = O.dims(P)
    theta = O.init_theta(seed, N, D).astype(np.float32)
    cost, fin, tape, grad = gpu_rollout(P, init, goal, theta, seed, it)
    assert np.isfinite(cost).all() and np.isfinite(grad).all()
    idx = np.random.default_rng(0).choice(N, size=sample, replace=False)
    gum = O.gumbel_noise(seed, it, N, P["H"], M)[idx]
    C, T, Pn = P["ckpt_every"], P["T"], M + 2
    first = Reference(theta[idx][:, :Pn], dict(P, H=1), init, goal, gum[:, :1], C=C,
                      need_grad=False)
    first.check(tape[idx][:, : T // C + 1], tape[idx][:, T // C], None, min_frac=0.03,
                min_count=min_count)
    few = idx[:12]
    whole = Reference(theta[few], P, init, goal, gum[:12], C=C)
    whole.check(tape[few], fin[few], cost[few], grad[few], min_frac=0.0)
    if P["n_blocks"] == 1 and C == 1:
        # the default sweep here is the time-parallel one; the sequential
        # sweep on the same tape sums the same derivatives in another order:
        # over all particles (chaotic ones included) the median gap stays far
        # below the gradient bar
        _, _, _, g_seq = gpu_rollout(P, init, goal, theta, seed, it, adj_mode=0)
        assert np.median(rel_err(grad, g_seq)) < 1e-4
    if C > 1:
        # the default sweep here rebuilds the per-substep tape by the segment
        # replay; the sequential sweep recomputes each segment on its serial
        # path: the same states up to the rounding of the force sums
        _, _, _, g_seq = gpu_rollout(P, init, goal, theta, seed, it, adj_mode=0)
        assert np.median(rel_err(grad, g_seq)) < 1e-4


def test_adjoint_requires_matching_forward():
    from paper_2310_01775_gb300 import stamp as S
    seed = 1
    P, init, goal, M, D, theta = setup("pusher1_h2", {}, 8, seed)
    prob = S.Problem(P, init, goal, 8, torch.cuda.current_stream().cuda_stream)
    th = torch.tensor(theta, device="cuda")
    g = torch.empty(8, D, device="cuda")
    c = torch.empty(8, device="cuda")
    with pytest.raises(S.StampError):
        prob.rollout_adjoint(th, 8, seed, 0, g)          # no forward yet
    prob.rollout_fwd(th, 8, seed, 0, 0, c)
    with pytest.raises(S.StampError):
        prob.rollout_adjoint(th, 8, seed + 1, 0, g)      # other noise
    with pytest.raises(S.StampError):
        prob.rollout_fwd(th, 9, seed, 0, 0, c)           # N above max_particles
    with pytest.raises(S.StampError):
        prob.rollout_fwd(th.cpu(), 8, seed, 0, 0, c)     # host theta
    prob.close()


# one-block, checkpoint-interval-1 cases: both reverse sweeps apply
ONE_BLOCK_C1 = [
    ("pusher1_h2", dict(H=1, ckpt_every=1), 37, 4, 0.3),
    ("pusher1_h2", dict(ckpt_every=1), 32, 2, 0.3),
    ("pusher1_h2", dict(SOFT, ckpt_every=1), 40, 4, 1.0),
    ("pusher1_h4", dict(SOFT), 40, 1, 1.0),
    ("pusher1_h4", dict(SOFT), 9, 4, 1.0),        # one partial group of 8
]


@pytest.mark.parametrize("mode", [0, 1])
@pytest.mark.parametrize("name,over,N,lanes,min_frac", ONE_BLOCK_C1)
def test_both_reverse_sweeps_meet_the_bar(name, over, N, lanes, min_frac, mode):
    """Sequential (0) and time-parallel (1) reverse sweeps against the FP64
    oracle, and against each other on the same tape: the same derivatives
    summed in another order."""
    seed, it = 5, 3
    P, init, goal, M, D, theta = setup(name, over, N, seed)
    cost, fin, tape, grad = gpu_rollout(P, init, goal, theta, seed, it, lanes, adj_mode=mode)
    gum = O.gumbel_noise(seed, it, N, P["H"], M)
    ref = Reference(theta, P, init, goal, gum, C=1)
    ok = ref.check(tape, fin, cost, grad, min_frac=min_frac)
    _, _, _, other = gpu_rollout(P, init, goal, theta, seed, it, lanes, adj_mode=1 - mode)
    assert rel_err(grad, other)[ok].max(initial=0) < 1e-4


def test_hard_rollout_time_parallel_gradient_has_no_logit_term():
    """The hard map's one-hot choice has no gradient; offset and distance do."""
    seed, it, N = 3, -1, 16
    P, init, goal, M, D, theta = setup("pusher1_h2", dict(SOFT, ckpt_every=1), N, seed)
    from paper_2310_01775_gb300 import stamp as S
    prob = S.Problem(P, init, goal, N, torch.cuda.current_stream().cuda_stream)
    assert prob.adjoint_mode(N) == S.STAMP_ADJ_TIME_PARALLEL
    th = torch.tensor(theta, device="cuda")
    c = torch.empty(N, device="cuda")
    g = torch.empty(N, D, device="cuda")
    g0 = torch.empty(N, D, device="cuda")
    prob.rollout_fwd(th, N, seed, it, 1, c)
    prob.rollout_adjoint(th, N, seed, it, g)
    prob.set_adjoint_mode(S.STAMP_ADJ_SEQUENTIAL)
    prob.rollout_adjoint(th, N, seed, it, g0)
    prob.sync()
    prob.close()
    g, g0 = g.cpu().numpy().reshape(N, P["H"], M + 2), g0.cpu().numpy().reshape(N, P["H"], M + 2)
    assert np.abs(g[:, :, :M]).max() == 0.0 and np.abs(g0[:, :, :M]).max() == 0.0
    assert np.abs(g[:, :, M:]).max() > 0.0
    assert np.median(rel_err(g, g0)) < 1e-5


def test_adjoint_mode_where_it_applies():
    from paper_2310_01775_gb300 import stamp as S
    for name, over, want in [("pusher1_h2", dict(ckpt_every=1), S.STAMP_ADJ_TIME_PARALLEL),
                             ("pusher1_h2", dict(ckpt_every=25), S.STAMP_ADJ_REPLAY),
                             ("pusher3_h6", dict(H=1, ckpt_every=1), S.STAMP_ADJ_SEQUENTIAL),
                             ("pusher3_h6", dict(H=1, ckpt_every=25), S.STAMP_ADJ_REPLAY)]:
        P = W.params(name, **over)
        init, goal = W.scene(P, 0)
        prob = S.Problem(P, init, goal, 8, torch.cuda.current_stream().cuda_stream)
        assert prob.adjoint_mode(8) == want, (name, over)
        prob.set_adjoint_mode(S.STAMP_ADJ_REPLAY)          # needs an interval > 1
        assert prob.adjoint_mode(8) == (S.STAMP_ADJ_REPLAY if over["ckpt_every"] > 1
                                        else S.STAMP_ADJ_SEQUENTIAL)
        prob.set_adjoint_mode(S.STAMP_ADJ_SEQUENTIAL)
        assert prob.adjoint_mode(8) == S.STAMP_ADJ_SEQUENTIAL
        with pytest.raises(S.StampError):
            prob.set_adjoint_mode(7)
        prob.close()
    # the automatic mode leaves a launch that would not fit on the GPU at once
    # to the sequential sweep
    P = W.params("pusher1_h4")
    init, goal = W.scene(P, 0)
    prob = S.Problem(P, init, goal, 16384, torch.cuda.current_stream().cuda_stream)
    assert prob.adjoint_mode(1024) == S.STAMP_ADJ_TIME_PARALLEL
    assert prob.adjoint_mode(16384) == S.STAMP_ADJ_SEQUENTIAL
    prob.set_adjoint_mode(S.STAMP_ADJ_TIME_PARALLEL)
    assert prob.adjoint_mode(16384) == S.STAMP_ADJ_TIME_PARALLEL
    prob.close()


@pytest.mark.parametrize("lanes", [4, 2])
def test_time_parallel_sweep_after_either_forward_team_width(lanes):
    """The time-parallel sweep reads only the tape and the relaxed parameters,
    so it serves a forward of any team width; both against the oracle."""
    seed, it, N = 5, 2, 45
    P, init, goal, M, D, theta = setup("pusher1_h4", dict(SOFT, H=2), N, seed)
    cost, fin, tape, grad = gpu_rollout(P, init, goal, theta, seed, it, lanes, adj_mode=1)
    gum = O.gumbel_noise(seed, it, N, P["H"], M)
    Reference(theta, P, init, goal, gum, C=1).check(tape, fin, cost, grad, min_frac=0.9)


# checkpoint interval > 1: the segment replay and the sequential sweep apply
REPLAY_CASES = [
    ("pusher1_h2", dict(ckpt_every=25), 33, 4, 0.3),
    ("pusher1_h2", dict(SOFT, ckpt_every=10), 40, 2, 1.0),
    ("pusher3_h6", dict(n_blocks=2, H=1, ckpt_every=25), 48, 16, 0.1),
    ("pusher3_h6", dict(H=1, ckpt_every=25), 48, 8, 0.1),
    ("pusher3_h6", dict(SOFT, H=2, ckpt_every=25), 24, 16, 0.6),
    ("pusher3_h6", dict(SOFT, H=2, ckpt_every=20), 70, 32, 0.6),   # ragged N, another interval
    ("pusher3_h6", dict(n_blocks=4, H=1, ckpt_every=25), 32, 16, 0.05),
]


@pytest.mark.parametrize("mode", [0, 3])
@pytest.mark.parametrize("name,over,N,lanes,min_frac", REPLAY_CASES)
def test_replay_and_sequential_sweeps_meet_the_bar(name, over, N, lanes, min_frac, mode):
    """Sequential (0) and segment-replay (3) reverse sweeps against the FP64
    oracle, and against each other: the replay rebuilds the states between
    checkpoints in parallel, the sequential sweep on its serial path, with
    force sums grouped by other team widths."""
    seed, it = 5, 3
    P, init, goal, M, D, theta = setup(name, over, N, seed)
    cost, fin, tape, grad = gpu_rollout(P, init, goal, theta, seed, it, lanes, adj_mode=mode)
    gum = O.gumbel_noise(seed, it, N, P["H"], M)
    ref = Reference(theta, P, init, goal, gum, C=P["ckpt_every"])
    ok = ref.check(tape, fin, cost, grad, min_frac=min_frac)
    _, _, _, other = gpu_rollout(P, init, goal, theta, seed, it, lanes, adj_mode=3 - mode)
    assert rel_err(grad, other)[ok].max(initial=0) < 1e-4
