"""Algorithm 1 end to end on the GPU (stamp_solve) against the oracle's solve.

Per-particle values after hundreds of iterations are chaotic under the stiff
contact model (parity unpinned for them); what must agree is the final set of
top-k discrete plans, and the two paths must reach comparable costs.
"""
import json
import os

import numpy as np
import pytest
import torch

from oracle import stamp_oracle as O
from paper_2310_01775_gb300 import workloads as W

pytestmark = pytest.mark.gpu


def gpu_solve(P, init, goal, N, iters, sgd, seed, k=3, host=False, theta0=None):
    from paper_2310_01775_gb300 import stamp as S
    prob = S.Problem(P, init, goal, N, torch.cuda.current_stream().cuda_stream)
    D = prob.D
    if host:
        th = np.zeros((N, D), dtype=np.float32)
        cost = np.zeros(N, dtype=np.float32)
    else:
        th = torch.zeros(N, D, device="cuda")
        cost = torch.zeros(N, device="cuda")
    topk = np.zeros(k, dtype=np.int32)
    stats = np.zeros(iters + sgd, dtype=np.float32)
    prob.solve(N, iters, sgd, seed, P["lr"], theta0, th, cost, k, topk, stats)
    prob.close()
    if not host:
        th, cost = th.cpu().numpy(), cost.cpu().numpy()
    return th, cost, topk, stats


def test_initial_particles_match_oracle_generator():
    P = W.params("pusher1_h2")
    init, goal = W.scene(P, 0)
    th, _, _, _ = gpu_solve(P, init, goal, 16, 0, 0, seed=12, k=0)
    assert np.array_equal(th, O.init_theta(12, 16, 12).astype(np.float32))


def test_host_and_device_buffers_agree_and_runs_are_deterministic():
    P = W.params("pusher1_h2")
    init, goal = W.scene(P, 1)
    a = gpu_solve(P, init, goal, 32, 20, 5, seed=3)
    b = gpu_solve(P, init, goal, 32, 20, 5, seed=3, host=True)
    for x, y in zip(a, b):
        assert np.array_equal(x, y)


def test_topk_is_first_distinct_plans_in_cost_order():
    """The top-k kernel's output satisfies its definition on the GPU's own
    hard costs: walking particles in (cost, index) order, each kept particle
    is the first one with its discrete plan Gamma(theta)."""
    P = W.params("pusher1_h2")
    init, goal = W.scene(P, 2)
    th, cost, topk, _ = gpu_solve(P, init, goal, 64, 10, 0, seed=5, k=5)
    plans = [tuple(r) for r in np.argmax(th.reshape(64, P["H"], -1)[:, :, :4], axis=-1)]
    order = sorted(range(64), key=lambda i: (cost[i], i))
    firsts = []
    for i in order:
        if plans[i] not in [plans[j] for j in firsts]:
            firsts.append(i)
    want = (firsts + [-1] * 5)[:5]
    assert list(topk) == want


GOLDEN = os.path.join(os.path.dirname(__file__), "golden")
SOFT = dict(k_contact=1e3, c_contact=10.0)


def golden(kind):
    with open(os.path.join(GOLDEN, f"solve_pusher1_h2_{kind}.json")) as f:
        return json.load(f)["seeds"]


@pytest.mark.parametrize("seed", [0, 1, 2, 3])
def test_solve_plan_set_matches_oracle(seed):
    """1 block, H=2, T=50, N=32, 200 SVGD iterations, Adam lr 1e-2, with the
    softer contact under which every rollout is well-conditioned: the final
    top-3 discrete plan set equals the FP64 oracle's (stored by
    tests/golden/make_solve_golden.py)."""
    P = W.params("pusher1_h2", **SOFT)
    init, goal = W.scene(P, seed)
    th, cost, topk, stats = gpu_solve(P, init, goal, P["N"], P["svgd_iters"], 0, seed)
    ref = golden("soft")[str(seed)]["f64"]
    gpu_plans = {tuple(int(x) for x in O.plan_codes(th[i:i + 1], P)[0]) for i in topk if i >= 0}
    assert gpu_plans == {tuple(p) for p in ref["topk_plans"]}
    # and the per-iteration minimum relaxed cost follows the oracle's course
    # (float32 Stein/Adam arithmetic lets it drift slowly; the plan set above
    # is the bar)
    ref_min = np.asarray(ref["min_cost"])
    rel = np.abs(stats - ref_min) / np.maximum(ref_min, 1e-8)
    assert np.median(rel) < 1e-2, np.median(rel)


def test_stiff_solve_matches_oracle_statistics():
    """Workload constants (k=1e4, c=50): per-particle values are chaotic, so
    the float32 oracle itself does not reproduce the float64 top-3.  Over six
    seeds the GPU must agree with the float64 oracle at least as well as the
    float32 oracle does (share of top-3 plans found among the oracle's five
    best plans), and reach comparable best hard costs."""
    P = W.params("pusher1_h2")
    G = golden("stiff")
    ours, f32, ratio = [], [], []
    for seed in range(10):
        init, goal = W.scene(P, seed)
        th, cost, topk, _ = gpu_solve(P, init, goal, P["N"], P["svgd_iters"], 0, seed)
        ref5 = {tuple(p) for p, _ in G[str(seed)]["f64"]["top5"]}
        plans = [tuple(int(x) for x in O.plan_codes(th[i:i + 1], P)[0]) for i in topk if i >= 0]
        ours.append(np.mean([p in ref5 for p in plans]))
        f32.append(np.mean([tuple(p) in ref5 for p in G[str(seed)]["f32"]["topk_plans"]]))
        ratio.append(float(cost.min()) / G[str(seed)]["f64"]["top5"][0][1])
    assert np.mean(ours) >= np.mean(f32) - 0.25, (ours, f32)
    assert 0.5 <= np.median(ratio) <= 2.0, ratio


def test_nonfinite_initial_particles_are_reported():
    from paper_2310_01775_gb300 import stamp as S
    P = W.params("pusher1_h2")
    init, goal = W.scene(P, 0)
    theta0 = np.zeros((8, 12), dtype=np.float32)
    theta0[2, 1] = np.inf
    with pytest.raises(S.StampError) as e:
        gpu_solve(P, init, goal, 8, 2, 0, seed=0, theta0=theta0)
    assert e.value.status == S.STAMP_ENONFINITE


@pytest.mark.parametrize("name,N,dsvgd", [("pusher1_h4", 300, False), ("pusher1_h2", 32, True)])
def test_bandwidth_beside_the_rollouts_changes_nothing(name, N, dsvgd):
    """The solves compute each iteration's bandwidth on a second stream beside
    the rollouts; the result must be bit for bit the one-stream solve's."""
    from paper_2310_01775_gb300 import stamp as S
    P = W.params(name)
    init, goal = W.scene(P, 6)
    out = []
    for overlap in (True, False):
        prob = S.Problem(P, init, goal, N, torch.cuda.current_stream().cuda_stream)
        prob.set_overlap(overlap)
        prob.set_dsvgd(dsvgd)
        th = torch.zeros(N, prob.D, device="cuda")
        cost = torch.zeros(N, device="cuda")
        topk = np.zeros(3, dtype=np.int32)
        stats = np.zeros(40, dtype=np.float32)
        prob.solve(N, 30, 10, 11, P["lr"], None, th, cost, 3, topk, stats)
        prob.close()
        out.append((th, cost, topk, stats))
    (a, ca, ka, sa), (b, cb, kb, sb) = out
    assert torch.equal(a, b) and torch.equal(ca, cb)
    assert np.array_equal(ka, kb) and np.array_equal(sa, sb)
