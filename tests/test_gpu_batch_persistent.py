"""The persistent batched iteration (one launch per Stein iteration of every
instance, stamp_batch_set_persistent) on the GPU, through the C ABI.

It runs the same rollout, adjoint, median, Stein-direction and Adam bodies
as the per-class launches, compiled into one kernel, where the compiler may
fuse multiply-adds differently: its results are held to the FP64 oracle's
parity bar directly (gradients on conditioned particles, and the float32
floor over all of them, at the literal contact constants; particles after
three iterations with the softer contact), and to the per-class launches at
the same bar.  Graph replay equals direct launches bit for bit (the work
queue changes which CTA does an item, never the order of any sum), and its
bounded dependency wait is made to run out.
"""
import numpy as np
import pytest
import torch

from paper_2310_01775_gb300 import workloads as W

pytestmark = pytest.mark.gpu

SHAPES = [(1, 2, 37), (2, 3, 64), (3, 2, 100), (4, 2, 45), (1, 4, 200), (3, 3, 33), (4, 3, 130)]
LANES = {1: 2, 2: 4, 3: 8, 4: 8}                       # the persistent kernel's teams
CONFIG = {1: (64, 25), 2: (64, 5), 3: (128, 25), 4: (128, 1)}   # cta, C: segments and C = 1
SOFT = dict(k_contact=1e3, c_contact=10.0)


def _S():
    from paper_2310_01775_gb300 import stamp as S
    return S


def _instances(T=50, physics=None, shapes=SHAPES, scene0=40, seed0=1000):
    out = []
    for g, (nb, H, N) in enumerate(shapes):
        p = dict(physics or W.PHYSICS, n_blocks=nb, H=H, T=T)
        init, goal = W.scene(p, scene0 + g)
        out.append({"n_blocks": nb, "H": H, "N": N, "seed": seed0 + g, "init": init, "goal": goal})
    return out


def _batch(insts, T=50, persistent=True, physics=None):
    S = _S()
    b = S.Batch(dict(physics or W.PHYSICS, T=T), insts, torch.cuda.current_stream().cuda_stream)
    for nb in {d["n_blocks"] for d in insts}:
        cta, C = CONFIG[nb]
        b.set_config(nb, LANES[nb], cta, C)
    b.set_persistent(persistent)
    return b


def _theta(b, insts):
    out = []
    for g, d in enumerate(insts):
        x = torch.empty(d["N"], d["H"] * (4 * d["n_blocks"] + 2), device="cuda")
        b.read_theta(g, x)
        out.append(x)
    return out


def _f32(P):
    return {k: (float(np.float32(v)) if isinstance(v, float) else v) for k, v in P.items()}


def _grad_bar(insts, grads, phys, T, Cs, sample=None):
    """One iteration's gradients (iteration 0 from the initial draws) of
    each instance against the FP64 oracle with the rollout parity bar."""
    from oracle import stamp_oracle as O
    from _common import GRAD_TOL, Reference, rel_err
    for g, d in enumerate(insts):
        if sample is not None and g not in sample:
            continue
        P = _f32(dict(phys, n_blocks=d["n_blocks"], H=d["H"], T=T, ckpt_every=Cs[d["n_blocks"]]))
        init = np.asarray(d["init"], dtype=np.float32).astype(np.float64)
        goal = np.asarray(d["goal"], dtype=np.float32).astype(np.float64)
        M, _, D = O.dims(P)
        # all particles, or sample[g] of them spread over the instance's warps
        idx = (np.arange(d["N"]) if sample is None or g not in sample
               else np.unique(np.linspace(0, d["N"] - 1, min(sample[g], d["N"])).astype(int)))
        theta = O.init_theta(d["seed"], d["N"], D).astype(np.float32)[idx]
        gum = O.gumbel_noise(d["seed"], 0, d["N"], d["H"], M)[idx]
        ref = Reference(theta, P, init, goal, gum, C=P["ckpt_every"])
        eg = rel_err(grads[g].cpu().numpy()[idx], ref.grad)
        assert eg[ref.ok].max(initial=0) < GRAD_TOL, (g, eg[ref.ok].max(initial=0))
        assert np.median(eg) <= 3 * np.median(ref.floor_grad) + 1e-6, (g, np.median(eg))


def _grads(b, insts):
    out = []
    for g, d in enumerate(insts):
        x = torch.empty(d["N"], d["H"] * (4 * d["n_blocks"] + 2), device="cuda")
        b.read_grad(g, x)
        out.append(x)
    return out


def test_persistent_gradients_meet_the_oracle_bar():
    """Literal contact constants: every instance's first-iteration gradient
    against the oracle (a checkpointed and an interval-1 tape, every block
    count, instances over several rollout items)."""
    T = 50
    insts = _instances(T, shapes=[(1, 2, 37), (2, 3, 64), (3, 2, 40), (4, 2, 45), (1, 4, 200)])
    b = _batch(insts, T)
    b.solve(1, 1e-2)
    _grad_bar(insts, _grads(b, insts), W.PHYSICS, T, {nb: c[1] for nb, c in CONFIG.items()},
              sample={0: 37, 1: 64, 2: 40, 3: 45, 4: 40})
    b.close()


def test_persistent_matches_per_class_launches():
    """Softer contact, three iterations in each mode: particles to the bar
    the oracle comparison uses (1e-4), hard costs to 1e-4 relative, units
    exactly."""
    T, iters, lr = 50, 3, 1e-2
    phys = dict(W.PHYSICS, **SOFT)
    insts = _instances(T, phys)
    a, p = _batch(insts, T, False, phys), _batch(insts, T, True, phys)
    assert p.persistent()[0] and not a.persistent()[0]
    a.solve(iters, lr)
    p.solve(iters, lr)
    ra, rp = a.results(), p.results()
    for g, (x, y) in enumerate(zip(_theta(a, insts), _theta(p, insts))):
        assert float((x - y).abs().max()) <= 1e-4, (g, float((x - y).abs().max()))
        c = float(ra["best_cost"][g])
        assert abs(float(rp["best_cost"][g]) - c) <= 1e-4 * max(c, 1e-6), g
    assert ra["units"] == rp["units"]
    assert (rp["iterations"] == iters).all()
    a.close()
    p.close()


def test_persistent_iterations_match_the_oracle():
    """The persistent launch against the FP64 oracle directly: one instance
    of each block-count class (ragged particle counts, a checkpointed and an
    interval-1 tape), three iterations with the softer contact."""
    from oracle import stamp_oracle as O
    T, iters, lr = 50, 3, 1e-2
    phys = dict(W.PHYSICS, **SOFT)
    insts = _instances(T, phys, [(1, 2, 37), (2, 2, 33), (3, 2, 20), (4, 2, 12)], 60, 2000)
    b = _batch(insts, T, True, phys)
    b.solve(iters, lr)
    res = b.results()
    for g, (d, got) in enumerate(zip(insts, _theta(b, insts))):
        P = dict(phys, n_blocks=d["n_blocks"], H=d["H"], T=T, ckpt_every=25)
        init = np.asarray(d["init"], dtype=np.float32).astype(np.float64)
        goal = np.asarray(d["goal"], dtype=np.float32).astype(np.float64)
        ref = O.solve(P, init, goal, d["N"], iters, 0, d["seed"], lr, k=0)
        err = np.abs(got.cpu().numpy() - ref["theta"])
        assert err.max() <= 1e-4, (g, float(err.max()))
        c_ref = float(ref["cost_hard"].min())
        assert abs(res["best_cost"][g] - c_ref) <= 1e-4 * max(c_ref, 1e-6) + 1e-7, g
    b.close()


def test_persistent_graph_replay_is_bitwise_and_early_stop_freezes():
    T = 50
    insts = _instances(T)
    a, b = _batch(insts, T), _batch(insts, T)
    a.solve(9, 1e-2, target_cost=0.0, check_every=4, use_graph=True)
    b.solve(9, 1e-2, target_cost=0.0, check_every=4, use_graph=False)
    for g, (x, y) in enumerate(zip(_theta(a, insts), _theta(b, insts))):
        assert torch.equal(x, y), g
    assert np.array_equal(a.results()["best_cost"], b.results()["best_cost"])
    # early stop: instances below the target after the first check freeze there
    target = float(np.median(_first_check(insts, T)))
    a.solve(12, 1e-2, target_cost=target, check_every=4)
    res = a.results()
    stopped = res["seconds_to_target"] >= 0
    assert stopped.any() and not stopped.all()
    assert (res["iterations"][~stopped] == 12).all()
    g = int(np.nonzero(stopped & (res["iterations"] == 4))[0][0])
    b.solve(4, 1e-2)
    assert torch.equal(_theta(a, insts)[g], _theta(b, insts)[g])
    a.close()
    b.close()


def _first_check(insts, T):
    c = _batch(insts, T)
    c.solve(4, 1e-2, target_cost=0.0, check_every=4)
    out = c.results()["best_cost"].copy()
    c.close()
    return out


def test_persistent_wait_runs_out_then_recovers():
    """A dependency wait that nothing satisfies (the Stein items wait for one
    rollout warp more than exist, 2 ms limit): the launch drains its queue,
    the solve reports STAMP_ETIMEOUT, and the next solve equals a fresh one."""
    S = _S()
    T = 50
    insts = _instances(T)
    b, ref = _batch(insts, T), _batch(insts, T)
    b.inject_wait_timeout()
    with pytest.raises(S.StampError) as e:
        b.solve(3, 1e-2)
    assert e.value.status == S.STAMP_ETIMEOUT
    b.solve(3, 1e-2)
    ref.solve(3, 1e-2)
    for g, (x, y) in enumerate(zip(_theta(b, insts), _theta(ref, insts))):
        assert torch.equal(x, y), g
    b.close()
    ref.close()


def test_autotune_times_both_modes_and_keeps_the_faster():
    insts = _instances(50)
    b = _batch(insts, 50, persistent=False)
    b.solve(0, 1e-2)                            # the initial draws
    th0 = _theta(b, insts)
    b.autotune(1)
    on, ms_a, ms_p = b.persistent()
    assert ms_a > 0 and ms_p > 0 and on == (ms_p < ms_a)
    for x, y in zip(th0, _theta(b, insts)):     # the particles are put back
        assert torch.equal(x, y)
    b.solve(3, 1e-2)
    assert np.isfinite(b.results()["best_cost"]).all()
    b.close()


def test_full_size_persistent_gradients_sampled():
    """The 256 uneven instances of the serving workload (1-4 blocks, H 2-8,
    N 64-1024, T = 100, interval-1 tapes) in one persistent launch, with
    the softer contact (at T = 100 few particles of the literal constants
    are conditioned; those are covered above at T = 50): for the first
    two-action instance of each block count, particles spread over its
    warps against the oracle with the parity bar."""
    phys = dict(W.PHYSICS, **SOFT)
    insts = W.batch_instances(256, 0)
    b = _batch(insts, 100, True, phys)
    for nb in range(1, 5):
        b.set_config(nb, LANES[nb], 128, 1)
    b.solve(1, 1e-2)
    pick = {}
    for g, d in enumerate(insts):
        if d["H"] == 2:
            pick.setdefault(d["n_blocks"], g)
    assert len(pick) == 4
    _grad_bar(insts, _grads(b, insts), phys, 100, {nb: 1 for nb in range(1, 5)},
              sample={g: (8 if nb == 4 else 12) for nb, g in pick.items()})
    b.close()


def test_trace_records_every_item_in_dependency_order():
    """stamp_batch_set_trace: every work item of the last launch is recorded
    once, with claim <= dependencies met <= end; a median pass, Stein block
    or Adam chunk starts only after its instance's earlier items, so each
    kind's first start follows the first end of the kind it waits on."""
    insts = _instances(50)
    b = _batch(insts, 50)
    b.set_trace(True)
    b.solve(2, 1e-2, use_graph=True)
    tr = b.read_trace()
    n = len(tr["kind"])
    assert n > 0 and np.array_equal(np.sort(tr["item"]), np.arange(n))
    assert (tr["claim"] >= 0).all() and (tr["start"] >= tr["claim"]).all()
    assert (tr["end"] >= tr["start"]).all()
    first_end = {k: tr["end"][tr["kind"] == k].min() for k in set(tr["kind"])}
    first_start = {k: tr["start"][tr["kind"] == k].min() for k in set(tr["kind"])}
    for later, earlier in (("median1", "pairwise"), ("median2", "median1"), ("stein", "median2"),
                           ("stein", "rollout"), ("adam", "stein")):
        assert first_start[later] >= first_end[earlier], (later, earlier)
    assert set(np.unique(tr["sm"])) <= set(range(1024))
    b.set_trace(False)
    b.close()


def test_persistent_largest_parameter_count_matches_per_class():
    """A 4-block, 16-action instance (D = 288: the Stein blocks' widest
    column layout and the largest shared-memory plan) beside a small one,
    softer contact, two iterations in each mode: particles to 1e-4."""
    T, iters, lr = 50, 2, 1e-2
    phys = dict(W.PHYSICS, **SOFT)
    insts = _instances(T, phys, [(4, 16, 40), (1, 2, 33)], 80, 3000)
    a, p = _batch(insts, T, False, phys), _batch(insts, T, True, phys)
    a.solve(iters, lr)
    p.solve(iters, lr)
    for g, (x, y) in enumerate(zip(_theta(a, insts), _theta(p, insts))):
        assert x.shape[1] == (288 if g == 0 else 12)
        assert float((x - y).abs().max()) <= 1e-4, (g, float((x - y).abs().max()))
    a.close()
    p.close()
