"""Throughput of STAMP's hot path on GB300: particle rollout+adjoint steps/s.

One step = one stamp_solve call: Algorithm 1 over the workload's particles
(every SVGD iteration = Gumbel-relaxed forward rollout, checkpointed adjoint,
median bandwidth, Stein direction, Adam), then the hard evaluation and the
distinct-plan top-k.  One unit = one particle advanced one substep forward and
back, so a step is N*H*T*iterations units.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--workload NAME]
    python bench.py --impl reference     # the FP64 CPU oracle on a bounded sample

Under torchrun every rank solves its own seeded instance (no collective on the
data path: the instances are independent); value = all ranks' units divided
by the slowest rank's time.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "particle rollout+adjoint steps/s"
UNIT = "particle-substeps/s"
# Algorithmic FLOPs per unit (one particle, one substep), counted over the
# oracle's own operations (oracle/flops.py): forward, reverse sweep.
FLOPS_PER_UNIT = {1: (447.2, 863.2), 2: (2544.4, 5005.0), 3: (6293.5, 12860.9),
                  4: (11694.7, 24711.2)}
FP32_LANES = 128                    # FP32 lanes per SM; 1 FMA = 2 FLOP
# DRAM bytes (read + write) per launch of a rollout kernel (for the reverse
# sweep: its replay and sweep launches together), from one cold-cache ncu
# capture of the workload, valid while the kernel sources are unchanged
# (sha256 prefix over the rollout sources at capture time).
TRAFFIC = {("pusher3_h6", "rollout_adj"): ("243c7f35e3b01a4a", 179.97e6)}   # replay + sweep
ROLLOUT_SOURCES = ("rollout.cuh", "adjoint_time.cu")


def peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        with open(path) as f:
            d = json.load(f)
        return d.get("sm_max_mhz", 2070.0), d.get("hbm_gbs", 6775.6), "measured"
    return 2070.0, 6800.0, "fallback"


def rollout_source_hash():
    h = hashlib.sha256()
    for name in ROLLOUT_SOURCES:
        path = os.path.join(ROOT, "paper_2310_01775_gb300", "csrc", name)
        if os.path.exists(path):
            h.update(open(path, "rb").read())
    return h.hexdigest()[:16]


def fp32_peak(local):
    """Measured FP32 FMA roof (the library's microbenchmark) with the SM
    clocks sampled while it runs."""
    from paper_2310_01775_gb300 import stamp as S
    clk = Clocks(local)
    tflops, ms = S.stamp_fp32_fma_peak(40)
    c = clk.stop()
    return tflops, ms, c


class Clocks:
    """nvidia-smi sampling of SM clocks and throttle reasons while timing."""
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu: int):
        self.gpu = gpu
        self.f = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)
        try:
            self.p = subprocess.Popen(["nvidia-smi", "-i", str(gpu), f"--query-gpu={self.Q}",
                                       "--format=csv,noheader,nounits", "-lms", "200"],
                                      stdout=self.f, stderr=subprocess.DEVNULL)
        except OSError:
            self.p = None

    def stop(self):
        if self.p is None:
            return None
        self.p.terminate()
        self.p.wait()
        self.f.seek(0)
        rows = [r.split(", ") for r in self.f.read().strip().splitlines() if r.count(",") >= 8]
        os.unlink(self.f.name)
        if not rows:
            return None
        sm = [float(r[1]) for r in rows]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({n for r in rows for n, v in zip(names, r[5:9]) if v.strip() == "Active"})
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": float(rows[0][2]),
                "reasons": reasons, "samples": len(rows)}


def cpu_oracle_sample(P, init, goal, seed, n_particles, iters=1, actions=None):
    """Time the FP64 oracle on a bounded sample: n_particles of the workload,
    `iters` iterations of rollout + reverse sweep + Stein step over the first
    `actions` pushes of the plan (all H by default)."""
    import torch
    from oracle import stamp_oracle as O
    if actions:
        P = dict(P, H=min(actions, P["H"]))
    M, _, D = O.dims(P)
    th = O.init_theta(seed, n_particles, D)
    m = np.zeros_like(th)
    v = np.zeros_like(th)
    t0 = time.perf_counter()
    for it in range(iters):
        gum = O.gumbel_noise(seed, it, n_particles, P["H"], M)
        _, g = O.rollout_grad(th, P, init, goal, gum)
        th, m, v, _, _ = O.svgd_step(th, g, m, v, it + 1, P["lr"])
    dt = time.perf_counter() - t0
    units = n_particles * P["H"] * P["T"] * iters
    return units / dt, dt, torch.get_num_threads()


def run_reference(args, P, world, rank):
    """The reference arm: the oracle as it stands on the host cores."""
    if rank != 0:
        return
    init, goal = __import__("paper_2310_01775_gb300.workloads", fromlist=["W"]).scene(P, args.seed)
    n, acts = args.ref_particles, min(args.ref_actions, P["H"])
    for _ in range(args.warmup):
        cpu_oracle_sample(P, init, goal, args.seed, max(2, n // 8), actions=1)
    times, vals = [], []
    for s in range(args.steps):
        v, dt, cores = cpu_oracle_sample(P, init, goal, args.seed + s, n, actions=acts)
        times.append(dt)
        vals.append(v)
    units = n * acts * P["T"]
    value = units * len(times) / sum(times)
    sample = (f"{n} of {P['N']} particles, the first {acts} of {P['H']} pushes "
              f"({acts * P['T']} substeps), 1 iteration per step")
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": 1e3 * sum(times) / len(times), "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": workload_config(args, P),
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle",
                             "sample": sample},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def surrogate_vs_plain(stream, seeds=(3, 4, 5)):
    """Time to cost < 1e-3 on planted 3-block problems (H=6, T=100, N=2048):
    plain SVGD (500 iterations) against the surrogate-assisted solve (surrogate
    trained on 2^20 simulator transitions; 131072 candidates screened to 2048;
    300 surrogate + 200 simulator iterations), both stopping at the target
    (hard simulator check every 10 iterations).  Also the time the surrogate
    arm needs to reach the cost plain SVGD ends at."""
    import torch
    from paper_2310_01775_gb300 import surrogate_compare as SC
    from paper_2310_01775_gb300 import workloads as W
    P = W.params("pusher3_h6")
    sur, train_s, losses = SC.train_surrogate(P, 1 << 20, stream, 131072, P["N"])
    res = SC.compare(P, seeds, sur, N=P["N"], n_candidates=131072, surrogate_iters=300,
                     sim_iters=200, stream=stream)
    # time for the surrogate arm to reach plain SVGD's final cost
    match = []
    for row in res["per_seed"]:
        r = SC.compare(P, (row["seed"],), sur, N=P["N"], n_candidates=131072, surrogate_iters=300,
                       sim_iters=200, target=row["plain"]["best_cost"] * (1 + 1e-6),
                       stream=stream)["per_seed"][0]
        match.append({"seed": row["seed"], "plain_final_cost": row["plain"]["best_cost"],
                      "plain_seconds": row["plain"]["seconds"],
                      "surrogate_seconds": r["surrogate"]["seconds"],
                      "surrogate_iterations": r["surrogate"]["iterations"],
                      "reached": r["surrogate"]["reached"]})
    sur.close()
    arms = {}
    for arm in ("plain", "surrogate"):
        rows = [r[arm] for r in res["per_seed"]]
        arms[arm] = {"reached_target": f"{sum(r['reached'] for r in rows)}/{len(rows)}",
                     "seconds": [r["seconds"] for r in rows],
                     "iterations": [r["iterations"] for r in rows],
                     "best_cost": [r["best_cost"] for r in rows]}
    return {"problem": "planted 3-block scenes (pusher3_h6 physics; goal = hard rollout of a "
                       "random plan), N=2048, lr 1e-2, seeds " + ",".join(map(str, seeds)),
            "target_cost": 1e-3, "surrogate_training": {
                "transitions": 1 << 20, "seconds": round(train_s, 3),
                "final_standardized_mse": float(losses[-1])},
            "plain": arms["plain"], "surrogate": arms["surrogate"],
            "time_to_plain_final_cost": match}


def batched_serving(stream, peak_tflops, peak_src, n=256, iters=500, target=1e-3, check_every=10,
                    screen=True, seed=0):
    """256 seeded uneven instances (1-4 blocks, H 2-8, N log-uniform 64-1024,
    T=100; goals planted: the end poses of a hard rollout of a random plan)
    solved together: autotuned launch configuration and launch mode (per-class
    launches or one persistent launch per iteration; both timed), graph-replayed
    iterations, per-instance early stop at the target (hard simulator check
    every 10 iterations), at most 500 iterations; then the same batch with
    surrogate screening (batched_screened)."""
    import torch
    from paper_2310_01775_gb300 import stamp as S
    from paper_2310_01775_gb300 import workloads as W
    insts = W.batch_instances(n, seed)
    for g, d in enumerate(insts):   # plant each goal
        P = dict(W.PHYSICS, n_blocks=d["n_blocks"], H=d["H"], T=100, ckpt_every=100)
        D = d["H"] * (4 * d["n_blocks"] + 2)
        prob = S.Problem(P, d["init"], d["init"], 1, stream)
        plan = torch.tensor(3.0 * W.random_theta(1, D, 9000 + 1000 * seed + g), device="cuda")
        c = torch.empty(1, device="cuda")
        fin = torch.empty(1, 6 * d["n_blocks"], device="cuda")
        prob.rollout_fwd(plan, 1, 0, -1, 1, c, fin)
        prob.sync()
        d["goal"] = fin.cpu().numpy().reshape(d["n_blocks"], 6)[:, :3].astype(np.float64)
        prob.close()
    b = S.Batch(dict(W.PHYSICS, T=100), insts, stream)
    t0 = time.perf_counter()
    b.autotune(2)
    tune_s = time.perf_counter() - t0
    cfg = {str(nb): dict(zip(("lanes", "cta", "ckpt_every"), b.get_config(nb))) for nb in range(1, 5)}
    persistent, tune_ms_a, tune_ms_p = b.persistent()
    # both launch modes over 20 graph-replayed iterations of every instance
    # (no early-stop checks; the second of two solves, after the capture)
    mode_ms = {}
    for name, flag in (("per_class", False), ("persistent", True)):
        b.set_persistent(flag)
        for _ in range(2):
            b.solve(20, 1e-2, 0.0, 0, True)
        mode_ms[name] = b.results()["seconds"] / 20 * 1e3
    b.set_persistent(persistent)
    b.solve(iters, 1e-2, target, check_every, True)
    r = b.results()
    stopped = r["seconds_to_target"] >= 0
    tts = np.sort(r["seconds_to_target"][stopped])
    # FP32-ALU roofline of the whole batch: the oracle's FLOPs per unit of each
    # block count (forward + reverse) over the units each instance ran
    flops = sum(int(r["iterations"][g]) * d["N"] * d["H"] * 100 * sum(FLOPS_PER_UNIT[d["n_blocks"]])
                for g, d in enumerate(insts))
    peak = peak_tflops
    ach = flops / r["seconds"] / 1e12
    done = np.where(stopped, r["seconds_to_target"], r["seconds"])
    b.close()
    pct = lambda a, q: float(np.percentile(a, q)) if len(a) else None
    screened = (batched_screened(insts, cfg, persistent, stream, iters, target, check_every,
                                 r["seconds_to_target"]) if screen else None)
    return {"instances": n, "particles": int(sum(d["N"] for d in insts)),
            "units_per_iteration_all_active": int(sum(d["N"] * d["H"] * 100 for d in insts)),
            "value": r["units"] / r["seconds"], "unit": UNIT, "seconds": r["seconds"],
            "autotune_seconds": round(tune_s, 3), "config_per_block_count": cfg,
            "launch_mode": "persistent" if persistent else "per-class",
            "ms_per_iteration_all_active": {
                "per_class": mode_ms["per_class"], "persistent": mode_ms["persistent"],
                "autotune_per_class": tune_ms_a, "autotune_persistent": tune_ms_p,
                "over": "20 graph-replayed iterations of every instance, solve wall time incl. "
                        "initialisation and final evaluation / 20"},
            "target_cost": target, "reached": int(stopped.sum()),
            "time_to_solution_s": {"p50": pct(tts, 50), "p99": pct(tts, 99),
                                   "over": "instances that reached the target"},
            "time_to_stop_s": {"p50": pct(done, 50), "p99": pct(done, 99),
                               "over": "all instances (unreached: the solve's end)"},
            "median_iterations": float(np.median(r["iterations"])),
            "roofline": {"bound": "alu", "achieved": ach, "peak": peak, "unit": "TFLOP/s",
                         "frac": ach / peak, "over": "the whole solve (all kernels, checks included)",
                         "peak_source": peak_src},
            "surrogate_screened": screened,
            "small_requests": small_requests(stream)}


def small_requests(stream, n=512, N=32, iters=40):
    """Many small requests: n seeded instances of N particles each (1-4
    blocks, H 2-4, T=100) -- the latency-bound end of serving.  Autotuned
    launch configuration and mode; milliseconds per graph-replayed iteration
    of every instance in both launch modes."""
    from paper_2310_01775_gb300 import stamp as S
    from paper_2310_01775_gb300 import workloads as W
    rng = np.random.default_rng(np.random.SeedSequence([0, 0x5A11]))
    insts = []
    for g in range(n):
        nb, H = int(rng.integers(1, 5)), int(rng.integers(2, 5))
        init, goal = W.scene(dict(W.PHYSICS, n_blocks=nb, H=H, T=100), 30011 + g)
        insts.append({"n_blocks": nb, "H": H, "N": N, "seed": 50021 + g, "init": init, "goal": goal})
    b = S.Batch(dict(W.PHYSICS, T=100), insts, stream)
    b.autotune(2)
    persistent, _, _ = b.persistent()
    ms = {}
    for name, flag in (("per_class", False), ("persistent", True)):
        b.set_persistent(flag)
        for _ in range(2):
            b.solve(iters, 1e-2, 0.0, 0, True)
        ms[name] = b.results()["seconds"] / iters * 1e3
    units = sum(d["N"] * d["H"] * 100 for d in insts)
    b.close()
    return {"instances": n, "particles_each": N, "launch_mode": "persistent" if persistent else "per-class",
            "ms_per_iteration_all_active": ms,
            "value": units / (min(ms.values()) / 1e3), "unit": UNIT,
            "over": f"{iters} graph-replayed iterations, solve wall time incl. initialisation and "
                    f"final evaluation / {iters}"}


def batched_screened(insts, cfg, persistent, stream, iters, target, check_every, plain_tts,
                     factor=64):
    """The same batch with surrogate screening: one surrogate per block count
    of 1-3 (trained on 2^20 simulator transitions of T=100 pushes; horizon up
    to 8), each instance of 1-3 blocks starting from the N of 64 N draws of
    lowest surrogate cost (4-block instances, which no surrogate models,
    start from their plain draws); same launch configuration, iterations,
    target and checks as the plain batch."""
    from paper_2310_01775_gb300 import stamp as S
    from paper_2310_01775_gb300 import surrogate_compare as SC
    from paper_2310_01775_gb300 import workloads as W
    max_n = max(d["N"] for d in insts)
    surs, train_s = {}, 0.0
    for nb in (1, 2, 3):
        P = dict(W.PHYSICS, n_blocks=nb, H=8, T=100, ckpt_every=25)
        surs[nb], secs, _ = SC.train_surrogate(P, 1 << 20, stream, factor * max_n, max_n)
        train_s += secs
    b = S.Batch(dict(W.PHYSICS, T=100), insts, stream)
    for nb, c in cfg.items():
        b.set_config(int(nb), c["lanes"], c["cta"], c["ckpt_every"])
    b.set_persistent(persistent)
    t0 = time.perf_counter()
    for g, d in enumerate(insts):
        if d["n_blocks"] in surs:
            b.screen(surs[d["n_blocks"]], g, factor * d["N"])
    screen_s = time.perf_counter() - t0
    b.solve(iters, 1e-2, target, check_every, True)
    r = b.results()
    b.close()
    for sur in surs.values():
        sur.close()
    stopped = r["seconds_to_target"] >= 0
    tts = np.sort(r["seconds_to_target"][stopped] + screen_s)
    pct = lambda a, q: float(np.percentile(a, q)) if len(a) else None
    both = stopped & (plain_tts >= 0)
    faster = int(np.sum(r["seconds_to_target"][both] + screen_s < plain_tts[both]))
    return {"reached": int(stopped.sum()), "reached_by_block_count": {
                str(nb): f"{int(sum(stopped[g] for g, d in enumerate(insts) if d['n_blocks'] == nb))}"
                         f"/{sum(1 for d in insts if d['n_blocks'] == nb)}" for nb in range(1, 5)},
            "reached_by_both_arms": int(both.sum()),
            "faster_than_plain_on_both_reached": faster,
            "time_to_solution_both_reached_s": {
                "screened_p50": pct(r["seconds_to_target"][both] + screen_s, 50),
                "plain_p50": pct(plain_tts[both], 50)},
            "seconds": r["seconds"], "screening_seconds": round(screen_s, 3),
            "surrogate_training_seconds": round(train_s, 3),
            "time_to_solution_s": {"p50": pct(tts, 50), "p99": pct(tts, 99),
                                   "over": "instances that reached the target, screening included"},
            "median_iterations": float(np.median(r["iterations"]))}


def workload_config(args, P):
    iters = P["svgd_iters"]
    return {"workload": (f"{args.workload}: {P['n_blocks']} block(s), H={P['H']}, T={P['T']}, "
                         f"N={P['N']}, D={P['H'] * (4 * P['n_blocks'] + 2)}, {iters} SVGD "
                         f"iterations + hard evaluation + top-3 per step"),
            "ckpt_every": P["ckpt_every"], "l2_flush": "256 MiB write between steps",
            "units_per_step": P["N"] * P["H"] * P["T"] * iters}


def time_solves(prob, P, N, seed, steps, warmup, flush, stream):
    """Per-step device times (ms) of `steps` solves after `warmup` untimed
    ones; CUDA events on the problem's stream, L2 flushed between steps."""
    import torch
    iters = P["svgd_iters"]
    th = torch.empty(N, prob.D, device="cuda")
    cost = torch.empty(N, device="cuda")
    topk = np.zeros(3, dtype=np.int32)
    for s in range(warmup):
        prob.solve(N, iters, 0, seed + s, P["lr"], None, th, cost, 3, topk, None)
    evs = []
    for s in range(steps):
        flush.fill_(float(s))
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        prob.solve(N, iters, 0, seed + warmup + s, P["lr"], None, th, cost, 3, topk, None)
        b.record(stream)
        evs.append((a, b))
    torch.cuda.synchronize()
    return [a.elapsed_time(b) for a, b in evs]


def secondary_workload(name, seed, flush, stream, steps=5, warmup=3):
    """The same measurement on another workload (fewer steps), for context."""
    from paper_2310_01775_gb300 import stamp as S
    from paper_2310_01775_gb300 import workloads as W
    P = W.params(name)
    init, goal = W.scene(P, seed)
    prob = S.Problem(P, init, goal, P["N"], stream.cuda_stream)
    ms = time_solves(prob, P, P["N"], seed, steps, warmup, flush, stream)
    units = P["N"] * P["H"] * P["T"] * P["svgd_iters"]
    mode = {S.STAMP_ADJ_TIME_PARALLEL: "time-parallel", S.STAMP_ADJ_REPLAY: "segment replay + sequential",
            S.STAMP_ADJ_SEQUENTIAL: "sequential"}[prob.adjoint_mode(P["N"])]
    prob.close()
    return {"workload": f"{name}: {P['n_blocks']} block(s), H={P['H']}, T={P['T']}, N={P['N']}, "
                        f"C={P['ckpt_every']}, {P['svgd_iters']} SVGD iterations per step",
            "value": units * steps / (sum(ms) / 1e3), "unit": UNIT, "steps": steps,
            "ms_per_step": sum(ms) / steps, "reverse_sweep": mode}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--workload", default="pusher3_h6")
    ap.add_argument("--secondary", default="pusher1_h4",
                    help="a second workload measured with fewer steps ('' to skip)")
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--seed", type=int, default=0)
    ap.add_argument("--ref-particles", type=int, default=32)
    ap.add_argument("--ref-actions", type=int, default=1,
                    help="pushes of the plan in each reference-arm sample")
    ap.add_argument("--baseline-particles", type=int, default=32)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--lanes", type=int, nargs=2, default=None)
    ap.add_argument("--ckpt", type=int, default=None, help="checkpoint interval override")
    ap.add_argument("--no-surrogate", action="store_true",
                    help="skip the surrogate-assisted vs plain SVGD comparison")
    ap.add_argument("--no-batched", action="store_true",
                    help="skip the 256-instance batched serving run")
    ap.add_argument("--no-variants", action="store_true",
                    help="skip the SVGD / SVGD+SGD / DSVGD cost-evolution comparison")
    args = ap.parse_args()

    from paper_2310_01775_gb300 import workloads as W
    P = W.params(args.workload, **({"ckpt_every": args.ckpt} if args.ckpt else {}))
    from paper_2310_01775_gb300 import replicas as R
    world, rank, local = R.init() if args.impl == "ours" else R.env()
    if args.impl == "reference":
        run_reference(args, P, world, rank)
        return

    import torch
    from paper_2310_01775_gb300 import stamp as S
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    stream = torch.cuda.current_stream()
    seed = R.rank_seed(args.seed, rank)
    init, goal = W.scene(P, seed)
    N, H, T, iters = P["N"], P["H"], P["T"], P["svgd_iters"]
    prob = S.Problem(P, init, goal, N, stream.cuda_stream)
    if args.lanes:
        prob.set_lanes(*args.lanes)
    D = prob.D
    th = torch.empty(N, D, device=dev)
    cost = torch.empty(N, device=dev)
    topk = np.zeros(3, dtype=np.int32)
    flush = torch.empty(256 * 1024 * 1024 // 4, device=dev)
    units = N * H * T * iters

    def step(s):
        prob.solve(N, iters, 0, seed + s, P["lr"], None, th, cost, 3, topk, None)

    for s in range(args.warmup):
        step(s)
    # one untimed step with events around every launch: the per-kernel
    # breakdown and the dominant kernel
    prob.set_profiling(True)
    step(args.warmup)
    torch.cuda.synchronize()
    kt_all = prob.kernel_times()
    prob.set_profiling(False)
    dom = max(kt_all, key=lambda k: kt_all[k][0])
    # timed region: per-step CUDA events on the problem's stream, L2 flushed
    # in between, no events inside the solves
    R.barrier()
    torch.cuda.synchronize()
    clk = Clocks(local)
    evs = []
    for s in range(args.steps):
        flush.fill_(float(s))
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        step(args.warmup + 1 + s)
        b.record(stream)
        evs.append((a, b))
    torch.cuda.synchronize()
    clocks = clk.stop()
    ms = sum(a.elapsed_time(b) for a, b in evs)
    ms_max = R.max_over_ranks(ms, device=dev)
    R.barrier()
    value = R.throughput(units * args.steps, world, ms_max)
    # the dominant kernel's launch time: one more step of the same solve with
    # events around that kernel's launches only
    prob.set_profiling_kernels([dom])
    flush.fill_(-1.0)
    step(args.warmup + 1 + args.steps)
    torch.cuda.synchronize()
    kt = prob.kernel_times()
    prob.set_profiling(False)

    # end to end through the public call with host buffers (pinned)
    th_h = torch.empty(N, D, pin_memory=True)
    th0_h = torch.tensor(W.random_theta(N, D, seed), dtype=torch.float32).pin_memory()
    cost_h = torch.empty(N, pin_memory=True)
    e2e_t = []
    for s in range(2):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        prob.solve(N, iters, 0, seed + s, P["lr"], th0_h, th_h, cost_h, 3, topk, None)
        e2e_t.append(time.perf_counter() - t0)
    e2e = {"value": units / min(e2e_t), "unit": UNIT, "h2d_bytes_per_step": N * D * 4,
           "d2h_bytes_per_step": N * D * 4 + N * 4 + 3 * 4}

    if rank != 0:
        prob.close()
        R.finish()
        return

    # kernels per recorded launch of the reverse sweep
    adj_mode = prob.adjoint_mode(N)
    per_rec = {"rollout_adj": prob.adjoint_launches(N)}
    gpu_launches = int(sum(n * per_rec.get(k, 1) for k, (_, n) in kt_all.items())) * args.steps
    # roofline of the dominant kernel: FP32-ALU bound, FLOPs from the oracle's
    # count, against the measured FMA roof
    peak_tflops, peak_ms, peak_clocks = fp32_peak(local)
    peak_src = (f"measured: independent fmaf chains on every SM, {peak_ms:.3f} ms per launch, "
                f"SM clock {peak_clocks['sm_mhz'] if peak_clocks else 'unsampled'} MHz")
    fpu = FLOPS_PER_UNIT.get(P["n_blocks"])
    roof = None
    if fpu and dom in ("rollout_fwd", "rollout_adj") and kt[dom][1]:
        per_launch_ms = kt[dom][0] / kt[dom][1]
        flops = (fpu[0] if dom == "rollout_fwd" else fpu[1]) * N * H * T
        ach = flops / (per_launch_ms / 1e3) / 1e12
        rec = TRAFFIC.get((args.workload, dom))
        traffic = rec[1] if rec and rec[0] == rollout_source_hash() else None
        roof = {"bound": "alu", "kernel": dom, "achieved": ach, "peak": peak_tflops,
                "unit": "TFLOP/s", "frac": ach / peak_tflops, "traffic": traffic,
                "peak_source": peak_src, "ms_per_launch": per_launch_ms,
                "flop_per_unit": fpu[0] if dom == "rollout_fwd" else fpu[1],
                "units_per_launch": N * H * T,
                "share_of_step": kt_all[dom][0] / sum(v[0] for v in kt_all.values())}
    cpu = None
    if not args.no_cpu_baseline:
        v, dt, cores = cpu_oracle_sample(P, init, goal, seed, args.baseline_particles)
        cpu = {"value": v, "unit": UNIT, "cores": cores, "kind": "oracle",
               "sample": f"{args.baseline_particles} of {N} particles, all {H} pushes, "
                         f"1 iteration ({dt:.1f} s)"}
    sec = secondary_workload(args.secondary, seed, flush, stream) if args.secondary else None
    sur = bat = None
    if world == 1 and not args.no_surrogate:
        sur = surrogate_vs_plain(stream.cuda_stream)
    if world == 1 and not args.no_batched:
        bat = batched_serving(stream.cuda_stream, peak_tflops, peak_src)
    var = None
    if world == 1 and not args.no_variants:
        from paper_2310_01775_gb300 import variants as V
        var = V.cost_evolution("pusher1_h4", (0, 1, 2, 3, 4), stream=stream.cuda_stream)
    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms_max / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": dict(workload_config(args, P),
                           reverse_sweep={S.STAMP_ADJ_TIME_PARALLEL: "time-parallel",
                                          S.STAMP_ADJ_REPLAY: "segment replay + sequential",
                                          S.STAMP_ADJ_SEQUENTIAL: "sequential"}.get(adj_mode, str(adj_mode))),
            "roofline": roof, "cpu_baseline": cpu,
            "clocks": clocks, "e2e": e2e,
            "gpu_launches": gpu_launches,
            "kernels_ms_one_step": {k: round(v[0], 3) for k, v in kt_all.items() if v[1]},
            "secondary": sec,
            "surrogate_vs_plain": sur, "batched_serving": bat, "solver_variants": var}
    print(json.dumps(line), flush=True)
    prob.close()
    R.finish()


if __name__ == "__main__":
    main()
