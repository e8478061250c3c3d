"""Write tests/golden/solve_*.json: whole-solve results of the FP64 oracle.

Calls only oracle/ (and the seeded scene generator).  For each seed: the
top-k particles and their discrete plans, the five best distinct plans with
their hard costs, and the minimum relaxed cost of every iteration.  The
stiff-contact workload is also solved by the oracle in float32, which
calibrates how much a float32 solve can differ from the float64 one.

    python tests/golden/make_solve_golden.py
"""
from __future__ import annotations

import json
import multiprocessing as mp
import os
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

SOFT = dict(k_contact=1e3, c_contact=10.0)
JOBS = ([("soft", s, "f64") for s in range(4)]
        + [("stiff", s, dt) for s in range(10) for dt in ("f64", "f32")])


def summarise(r, P):
    import numpy as np
    from oracle import stamp_oracle as O
    codes = O.plan_codes(r["theta"], P)
    c = r["cost_hard"]
    best = {}
    for i in np.lexsort((np.arange(len(c)), c)):
        best.setdefault(tuple(int(x) for x in codes[i]), float(c[i]))
    top = sorted(best.items(), key=lambda kv: kv[1])[:5]
    return dict(topk=[int(i) for i in r["topk"]],
                topk_plans=[[int(x) for x in codes[i]] for i in r["topk"] if i >= 0],
                top5=[[list(k), v] for k, v in top],
                min_cost=[float(x) for x in r["min_cost"]])


def run(job):
    import torch
    from oracle import stamp_oracle as O
    from paper_2310_01775_gb300 import workloads as W
    kind, seed, dt = job
    P = W.params("pusher1_h2", **(SOFT if kind == "soft" else {}))
    init, goal = W.scene(P, seed)
    torch.set_num_threads(1)
    r = O.solve(P, init, goal, P["N"], P["svgd_iters"], 0, seed, P["lr"], k=3,
                dtype=torch.float64 if dt == "f64" else torch.float32)
    return job, summarise(r, P)


if __name__ == "__main__":
    with mp.get_context("spawn").Pool(min(len(JOBS), os.cpu_count() or 1)) as pool:
        results = pool.map(run, JOBS)
    for kind in ("soft", "stiff"):
        out = {"workload": "pusher1_h2" + (" with k_contact=1e3, c_contact=10" if kind == "soft" else ""),
               "N": 32, "svgd_iters": 200, "seeds": {}}
        for (k, seed, dt), summ in results:
            if k == kind:
                out["seeds"].setdefault(str(seed), {})[dt] = summ
        with open(os.path.join(HERE, f"solve_pusher1_h2_{kind}.json"), "w") as f:
            json.dump(out, f, indent=1)
    print("wrote", [f"solve_pusher1_h2_{k}.json" for k in ("soft", "stiff")])
