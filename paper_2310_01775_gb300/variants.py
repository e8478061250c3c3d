"""The paper's solver variants on one workload, through the C ABI.

Sec. IV-C / Algorithm 1 run SVGD until convergence and then refine with SGD
(the repulsive term can hold plans away from optima; Sec. V shows the cost
evolution of both).  This runs, on the same seeded problems and the same
total iteration budget:
  * "svgd":        SVGD for every iteration;
  * "svgd+sgd":    SVGD, then plain-gradient (SGD-phase) iterations;
  * "dsvgd":       SVGD with the importance weights of Eq. dsvgd;
  * "dsvgd+sgd":   the weighted SVGD, then SGD;
  * "structured", "structured+sgd": SVGD with the structured kernel of
    App. D.3 (restated: per-action RBFs on the push parameters and on the
    choice probabilities), without and with the SGD refinement;
and reports per variant the lowest relaxed cost at a few iterations (the
cost-evolution curve), the final lowest hard cost and the wall time.
"""
from __future__ import annotations

import time

import numpy as np
import torch

from . import stamp as S
from . import workloads as W

# name: (DSVGD weights, SGD refinement, structured kernel)
VARIANTS = {"svgd": (False, False, 0), "svgd+sgd": (False, True, 0), "dsvgd": (True, False, 0),
            "dsvgd+sgd": (True, True, 0), "structured": (False, False, 1),
            "structured+sgd": (False, True, 1)}


def cost_evolution(name: str, seeds, iters: int = 500, sgd_iters: int = 200,
                   marks=(50, 100, 200, 300, 400, 500), stream=None) -> dict:
    P = W.params(name)
    N = P["N"]
    out = {}
    for var, (weighted, refine, kind) in VARIANTS.items():
        curves, finals, secs = [], [], []
        for seed in seeds:
            init, goal = W.scene(P, seed)
            prob = S.Problem(P, init, goal, N, stream)
            prob.set_dsvgd(weighted)
            prob.set_svgd_kernel(kind)
            th = torch.empty(N, prob.D, device="cuda")
            cost = torch.empty(N, device="cuda")
            stats = np.zeros(iters, dtype=np.float32)
            n_sgd = sgd_iters if refine else 0
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            prob.solve(N, iters - n_sgd, n_sgd, seed, P["lr"], None, th, cost, 0, None, stats)
            secs.append(time.perf_counter() - t0)
            curves.append(np.minimum.accumulate(stats))
            finals.append(float(cost.min()))
            prob.close()
        c = np.stack(curves)
        out[var] = {"min_relaxed_cost_at": {str(m): float(np.mean(c[:, m - 1])) for m in marks if m <= iters},
                    "final_hard_cost": finals, "mean_final_hard_cost": float(np.mean(finals)),
                    "seconds": float(np.mean(secs))}
    return {"workload": name, "seeds": list(seeds), "iterations": iters, "sgd_iters": sgd_iters,
            "variants": out}
