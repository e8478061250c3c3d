"""One stamp_solve of a named workload, for profiler captures.

    python -m paper_2310_01775_gb300.profile_case pusher1_h4 20
    python -m paper_2310_01775_gb300.profile_case surrogate 20
    python -m paper_2310_01775_gb300.profile_case batch 20      # or batch64: first 64 instances
    python -m paper_2310_01775_gb300.profile_case pbatch 20     # the same, persistent launch
    python -m paper_2310_01775_gb300.profile_case structured 20  # or dsvgd: pusher1_h4 variants

Builds the workload's problem (seed 0 scene), runs `iters` SVGD iterations
plus the hard evaluation and top-3 on the current CUDA device, and prints the
best hard cost.  Small iteration counts keep an ncu capture short.
`surrogate`: the 3-block workload's surrogate-assisted solve (a surrogate
trained for one epoch on 2^16 transitions; 131072 candidates screened to
2048; `iters` surrogate iterations, then 2 on the simulator).
"""
from __future__ import annotations

import sys

import numpy as np
import torch

from paper_2310_01775_gb300 import stamp as S
from paper_2310_01775_gb300 import workloads as W


def surrogate_case(iters: int) -> float:
    P = W.params("pusher3_h6")
    stream = torch.cuda.current_stream().cuda_stream
    init, goal = W.scene(P, 0)
    N = P["N"]
    sur = S.Surrogate(P, 131072, N, stream)
    n = 1 << 16
    x = torch.empty(n, sur.in_dim, device="cuda")
    y = torch.empty(n, sur.out_dim, device="cuda")
    sur.transitions(n, 1, x, y)
    sur.init_params(2)
    sur.train(x, y, n, 1, 4096, 2e-3)
    prob = S.Problem(P, init, goal, N, stream)
    theta = torch.empty(N, prob.D, device="cuda")
    cost = torch.empty(N, device="cuda")
    prob.solve_surrogate(sur, 131072, N, iters, 2, 0, 1e-2, theta, cost)
    torch.cuda.synchronize()
    prob.close()
    sur.close()
    return float(cost.min())


def batch_case(iters: int, n: int = 256, persistent: bool = False) -> float:
    """The first n of the 256 seeded serving instances (uniform goals), with the
    launch configuration the autotuner picks on GB300, `iters` iterations
    launched one by one (persistent: one launch per iteration)."""
    insts = W.batch_instances(256)[:n]
    b = S.Batch(dict(W.PHYSICS, T=100), insts, torch.cuda.current_stream().cuda_stream)
    for nb, cfg in {1: (2, 64, 1), 2: (4, 128, 1), 3: (8, 128, 1), 4: (8, 128, 1)}.items():
        if any(d["n_blocks"] == nb for d in insts):
            b.set_config(nb, *cfg)
    b.set_persistent(persistent)
    b.solve(iters, 1e-2, use_graph=False)
    best = float(b.results()["best_cost"].min())
    b.close()
    return best


def variant_case(name: str, iters: int) -> float:
    """pusher1_h4 solve with the Stein-step variant `name`: "dsvgd" (importance
    weights) or "structured" (the structured kernel)."""
    P = W.params("pusher1_h4")
    init, goal = W.scene(P, 0)
    N = P["N"]
    prob = S.Problem(P, init, goal, N, torch.cuda.current_stream().cuda_stream)
    prob.set_dsvgd(name == "dsvgd")
    prob.set_svgd_kernel(1 if name == "structured" else 0)
    theta = torch.empty(N, prob.D, device="cuda")
    cost = torch.empty(N, device="cuda")
    prob.solve(N, iters, 0, 0, P["lr"], None, theta, cost)
    torch.cuda.synchronize()
    prob.close()
    return float(cost.min())


def main(name: str = "pusher1_h4", iters: int = 2) -> float:
    if name in ("dsvgd", "structured"):
        return variant_case(name, iters)
    if name == "surrogate":
        return surrogate_case(iters)
    if name.startswith("batch"):
        return batch_case(iters, int(name[5:] or 256))
    if name.startswith("pbatch"):
        return batch_case(iters, int(name[6:] or 256), persistent=True)
    P = W.params(name)
    init, goal = W.scene(P, 0)
    N = P["N"]
    prob = S.Problem(P, init, goal, N, torch.cuda.current_stream().cuda_stream)
    theta = torch.empty(N, prob.D, device="cuda")
    cost = torch.empty(N, device="cuda")
    topk = np.zeros(3, dtype=np.int32)
    prob.solve(N, iters, 0, 0, P["lr"], None, theta, cost, 3, topk, None)
    torch.cuda.synchronize()
    prob.close()
    return float(cost.min())


if __name__ == "__main__":
    name = sys.argv[1] if len(sys.argv) > 1 else "pusher1_h4"
    iters = int(sys.argv[2]) if len(sys.argv) > 2 else 2
    print("ok", name, iters, main(name, iters))
