"""One stamp_solve of a named workload, for profiler captures.

    python -m paper_2310_01775_gb300.profile_case pusher1_h4 20

Builds the workload's problem (seed 0 scene), runs `iters` SVGD iterations
plus the hard evaluation and top-3 on the current CUDA device, and prints the
best hard cost.  Small iteration counts keep an ncu capture short.
"""
from __future__ import annotations

import sys

import numpy as np
import torch

from paper_2310_01775_gb300 import stamp as S
from paper_2310_01775_gb300 import workloads as W


def main(name: str = "pusher1_h4", iters: int = 2) -> float:
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
