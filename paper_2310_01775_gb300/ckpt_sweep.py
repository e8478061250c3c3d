"""Checkpoint interval against tape memory and adjoint time.

    python -m paper_2310_01775_gb300.ckpt_sweep pusher1_h4 1,5,10,25,50,100

For each interval C (T % C == 0) prints one JSON line: tape bytes in HBM,
(H*T/C + 1) * N * S * 4, and the forward and adjoint kernel times (CUDA
events, mean of 20 launches after 3 warm-up launches) on the workload's
particles at initialisation.
"""
from __future__ import annotations

import json
import sys

import torch

from paper_2310_01775_gb300 import stamp as S
from paper_2310_01775_gb300 import workloads as W


def sweep(name: str, intervals):
    base = W.params(name)
    out = []
    for C in intervals:
        P = dict(base, ckpt_every=C)
        init, goal = W.scene(P, 0)
        N = P["N"]
        prob = S.Problem(P, init, goal, N, torch.cuda.current_stream().cuda_stream)
        theta = torch.tensor(W.random_theta(N, prob.D, 1), device="cuda")
        cost = torch.empty(N, device="cuda")
        grad = torch.empty(N, prob.D, device="cuda")
        ev = [torch.cuda.Event(enable_timing=True) for _ in range(4)]
        for _ in range(3):
            prob.rollout_fwd(theta, N, 0, 0, 0, cost)
            prob.rollout_adjoint(theta, N, 0, 0, grad)
        torch.cuda.synchronize()
        t_f = t_a = 0.0
        for _ in range(20):
            ev[0].record()
            prob.rollout_fwd(theta, N, 0, 0, 0, cost)
            ev[1].record()
            prob.rollout_adjoint(theta, N, 0, 0, grad)
            ev[2].record()
            torch.cuda.synchronize()
            t_f += ev[0].elapsed_time(ev[1])
            t_a += ev[1].elapsed_time(ev[2])
        rec = dict(workload=name, ckpt_every=C,
                   tape_bytes=(P["H"] * P["T"] // C + 1) * N * prob.S * 4,
                   fwd_ms=t_f / 20, adj_ms=t_a / 20)
        print(json.dumps(rec), flush=True)
        out.append(rec)
        prob.close()
    return out


if __name__ == "__main__":
    name = sys.argv[1] if len(sys.argv) > 1 else "pusher1_h4"
    cs = [int(c) for c in (sys.argv[2] if len(sys.argv) > 2 else "1,5,10,25,50,100").split(",")]
    sweep(name, cs)
