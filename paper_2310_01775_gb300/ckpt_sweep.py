"""Checkpoint interval against tape memory and adjoint time.

    python -m paper_2310_01775_gb300.ckpt_sweep pusher1_h4 1,5,10,25,50,100

For each interval C (T % C == 0) and each reverse sweep that applies (the
automatic choice, and the sequential sweep when that differs) prints one
JSON line: the checkpoint tape in HBM, (H*T/C + 1) * N * S * 4 bytes; the
segment replay's scratch, when it runs ((H*T + 1) * N * S floats of states
plus H*T * N * 2 n_blocks of yaw sines and cosines); and the forward and
reverse-sweep times (CUDA events, mean of 20 launches after 3 warm-up
launches) on the workload's particles at initialisation.
"""
from __future__ import annotations

import json
import sys

import torch

from paper_2310_01775_gb300 import stamp as S
from paper_2310_01775_gb300 import workloads as W


MODES = {S.STAMP_ADJ_SEQUENTIAL: "sequential", S.STAMP_ADJ_TIME_PARALLEL: "time-parallel",
         S.STAMP_ADJ_REPLAY: "segment replay"}


def sweep(name: str, intervals):
    base = W.params(name)
    out = []
    for C, mode in [(C, m) for C in intervals for m in (S.STAMP_ADJ_AUTO, S.STAMP_ADJ_SEQUENTIAL)]:
        P = dict(base, ckpt_every=C)
        init, goal = W.scene(P, 0)
        N = P["N"]
        prob = S.Problem(P, init, goal, N, torch.cuda.current_stream().cuda_stream)
        prob.set_adjoint_mode(mode)
        used = prob.adjoint_mode(N)
        if mode == S.STAMP_ADJ_SEQUENTIAL and out and out[-1]["ckpt_every"] == C \
                and out[-1]["reverse_sweep"] == MODES[used]:
            prob.close()
            continue
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
        HT = P["H"] * P["T"]
        rec = dict(workload=name, ckpt_every=C, reverse_sweep=MODES[used],
                   tape_bytes=(HT // C + 1) * N * prob.S * 4,
                   replay_scratch_bytes=((HT + 1) * N * prob.S + HT * N * 2 * P["n_blocks"]) * 4
                   if used == S.STAMP_ADJ_REPLAY else 0,
                   fwd_ms=t_f / 20, adj_ms=t_a / 20)
        print(json.dumps(rec), flush=True)
        out.append(rec)
        prob.close()
    return out


if __name__ == "__main__":
    name = sys.argv[1] if len(sys.argv) > 1 else "pusher1_h4"
    cs = [int(c) for c in (sys.argv[2] if len(sys.argv) > 2 else "1,5,10,25,50,100").split(",")]
    sweep(name, cs)
