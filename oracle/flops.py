"""Algorithmic FLOP count of the rollout and its reverse sweep, per unit.

TEST INFRASTRUCTURE ONLY (run by hand; the resulting constants are quoted in
the bench and the design notes).  One unit = one particle advanced one
substep forward and back.  The count runs the oracle's own rollout for a
single particle under a dispatch mode that tallies every arithmetic aten op:
one FLOP per output element of an elementwise op (add, mul, div, sqrt, exp,
sin, atan2, comparisons, where, clamp, ...), n_in - n_out for a reduction,
2mnk for a matmul; views, copies, stacking and indexing count zero.  Forward
ops are those run while building the tape, reverse ops those run by
autograd.  Both branches of a masked select are counted, as the oracle
evaluates them, so these are upper bounds of the useful arithmetic.

    python oracle/flops.py pusher1_h4
"""
from __future__ import annotations

import os
import sys

import torch
from torch.utils._python_dispatch import TorchDispatchMode

sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
from oracle import stamp_oracle as O  # noqa: E402

ZERO = {"view", "_unsafe_view", "expand", "clone", "copy_", "copy", "stack", "cat", "select",
        "slice", "unsqueeze", "squeeze", "permute", "t", "transpose", "reshape", "unbind",
        "lift_fresh", "detach", "alias", "empty_like", "zeros_like", "ones_like", "ones",
        "zeros", "full", "full_like", "scalar_tensor", "new_zeros", "new_empty", "new_ones",
        "one_hot", "index", "index_select", "gather", "_to_copy", "as_strided", "fill_",
        "zero_", "split", "split_with_sizes", "repeat", "arange", "empty", "lift_fresh_copy",
        "_local_scalar_dense", "unsqueeze_", "masked_fill", "slice_backward", "select_backward",
        "new_empty_strided", "empty_strided", "sum_to_size", "expand_as"}
REDUCE = {"sum", "amax", "max", "min", "mean", "logsumexp", "prod"}


class Counter(TorchDispatchMode):
    def __init__(self):
        super().__init__()
        self.flops = 0
        self.by_op = {}

    def __torch_dispatch__(self, func, types, args=(), kwargs=None):
        out = func(*args, **(kwargs or {}))
        name = func.__name__.split(".")[0]
        n = 0
        if name in ZERO:
            n = 0
        elif name in ("mm", "bmm", "matmul", "addmm"):
            a, b = args[-2], args[-1]
            n = 2 * a.numel() * b.shape[-1]
        elif name in REDUCE:
            n = max(args[0].numel() - (out.numel() if torch.is_tensor(out) else 1), 0)
        elif torch.is_tensor(out):
            n = out.numel()
        self.flops += n
        self.by_op[name] = self.by_op.get(name, 0) + n
        return out


def count(P, init, goal):
    """(forward FLOPs per unit, reverse FLOPs per unit) for one particle."""
    M, _, D = O.dims(P)
    th = torch.zeros(1, D, dtype=torch.float64, requires_grad=True)
    gum = torch.zeros(1, P["H"], M, dtype=torch.float64).numpy()
    fwd = Counter()
    with fwd:
        q, v, _, _, dist, _ = O.simulate(th, P, init, gum, False, False)
        c = O.cost(q, dist, goal, P)
    rev = Counter()
    with rev:
        torch.autograd.grad(c.sum(), th)
    units = P["H"] * P["T"]
    return fwd.flops / units, rev.flops / units


if __name__ == "__main__":
    from paper_2310_01775_gb300 import workloads as W
    for name in (sys.argv[1:] or list(W.CONFIGS)):
        P = W.params(name)
        init, goal = W.scene(P, 0)
        f, r = count(P, init, goal)
        print(f"{name}: forward {f:.1f} FLOP/unit, reverse {r:.1f} FLOP/unit, total {f + r:.1f}")
