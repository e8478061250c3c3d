"""The BF16 tcgen05 MLP against the FP64 MLP reference (oracle/mlp_oracle.py).

Tight bar: against a float64 evaluation of the same rounded network (weights,
inputs and the activations between layers rounded to bfloat16 as the kernel
stores them) the outputs agree to 2e-3 of their largest magnitude (the
remaining difference is float32 vs float64 accumulation of 256-term sums and
rare rounding-boundary flips).  Loose bar: against the unrounded FP64 network,
3e-2 (bfloat16 keeps 8 significant bits)."""
import numpy as np
import pytest
import torch

from oracle import mlp_oracle as MO
from paper_2310_01775_gb300 import workloads as W

pytestmark = pytest.mark.gpu
IN, OUT = 26, 9
SIZES = [IN, 256, 256, 256, OUT]


def bf16(a):
    return torch.tensor(np.asarray(a), dtype=torch.float64).to(torch.bfloat16).double().numpy()


def packed(params):
    return np.concatenate([np.concatenate([Wl.ravel(), bl]) for Wl, bl in params]).astype(np.float32)


def rounded_reference(params, x):
    a = bf16(x)
    for l, (Wl, bl) in enumerate(params):
        z = a @ bf16(Wl).T + bl.astype(np.float32).astype(np.float64)
        a = bf16(MO.silu(z)) if l < len(params) - 1 else z
    return a


@pytest.mark.parametrize("rows", [1, 127, 128, 300, 5000])
def test_mlp_forward_matches_reference(rows):
    from paper_2310_01775_gb300 import stamp as S
    params = W.mlp_init(SIZES, 11)
    x = np.random.default_rng(rows).uniform(-1, 1, size=(rows, IN))
    net = S.MLP(IN, OUT, rows, torch.cuda.current_stream().cuda_stream)
    assert net.n_params == packed(params).size
    net.set_params(torch.tensor(packed(params), device="cuda"))
    y = torch.empty(rows, OUT, device="cuda")
    net.forward(torch.tensor(x, dtype=torch.float32, device="cuda"), rows, y)
    net.sync()
    net.close()
    y = y.cpu().numpy().astype(np.float64)
    ref = rounded_reference(params, x)
    scale = np.abs(ref).max()
    assert np.abs(y - ref).max() <= 2e-3 * scale, np.abs(y - ref).max() / scale
    full, _ = MO.forward(params, x)
    assert np.abs(y - full).max() <= 3e-2 * np.abs(full).max()
