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
    net = S.MLP(IN, OUT, rows, 0, torch.cuda.current_stream().cuda_stream)
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


def rounded_backward(params, x, dy):
    """float64 reverse sweep with the kernel's bfloat16 storage points: the
    layer inputs a_l, the pre-activations z_l and the back-propagated dz_l are
    stored in bfloat16; dx stays float32."""
    a, zs, acts = bf16(x), [], []
    for l, (Wl, bl) in enumerate(params):
        acts.append(a)
        z = a @ bf16(Wl).T + bl.astype(np.float32).astype(np.float64)
        zs.append(bf16(z))
        a = bf16(MO.silu(z)) if l < len(params) - 1 else z
    dz = bf16(dy)
    grads = [None] * len(params)
    for m in range(len(params) - 1, -1, -1):
        grads[m] = (dz.T @ acts[m], dz.sum(0))
        da = dz @ bf16(params[m][0])
        if m > 0:
            dz = bf16(da * MO.silu_grad(zs[m - 1]))
    return grads, da


@pytest.mark.parametrize("rows", [1, 300, 2000])
def test_mlp_backward_matches_reference(rows):
    from paper_2310_01775_gb300 import stamp as S
    params = W.mlp_init(SIZES, 12)
    rng = np.random.default_rng(100 + rows)
    x = rng.uniform(-1, 1, size=(rows, IN))
    dy = rng.standard_normal((rows, OUT))
    net = S.MLP(IN, OUT, rows, rows, torch.cuda.current_stream().cuda_stream)
    net.set_params(torch.tensor(packed(params), device="cuda"))
    y = torch.empty(rows, OUT, device="cuda")
    dx = torch.empty(rows, IN, device="cuda")
    dp = torch.empty(net.n_params, device="cuda")
    net.forward_saved(torch.tensor(x, dtype=torch.float32, device="cuda"), rows, y, 0)
    net.backward(torch.tensor(dy, dtype=torch.float32, device="cuda"), rows, 0, dx, dp)
    net.sync()
    net.close()
    grads, dx_ref = rounded_backward(params, x, dy)
    dx = dx.cpu().numpy()
    assert np.abs(dx - dx_ref).max() <= 2e-2 * np.abs(dx_ref).max()
    dp_ref = packed([(gW, gb) for gW, gb in grads]).astype(np.float64)
    dp = dp.cpu().numpy()
    off = 0
    for (gW, gb) in grads:
        n = gW.size + gb.size
        seg, ref = dp[off:off + n], dp_ref[off:off + n]
        assert np.abs(seg - ref).max() <= 2e-2 * np.abs(ref).max(), off
        off += n
    # and against the unrounded float64 network
    full_grads, full_dx = MO.backward(params, MO.forward(params, x)[1], dy)
    assert np.abs(dx - full_dx).max() <= 6e-2 * np.abs(full_dx).max()


def test_mlp_training_fits_a_teacher_network():
    """Adam on the mean squared error drives a student to a random teacher's
    outputs (the teacher evaluated by the float64 reference)."""
    from paper_2310_01775_gb300 import stamp as S
    rows, batch = 16384, 1024
    teacher = W.mlp_init(SIZES, 21)
    x = np.random.default_rng(3).uniform(-1, 1, size=(rows, IN))
    t, _ = MO.forward(teacher, x)
    net = S.MLP(IN, OUT, batch, batch, torch.cuda.current_stream().cuda_stream)
    params = torch.tensor(packed(W.mlp_init(SIZES, 22)), device="cuda")
    losses = net.train(params, torch.tensor(x, dtype=torch.float32, device="cuda"),
                       torch.tensor(t, dtype=torch.float32, device="cuda"), rows, 8, batch, 1e-3)
    net.close()
    assert np.isfinite(losses).all()
    assert losses[-1] < 0.2 * losses[0], losses


def test_weight_gradients_and_training_are_reproducible():
    """The weight gradients run on the tensor cores per row split and are
    summed over the splits in a fixed order (no atomics): two backward passes
    give the same bits, and so do two trainings from the same start."""
    from paper_2310_01775_gb300 import stamp as S
    rows = 3000                                      # 24 tiles: several row splits
    params = torch.tensor(packed(W.mlp_init(SIZES, 13)), device="cuda")
    rng = np.random.default_rng(7)
    x = torch.tensor(rng.uniform(-1, 1, size=(rows, IN)), dtype=torch.float32, device="cuda")
    dy = torch.tensor(rng.standard_normal((rows, OUT)), dtype=torch.float32, device="cuda")
    stream = torch.cuda.current_stream().cuda_stream
    net = S.MLP(IN, OUT, rows, rows, stream)
    net.set_params(params)
    y = torch.empty(rows, OUT, device="cuda")
    dps = []
    for _ in range(2):
        dp = torch.empty(net.n_params, device="cuda")
        net.forward_saved(x, rows, y, 0)
        net.backward(dy, rows, 0, None, dp)
        dps.append(dp)
    net.sync()
    net.close()
    assert torch.equal(dps[0], dps[1])
    t = torch.tensor(rng.uniform(-1, 1, size=(rows, OUT)), dtype=torch.float32, device="cuda")
    outs = []
    for _ in range(2):
        p = params.clone()
        net = S.MLP(IN, OUT, 1000, 1000, stream)
        net.train(p, x, t, rows, 2, 1000, 1e-3)
        net.close()
        outs.append(p)
    assert torch.equal(outs[0], outs[1])
