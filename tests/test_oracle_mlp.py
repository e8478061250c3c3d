"""Pins for the FP64 MLP reference (oracle/mlp_oracle.py): torch.nn layers,
a one-layer linear special case, and central finite differences."""
import numpy as np
import torch

from oracle import mlp_oracle as MO
from paper_2310_01775_gb300 import workloads as W


def test_matches_torch_nn_forward_and_gradients():
    sizes = [7, 16, 16, 5]
    params = W.mlp_init(sizes, 3)
    x = np.random.default_rng(1).standard_normal((9, 7))
    dy = np.random.default_rng(2).standard_normal((9, 5))
    y, cache = MO.forward(params, x)
    grads, dx = MO.backward(params, cache, dy)
    layers = []
    for l, (Wl, bl) in enumerate(params):
        lin = torch.nn.Linear(Wl.shape[1], Wl.shape[0]).double()
        with torch.no_grad():
            lin.weight.copy_(torch.tensor(Wl))
            lin.bias.copy_(torch.tensor(bl))
        layers += [lin] + ([torch.nn.SiLU()] if l < len(params) - 1 else [])
    net = torch.nn.Sequential(*layers)
    xt = torch.tensor(x, requires_grad=True)
    yt = net(xt)
    (yt * torch.tensor(dy)).sum().backward()
    assert np.allclose(y, yt.detach().numpy(), rtol=1e-13, atol=1e-13)
    assert np.allclose(dx, xt.grad.numpy(), rtol=1e-12, atol=1e-13)
    lins = [m for m in net if isinstance(m, torch.nn.Linear)]
    for (gW, gb), lin in zip(grads, lins):
        assert np.allclose(gW, lin.weight.grad.numpy(), rtol=1e-12, atol=1e-13)
        assert np.allclose(gb, lin.bias.grad.numpy(), rtol=1e-12, atol=1e-13)


def test_single_linear_layer_closed_form():
    Wl = np.arange(6.0).reshape(2, 3)
    bl = np.array([1.0, -1.0])
    x = np.array([[1.0, 2.0, 3.0]])
    y, cache = MO.forward([(Wl, bl)], x)
    assert np.allclose(y, [[0 + 2 + 6 + 1, 3 + 8 + 15 - 1]])
    (g,), dx = MO.backward([(Wl, bl)], cache, np.array([[1.0, 2.0]]))
    assert np.allclose(g[0], [[1, 2, 3], [2, 4, 6]]) and np.allclose(g[1], [1, 2])
    assert np.allclose(dx, [[0 + 6, 1 + 8, 2 + 10]])


def test_backward_matches_central_differences():
    sizes = [4, 8, 3]
    params = W.mlp_init(sizes, 5)
    x = np.random.default_rng(7).standard_normal((3, 4))
    dy = np.random.default_rng(8).standard_normal((3, 3))
    grads, dx = MO.backward(params, MO.forward(params, x)[1], dy)
    f = lambda p, xx: (MO.forward(p, xx)[0] * dy).sum()
    h = 1e-6
    for l in range(len(params)):
        for idx in [(0, 0), (1, 2), (2, 1)]:
            if idx[0] >= params[l][0].shape[0] or idx[1] >= params[l][0].shape[1]:
                continue
            pp = [(Wl.copy(), bl.copy()) for Wl, bl in params]
            pm = [(Wl.copy(), bl.copy()) for Wl, bl in params]
            pp[l][0][idx] += h
            pm[l][0][idx] -= h
            assert abs((f(pp, x) - f(pm, x)) / (2 * h) - grads[l][0][idx]) < 1e-7
    for i in range(3):
        for j in range(4):
            e = np.zeros_like(x)
            e[i, j] = h
            assert abs((f(params, x + e) - f(params, x - e)) / (2 * h) - dx[i, j]) < 1e-7
    assert np.allclose(MO.silu_grad(np.array([0.3])), (MO.silu(0.3 + h) - MO.silu(0.3 - h)) / (2 * h))
