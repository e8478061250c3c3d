"""Pins for the oracle's SVGD update [Eq. svgd], bandwidth and Adam.

* the lower-median bandwidth agrees with scipy's pairwise distances;
* the repulsive term equals the autograd gradient of the RBF kernel in its
  first argument (sign and the 2/h factor), the attractive term a plain
  kernel-weighted mean;
* with one particle the update is plain Adam on grad log p (torch.optim.Adam);
* SVGD fits a 1-D Gaussian target: mean and variance of the particles;
* the distinct-plan top-k on hand-made cases.
"""
import math

import numpy as np
import pytest
import torch
from scipy.spatial.distance import pdist

from oracle import stamp_oracle as O


def test_median_bandwidth_matches_scipy_lower_median():
    rng = np.random.default_rng(0)
    for n in (2, 3, 17, 64):
        th = rng.standard_normal((n, 5))
        vals = np.sort(pdist(th, "sqeuclidean"))
        assert abs(O.median_bandwidth(th) - vals[(vals.size - 1) // 2] / math.log(n + 1)) < 1e-12


def test_bandwidth_degenerate_cases():
    assert O.median_bandwidth(np.ones((1, 4))) == 1.0
    assert O.median_bandwidth(np.ones((5, 4))) == 1.0     # all distances zero


def test_stein_direction_against_autograd_kernel_gradient():
    rng = np.random.default_rng(1)
    n, d = 9, 4
    th = rng.standard_normal((n, d))
    g = rng.standard_normal((n, d))
    h = 0.7
    phi = O.stein_direction(th, g, h)
    T = torch.tensor(th, requires_grad=True)
    ref = np.zeros((n, d))
    for i in range(n):
        for j in range(n):
            tj = T[j].detach().clone().requires_grad_(True)
            kji = torch.exp(-((tj - T[i].detach()) ** 2).sum() / h)
            (gk,) = torch.autograd.grad(kji, tj)
            ref[i] += float(kji.detach()) * g[j] + gk.numpy()
    assert np.allclose(phi, ref / n, rtol=1e-12, atol=1e-12)


def test_single_particle_svgd_is_adam_on_grad_log_p():
    rng = np.random.default_rng(2)
    th = rng.standard_normal((1, 6))
    x = torch.tensor(th.copy(), requires_grad=True)
    opt = torch.optim.Adam([x], lr=0.05)
    m = np.zeros_like(th)
    v = np.zeros_like(th)
    for step in range(1, 30):
        g = -(th - 0.3) * 2.0                                 # grad log p of a Gaussian
        th, m, v, h, phi = O.svgd_step(th, g, m, v, step, 0.05)
        assert h == 1.0 and np.allclose(phi, g, rtol=1e-13)
        opt.zero_grad()
        x.grad = torch.tensor(-(-(x.detach().numpy() - 0.3) * 2.0))
        opt.step()
        assert np.allclose(th, x.detach().numpy(), rtol=1e-12, atol=1e-13)


def test_sgd_phase_follows_grad_log_p():
    rng = np.random.default_rng(3)
    th = rng.standard_normal((7, 3))
    g = rng.standard_normal((7, 3))
    th2, _, _, h, phi = O.svgd_step(th, g, np.zeros_like(th), np.zeros_like(th), 1, 0.01, sgd_phase=True)
    assert np.array_equal(phi, g)
    # first Adam step moves every coordinate by lr along sign(phi)
    assert np.allclose(th2 - th, 0.01 * np.sign(g), rtol=1e-6)


def test_svgd_fits_1d_gaussian():
    """SVGD with the RBF kernel and median bandwidth recovers N(mu, s^2)."""
    mu, s = 1.5, 0.7
    th = np.random.default_rng(4).uniform(-3, 3, size=(512, 1))
    for _ in range(1500):
        g = -(th - mu) / s ** 2
        h = O.median_bandwidth(th)
        th = th + 0.05 * O.stein_direction(th, g, h)
    assert abs(th.mean() - mu) < 0.02 * s
    assert abs(th.var() - s * s) < 0.05 * s * s


def test_topk_distinct_plans():
    costs = np.array([0.5, 0.1, 0.1, 0.3, 0.2, 0.05])
    codes = np.array([[0, 1], [2, 2], [2, 2], [0, 1], [3, 0], [2, 2]])
    # order by (cost, index): 5, 1, 2, 4, 3, 0 -> plans (2,2), (3,0), (0,1)
    assert O.topk_plans(costs, codes, 3) == [5, 4, 3]
    assert O.topk_plans(costs, codes, 5) == [5, 4, 3, -1, -1]
    # equal costs: the lower index wins
    assert O.topk_plans(np.array([1.0, 1.0]), np.array([[0], [1]]), 1) == [0]


# ---- Eq. dsvgd importance weights ---------------------------------------------


def test_weighted_stein_direction_against_autograd_loop():
    """sum_j (w_j/w) [k_ji g_j + grad_{theta_j} k_ji], written out pair by pair
    with autograd for the kernel gradient."""
    rng = np.random.default_rng(5)
    n, d, h = 7, 3, 0.9
    th, g = rng.standard_normal((n, d)), rng.standard_normal((n, d))
    w = rng.uniform(0.1, 3.0, n)
    phi = O.stein_direction(th, g, h, weights=w)
    T = torch.tensor(th)
    ref = np.zeros((n, d))
    for i in range(n):
        for j in range(n):
            tj = T[j].clone().requires_grad_(True)
            kji = torch.exp(-((tj - T[i]) ** 2).sum() / h)
            (gk,) = torch.autograd.grad(kji, tj)
            ref[i] += w[j] / w.sum() * (float(kji.detach()) * g[j] + gk.numpy())
    assert np.allclose(phi, ref, rtol=1e-12, atol=1e-13)


def test_equal_weights_are_plain_svgd_and_one_weight_is_one_particle():
    rng = np.random.default_rng(6)
    n, d, h = 8, 4, 1.3
    th, g = rng.standard_normal((n, d)), rng.standard_normal((n, d))
    assert np.allclose(O.stein_direction(th, g, h, weights=np.full(n, 2.5)),
                       O.stein_direction(th, g, h), rtol=1e-13, atol=1e-14)
    # all weight on particle 3: phi_i = k_i3 g_3 + (2/h) k_i3 (theta_i - theta_3)
    w = np.zeros(n)
    w[3] = 1.0
    k = np.exp(-((th - th[3]) ** 2).sum(1) / h)
    want = k[:, None] * g[3] + (2 / h) * k[:, None] * (th - th[3])
    assert np.allclose(O.stein_direction(th, g, h, weights=w), want, rtol=1e-12, atol=1e-14)


def test_dsvgd_weights_definition_and_shift_invariance():
    """w_j proportional to exp(C_j - C~_j) (hard against relaxed cost), summing
    to one; adding one constant to every cost leaves them unchanged; a
    particle whose relaxed plan is as good as its hard plan weighs e^{-1}
    of one whose relaxed cost is lower by one."""
    cr = np.array([1.0, 2.0, 0.5, 3.0])
    ch = np.array([1.0, 3.0, 0.5, 3.0])
    w = O.dsvgd_weights(cr, ch)
    assert abs(w.sum() - 1) < 1e-15
    assert np.allclose(w / w[0], [1.0, math.e, 1.0, 1.0])
    assert np.allclose(O.dsvgd_weights(cr + 7.0, ch + 7.0), w)
    big = O.dsvgd_weights(np.zeros(3), np.array([0.0, 800.0, 0.0]))   # no overflow
    assert np.isfinite(big).all() and abs(big[1] - 1.0) < 1e-12


# ---- the structured kernel (App. D.3, restated for offset/distance and choice parameters)


def _struct_case(n=6, nb=2, H=2, seed=0):
    from paper_2310_01775_gb300 import workloads as W
    P = W.params("pusher1_h2", n_blocks=nb, H=H)
    M, _, D = O.dims(P)
    th = np.random.default_rng(seed).standard_normal((n, D))
    return P, M, D, th


def test_structured_kernel_is_one_on_the_diagonal_symmetric_and_psd():
    P, M, D, th = _struct_case(n=12)
    h_c, h_z = O.structured_bandwidths(th, P)
    T = torch.tensor(th)
    G = np.array([[float(O.structured_kernel(T[i], T[j], P, h_c, h_z)) for j in range(12)]
                  for i in range(12)])
    assert np.allclose(np.diag(G), 1.0) and np.allclose(G, G.T)
    assert np.linalg.eigvalsh(G).min() > -1e-12


def test_structured_bandwidths_are_per_action_mean_medians():
    P, M, D, th = _struct_case(n=9, nb=1, H=3)
    c, z = O.structured_parts(th, P)
    for x, h in zip((c, z), O.structured_bandwidths(th, P)):
        f = x.reshape(9, -1).numpy()
        vals = np.sort(pdist(f, "sqeuclidean")) / P["H"]
        assert abs(h - vals[(vals.size - 1) // 2] / math.log(10)) < 1e-12


def test_structured_kernel_gradient_against_central_differences():
    P, M, D, th = _struct_case(n=5, seed=3)
    h_c, h_z = O.structured_bandwidths(th, P)
    a, b = torch.tensor(th[1]), torch.tensor(th[3])
    ar = a.clone().requires_grad_(True)
    (g,) = torch.autograd.grad(O.structured_kernel(ar, b, P, h_c, h_z), ar)
    eps = 1e-6
    for d in range(D):
        e = torch.zeros(D, dtype=torch.float64)
        e[d] = eps
        fd = (O.structured_kernel(a + e, b, P, h_c, h_z) - O.structured_kernel(a - e, b, P, h_c, h_z)) / (2 * eps)
        assert abs(float(fd) - float(g[d])) < 1e-8


def test_structured_repulsion_ignores_a_common_logit_shift():
    """softmax(a_k) is unchanged by adding one constant to all of action k's
    logits, so the kernel is, and its gradient has no component along that
    direction: each action's logit entries of the repulsive term sum to zero
    (with grad log p = 0 the Stein direction is the repulsion alone)."""
    P, M, D, th = _struct_case(n=7, nb=2, H=2, seed=4)
    phi = O.stein_direction_structured(th, np.zeros_like(th), P)
    Pn = M + 2
    for k in range(P["H"]):
        assert np.abs(phi[:, k * Pn:k * Pn + M].sum(1)).max() < 1e-13
    shifted = th.copy()
    shifted[:, :M] += 0.7
    assert np.allclose(O.stein_direction_structured(shifted, np.zeros_like(th), P), phi, atol=1e-13)


def test_structured_direction_written_out_for_one_action():
    """H = 1, one block: the attraction is K_ij g_j, the repulsion's offset and
    distance entries (2/h_c)(c_i - c_j) e^c_ij / (2H) and its logit entries
    (2/h_z) e^z_ij J(a_j)^T (s_i - s_j) / (2H), J the softmax Jacobian."""
    P, M, D, th = _struct_case(n=5, nb=1, H=1, seed=8)
    g = np.random.default_rng(9).standard_normal(th.shape)
    h_c, h_z = O.structured_bandwidths(th, P)
    a, c = th[:, :M], th[:, M:]
    s = np.exp(a - a.max(1, keepdims=True))
    s /= s.sum(1, keepdims=True)
    want = np.zeros_like(th)
    for i in range(5):
        for j in range(5):
            ec = math.exp(-((c[i] - c[j]) ** 2).sum() / h_c)
            ez = math.exp(-((s[i] - s[j]) ** 2).sum() / h_z)
            kij = (ec + ez) / 2
            J = np.diag(s[j]) - np.outer(s[j], s[j])
            rep = np.concatenate([(2 / h_z) * ez * J.T @ (s[i] - s[j]), (2 / h_c) * ec * (c[i] - c[j])]) / 2
            want[i] += (kij * g[j] + rep) / 5
    assert np.allclose(O.stein_direction_structured(th, g, P), want, rtol=1e-11, atol=1e-13)
