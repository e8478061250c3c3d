"""Pins for the oracle's random numbers and the discrete relaxation.

* SplitMix64 against published reference outputs (tests/golden).
* Gumbel(0,1) moments and the Gumbel-max property: argmax(a + g) is
  distributed as softmax(a) (the relaxation of Eq. gamma_map).
* Even partition of the uniform base distribution by Gamma (App. A.2-A.3):
  each of the m^K discrete plans has probability 1/m^K.
"""
import math
import os

import numpy as np
import pytest
import torch

from oracle import stamp_oracle as O
from paper_2310_01775_gb300 import workloads as W

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def test_splitmix64_reference_outputs():
    vals = [int(l) for l in open(os.path.join(GOLDEN, "splitmix64_seed1234567.txt"))
            if l.strip() and not l.startswith("#")]
    got = [int(O.sm64(1234567, i)) for i in range(len(vals))]
    assert got == vals


def test_uniform23_range_and_mean():
    x = O.sm64(O.sm64(7, 0), np.arange(200000, dtype=np.uint64))
    u = O.uniform23(x)
    assert u.min() > 0.0 and u.max() < 1.0
    assert abs(u.mean() - 0.5) < 4 * math.sqrt(1 / 12 / u.size)


def test_gumbel_moments():
    g = O.gumbel_noise(3, 5, 4000, 5, 10).ravel()
    euler_gamma = 0.5772156649015329
    se = math.pi / math.sqrt(6 * g.size)
    assert abs(g.mean() - euler_gamma) < 4 * se
    assert abs(g.var() - math.pi ** 2 / 6) < 0.05


def test_gumbel_streams_differ_by_iteration_and_seed():
    a = O.gumbel_noise(1, 0, 8, 2, 4)
    assert not np.allclose(a, O.gumbel_noise(1, 1, 8, 2, 4))
    assert not np.allclose(a, O.gumbel_noise(2, 0, 8, 2, 4))
    # particle i's draws do not depend on how many particles are drawn
    assert np.array_equal(a[:3], O.gumbel_noise(1, 0, 3, 2, 4))


def test_gumbel_max_matches_softmax():
    """P(argmax(a + g) = c) = softmax(a)_c for Gumbel g (Gumbel-max trick)."""
    a = np.array([0.3, -1.0, 1.2, 0.0])
    n = 200000
    g = O.gumbel_noise(11, 0, n, 1, 4)[:, 0, :]
    freq = np.bincount(np.argmax(a + g, axis=1), minlength=4) / n
    p = np.exp(a) / np.exp(a).sum()
    assert np.all(np.abs(freq - p) < 4 * np.sqrt(p * (1 - p) / n))


@pytest.mark.parametrize("m,K", [(4, 1), (4, 2), (3, 3)])
def test_even_partition_uniform_base(m, K):
    """App. A.2/A.3: Gamma splits U([-u,u]^{mK}) into m^K equal parts."""
    P = dict(W.PHYSICS, n_blocks=1, H=K)
    n = 120000
    u = 7.0
    th = np.random.default_rng(5).uniform(-u, u, size=(n, K, m + 2))
    if m != 4:  # use a plain logit block of width m
        codes = np.argmax(th[:, :, :m], axis=-1)
    else:
        codes = O.plan_codes(th.reshape(n, -1), P)
    idx = (codes * (m ** np.arange(K))).sum(1)
    freq = np.bincount(idx, minlength=m ** K) / n
    p = 1.0 / m ** K
    assert np.all(np.abs(freq - p) < 5 * math.sqrt(p * (1 - p) / n))


def test_relax_soft_and_hard():
    P = W.params("pusher1_h2")
    M, Pn, D = O.dims(P)
    th = torch.tensor(O.init_theta(4, 6, D))
    g = O.gumbel_noise(4, 0, 6, P["H"], M)
    z, off, dist = O.relax(th, P, g)
    a = th.numpy().reshape(6, P["H"], Pn)
    e = np.exp((a[:, :, :M] + g) / P["tau"])
    assert np.allclose(z.numpy(), e / e.sum(-1, keepdims=True), rtol=1e-12)
    assert np.all(np.abs(off.numpy()) < P["offset_max"])
    assert np.all((dist.numpy() > 0) & (dist.numpy() < P["dist_max"]))
    zh, _, _ = O.relax(th, P, None, hard=True)
    assert np.array_equal(zh.numpy().argmax(-1), O.plan_codes(th.numpy(), P))
    assert np.all(zh.numpy().sum(-1) == 1)


def test_hard_ties_pick_lowest_index():
    P = W.params("pusher1_h2")
    th = np.zeros((1, 12))
    th[0, 1] = th[0, 3] = 0.5          # action 0: tie between choices 1 and 3
    assert list(O.plan_codes(th, P)[0]) == [1, 0]


def test_init_theta_uniform():
    th = O.init_theta(9, 4000, 24)
    assert th.min() >= -1 and th.max() <= 1
    assert abs(th.mean()) < 0.01 and abs(th.var() - 1 / 3) < 0.01
