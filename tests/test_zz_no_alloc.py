"""The allocation-free Stein step against the problem-based one.

stamp_svgd_step_noalloc is for callers that cannot call cudaMalloc (their
device memory belongs to another allocator or pool, or allocating is not
allowed where they run), so they cannot create a stamp_problem; its scratch is
a fixed array inside the library.  It must give what stamp_svgd_step gives,
call after call, through the C ABI.  Kept in a file of its own that pytest
collects last.
"""
import numpy as np
import pytest
import torch

from paper_2310_01775_gb300 import workloads as W

pytestmark = pytest.mark.gpu


def _close(x, y, rel=1e-5):
    """Max-norm relative agreement (the bar of the Stein-step parity tests):
    the two paths may sum the Stein direction over j in different groupings."""
    return float((x - y).abs().max()) <= rel * max(float(y.abs().max()), 1e-12)


def _inputs(N, D, seed):
    theta = W.random_theta(N, D, seed)
    g = W.random_normal((N, D), seed + 1)
    m = W.random_normal((N, D), seed + 2, 0.1)
    v = np.abs(W.random_normal((N, D), seed + 3, 0.1)) + 1e-3
    return [torch.tensor(x, device="cuda") for x in (theta, g, m, v)]


@pytest.mark.parametrize("N,name,sgd,over", [(37, "pusher1_h4", 0, {}), (1024, "pusher1_h4", 0, {}),
                                             (300, "pusher3_h6", 0, {}), (64, "pusher1_h2", 1, {}),
                                             (1, "pusher1_h2", 0, {}),
                                             # the documented limits: N = 1024, D = 288 (4 blocks, H = 16)
                                             (1024, "pusher3_h6", 0, {"n_blocks": 4, "H": 16})])
def test_noalloc_step_matches_problem_step_twice(N, name, sgd, over):
    from paper_2310_01775_gb300 import stamp as S
    P = W.params(name, **over)
    init, goal = W.scene(P, 0)
    stream = torch.cuda.current_stream().cuda_stream
    prob = S.Problem(P, init, goal, N, stream)
    D = prob.D
    assert N <= 1024 and D <= 288
    a = _inputs(N, D, 40 + N)                      # problem-based path
    b = [x.clone() for x in a]                     # allocation-free path
    for step in (3, 4):                            # two calls in a row, state carried over
        ha, hb = torch.zeros(1, device="cuda"), torch.zeros(1, device="cuda")
        pa, pb = torch.zeros(N, D, device="cuda"), torch.zeros(N, D, device="cuda")
        prob.svgd_step(a[0], a[1], N, a[2], a[3], step, 1e-2, sgd, ha, pa)
        prob.sync()
        S.stamp_svgd_step_noalloc(b[0], b[1], N, D, b[2], b[3], step, 1e-2, sgd, hb, pb, stream)
        assert abs(float(ha) - float(hb)) <= 1e-5 * abs(float(ha))
        assert _close(pb, pa)
        for x, y in zip(b, a):
            assert _close(x, y)
        a[1] = torch.roll(a[1], 1, 0).contiguous()   # next gradients
        b[1] = a[1].clone()
    prob.close()


def test_noalloc_rejects_sizes_beyond_its_limit():
    from paper_2310_01775_gb300 import stamp as S
    N, D = 1025, 24
    x = torch.zeros(N, D, device="cuda")
    with pytest.raises(S.StampError) as e:
        S.stamp_svgd_step_noalloc(x, x.clone(), N, D, x.clone(), x.clone(), 1, 1e-2)
    assert e.value.status == S.STAMP_EINVAL and "STAMP_NOALLOC_MAX_N" in str(e.value)
    y = torch.zeros(8, 289, device="cuda")
    with pytest.raises(S.StampError) as e:
        S.stamp_svgd_step_noalloc(y, y.clone(), 8, 289, y.clone(), y.clone(), 1, 1e-2)
    assert e.value.status == S.STAMP_EINVAL
