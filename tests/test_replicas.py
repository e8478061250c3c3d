"""The multi-rank host path on CPU: two gloo ranks.

Every rank solves its own seeded instance (no collective on the data path);
the ranks exchange only their timings, and the whole-job throughput is all
ranks' units over the slowest rank's time.  These tests run that exchange
with two processes, and the benchmark's reference arm under the same
launcher the multi-GPU runs use (rank 0 alone reports).
"""
import json
import os
import socket
import subprocess
import sys

import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, out):
    os.environ.update(WORLD_SIZE=str(world), RANK=str(rank), LOCAL_RANK=str(rank),
                      MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    sys.path.insert(0, ROOT)
    from paper_2310_01775_gb300 import replicas as R
    w, r, _ = R.init("gloo")
    ms_local = 10.0 * (r + 1)                 # rank 1 is the slower one
    ms_max = R.max_over_ranks(ms_local)
    R.barrier()
    out.put((r, w, R.rank_seed(7, r), ms_max, R.throughput(1000.0, w, ms_max)))
    R.finish()


def test_two_gloo_ranks_agree_on_the_slowest_time():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    got = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    (r0, w0, s0, m0, v0), (r1, w1, s1, m1, v1) = got
    assert (r0, r1) == (0, 1) and w0 == w1 == 2
    assert s0 != s1                                   # disjoint problems per rank
    assert m0 == m1 == 20.0                           # both see the slowest rank's time
    assert v0 == v1 == 1000.0 * 2 / 0.020             # all ranks' units over that time


def test_reference_arm_under_two_ranks_prints_one_line_from_rank_zero():
    port = _free_port()
    cmd = [sys.executable, "-m", "torch.distributed.run", "--nnodes=1", "--nproc-per-node", "2",
           "--master-addr", "127.0.0.1", "--master-port", str(port), "bench.py", "--impl",
           "reference", "--gpus", "2", "--steps", "1", "--warmup", "0", "--ref-particles", "2"]
    r = subprocess.run(cmd, cwd=ROOT, capture_output=True, text=True, timeout=600)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [json.loads(x) for x in r.stdout.splitlines() if x.startswith("{")]
    assert len(lines) == 1, r.stdout
    line = lines[0]
    assert line["impl"] == "reference" and line["n_gpus"] == 2 and line["value"] > 0
    assert line["e2e"]["h2d_bytes_per_step"] == 0
