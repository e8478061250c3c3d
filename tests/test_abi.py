"""The C ABI library builds, loads and exports every entry point that
include/stamp.h declares; argument checks that need no GPU reject bad input."""
import ctypes
import os
import re
import subprocess

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib_path():
    from paper_2310_01775_gb300 import build
    return build.build()


def declared_functions():
    src = open(os.path.join(ROOT, "include", "stamp.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(stamp_[a-z_]+)\s*\(", src)))


def test_header_declares_the_hot_path_calls():
    names = declared_functions()
    for n in ("stamp_problem_create", "stamp_problem_destroy", "stamp_rollout_fwd",
              "stamp_rollout_adjoint", "stamp_svgd_step", "stamp_solve"):
        assert n in names


def test_library_exports_every_declared_symbol(lib_path):
    out = subprocess.run(["nm", "-D", "--defined-only", lib_path], capture_output=True,
                         text=True, check=True).stdout
    exported = set(re.findall(r"\sT\s(\S+)", out))
    missing = [n for n in declared_functions() if n not in exported]
    assert not missing, missing
    lib = ctypes.CDLL(lib_path)
    for n in declared_functions():
        getattr(lib, n)


def test_binding_loads_and_rejects_bad_descriptions(lib_path):
    from paper_2310_01775_gb300 import stamp as S
    from paper_2310_01775_gb300 import workloads as W
    assert os.path.samefile(S.library_path(), lib_path)
    P = W.params("pusher1_h2")
    init, goal = W.scene(P, 0)
    for bad in (dict(n_blocks=0), dict(n_blocks=5), dict(H=0), dict(H=17), dict(T=50, ckpt_every=7),
                dict(dt=0.0), dict(mass=-1.0), dict(mu=float("nan")), dict(k_contact=-1.0)):
        with pytest.raises(S.StampError) as e:
            S.Problem(dict(P, **bad), init, goal, 8)
        assert e.value.status == S.STAMP_EINVAL
    with pytest.raises(S.StampError):
        S.Problem(P, init, goal, 0)
    with pytest.raises(S.StampError):
        S.Problem(P, np.full((1, 3), np.inf), goal, 8)
    assert S._lib.stamp_status_str(S.STAMP_ENONFINITE) == b"non-finite value"
