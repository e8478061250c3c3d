"""ctypes binding of the STAMP C ABI (include/stamp.h).

Argument marshalling only: every step of the hot path runs in libstamp.so's
CUDA kernels.  Importing this module raises ImportError when the library has
not been built (there is no CPU fallback).

Pointer arguments accept a torch tensor (its data_ptr; float32/int32,
contiguous), a numpy array (host memory) or a raw integer address.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

_LIB_PATH = os.path.join(os.path.dirname(os.path.abspath(__file__)), "libstamp.so")
if not os.path.exists(_LIB_PATH):
    raise ImportError(f"{_LIB_PATH} is missing: build it with __graft_entry__.build() "
                      "(python paper_2310_01775_gb300/build.py)")
_lib = ctypes.CDLL(_LIB_PATH)

STAMP_OK, STAMP_EINVAL, STAMP_ENOMEM, STAMP_ECUDA, STAMP_ENONFINITE, STAMP_ETIMEOUT = range(6)
STAMP_ADJ_SEQUENTIAL, STAMP_ADJ_TIME_PARALLEL, STAMP_ADJ_AUTO, STAMP_ADJ_REPLAY = 0, 1, 2, 3
KERNELS = ("rollout_fwd", "rollout_adj", "pairwise", "median", "phi", "adam", "topk", "init",
           "surrogate", "screen")
STAMP_NKERNELS = len(KERNELS)


class StampError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"{_lib.stamp_status_str(status).decode()}: {msg}")
        self.status = status


class stamp_problem_desc(ctypes.Structure):
    _fields_ = [("n_blocks", ctypes.c_int), ("H", ctypes.c_int), ("T", ctypes.c_int),
                ("ckpt_every", ctypes.c_int)] + [
        (n, ctypes.c_float) for n in (
            "half_size", "mass", "mu", "mu_c", "g", "pusher_r", "k_contact", "c_contact",
            "eps_v", "eps_w", "eps_t", "dt", "tau", "w_yaw", "w_push", "offset_max", "dist_max")]

    @classmethod
    def from_params(cls, p: dict) -> "stamp_problem_desc":
        return cls(**{n: p[n] for n, _ in cls._fields_})


class stamp_instance_desc(ctypes.Structure):
    _fields_ = [("n_blocks", ctypes.c_int), ("H", ctypes.c_int), ("N", ctypes.c_int),
                ("seed", ctypes.c_ulonglong), ("init", ctypes.c_float * 12),
                ("goal", ctypes.c_float * 12)]


_vp, _i, _ull, _f = ctypes.c_void_p, ctypes.c_int, ctypes.c_ulonglong, ctypes.c_float
_sigs = {
    "stamp_problem_create": [ctypes.POINTER(stamp_problem_desc), _vp, _vp, _i, _vp,
                             ctypes.POINTER(_vp)],
    "stamp_rollout_fwd": [_vp, _vp, _i, _ull, _i, _i, _vp, _vp],
    "stamp_rollout_adjoint": [_vp, _vp, _i, _ull, _i, _vp],
    "stamp_rollout_fwd_from": [_vp, _vp, _vp, _i, _ull, _i, _i, _vp, _vp],
    "stamp_read_tape": [_vp, _i, _vp],
    "stamp_svgd_step": [_vp, _vp, _vp, _i, _vp, _vp, _i, _f, _i, _vp, _vp],
    "stamp_solve": [_vp, _i, _i, _i, _ull, _f, _vp, _vp, _vp, _i, _vp, _vp],
    "stamp_sync": [_vp],
    "stamp_set_profiling": [_vp, _i],
    "stamp_set_profiling_mask": [_vp, ctypes.c_uint],
    "stamp_get_kernel_times": [_vp, _vp, _vp],
    "stamp_set_lanes": [_vp, _i, _i],
    "stamp_set_overlap": [_vp, _i],
    "stamp_set_adjoint_mode": [_vp, _i],
    "stamp_get_adjoint_mode": [_vp, _i, _vp],
    "stamp_dropped_gradients": [_vp, _vp],
    "stamp_svgd_step_noalloc": [_vp, _vp, _i, _i, _vp, _vp, _i, _f, _i, _vp, _vp, _vp],
    "stamp_mlp_create": [_i, _i, _i, _i, _vp, ctypes.POINTER(_vp)],
    "stamp_mlp_set_params": [_vp, _vp],
    "stamp_mlp_forward": [_vp, _vp, _i, _vp],
    "stamp_mlp_forward_saved": [_vp, _vp, _i, _vp, _i],
    "stamp_mlp_backward": [_vp, _vp, _i, _i, _vp, _vp],
    "stamp_mlp_train": [_vp, _vp, _vp, _vp, _i, _i, _i, _f, _vp],
    "stamp_mlp_sync": [_vp],
    "stamp_surrogate_create": [ctypes.POINTER(stamp_problem_desc), _i, _i, _vp, ctypes.POINTER(_vp)],
    "stamp_surrogate_init_params": [_vp, _ull],
    "stamp_surrogate_set_params": [_vp, _vp],
    "stamp_surrogate_get_params": [_vp, _vp],
    "stamp_surrogate_transitions": [_vp, _i, _ull, _vp, _vp],
    "stamp_surrogate_train": [_vp, _vp, _vp, _i, _i, _i, _f, _vp],
    "stamp_surrogate_rollout": [_vp, _vp, _vp, _i, _ull, _i, _vp, _vp],
    "stamp_surrogate_screen": [_vp, _vp, _vp, _i, _i, _vp, _vp],
    "stamp_surrogate_sync": [_vp],
    "stamp_surrogate_dims": [_vp, _vp, _vp],
    "stamp_solve_surrogate": [_vp, _vp, _i, _i, _i, _i, _i, _ull, _f, _vp, _vp, _i, _vp, _vp],
    "stamp_set_target": [_vp, _f, _i],
    "stamp_set_dsvgd": [_vp, _i],
    "stamp_set_svgd_kernel": [_vp, _i],
    "stamp_svgd_step_weighted": [_vp, _vp, _vp, _vp, _vp, _i, _vp, _vp, _i, _f, _vp, _vp],
    "stamp_batch_create": [ctypes.POINTER(stamp_problem_desc), _vp, _i, _vp, ctypes.POINTER(_vp)],
    "stamp_batch_set_config": [_vp, _i, _i, _i, _i],
    "stamp_batch_get_config": [_vp, _i, _vp, _vp, _vp],
    "stamp_batch_autotune": [_vp, _i],
    "stamp_batch_solve": [_vp, _i, _f, _f, _i, _i],
    "stamp_batch_results": [_vp, _vp, _vp, _vp, _vp, _vp, _vp],
    "stamp_batch_read_theta": [_vp, _i, _vp],
    "stamp_solve_info": [_vp, _vp, _vp],
    "stamp_fp32_fma_peak": [_i, _vp, _vp],
    "stamp_inject_wait_timeout": [_vp],
    "stamp_set_particle_offset": [_vp, _i],
    "stamp_svgd_step_rows": [_vp, _vp, _vp, _i, _i, _i, _vp, _vp, _vp, _i, _f, _i, _vp, _vp],
    "stamp_batch_screen": [_vp, _vp, _i, _i],
    "stamp_set_replay_lanes": [_vp, _i],
    "stamp_batch_set_persistent": [_vp, _i],
    "stamp_batch_get_persistent": [_vp, _vp, _vp, _vp],
    "stamp_batch_inject_wait_timeout": [_vp],
    "stamp_batch_read_grad": [_vp, _i, _vp],
    "stamp_batch_set_trace": [_vp, _i],
    "stamp_batch_read_trace": [_vp, _vp, _i, _vp, _vp],
}
for _name, _args in _sigs.items():
    getattr(_lib, _name).argtypes = _args
    getattr(_lib, _name).restype = ctypes.c_int
_lib.stamp_mlp_destroy.argtypes = [_vp]
_lib.stamp_mlp_destroy.restype = None
_lib.stamp_mlp_param_count.argtypes = [_i, _i]
_lib.stamp_mlp_param_count.restype = ctypes.c_size_t
_lib.stamp_batch_destroy.argtypes = [_vp]
_lib.stamp_batch_destroy.restype = None
_lib.stamp_surrogate_last_kept.argtypes = [_vp]
_lib.stamp_surrogate_last_kept.restype = ctypes.c_int
_lib.stamp_surrogate_destroy.argtypes = [_vp]
_lib.stamp_surrogate_destroy.restype = None
_lib.stamp_problem_destroy.argtypes = [_vp]
_lib.stamp_problem_destroy.restype = None
_lib.stamp_status_str.argtypes = [ctypes.c_int]
_lib.stamp_status_str.restype = ctypes.c_char_p
_lib.stamp_last_error.restype = ctypes.c_char_p


def _check(status: int) -> None:
    if status != STAMP_OK:
        raise StampError(status, _lib.stamp_last_error().decode())


def _ptr(x):
    """Address of a tensor / numpy array / int (None -> NULL)."""
    if x is None:
        return None
    if isinstance(x, int):
        return x
    if hasattr(x, "data_ptr"):
        if not x.is_contiguous():
            raise ValueError("tensor arguments must be contiguous")
        return x.data_ptr()
    if isinstance(x, np.ndarray):
        if not x.flags["C_CONTIGUOUS"]:
            raise ValueError("numpy arguments must be C-contiguous")
        return x.ctypes.data
    raise TypeError(f"cannot pass {type(x)} as a pointer")


def _f32(x, name):
    if x is not None and hasattr(x, "dtype") and str(x.dtype) not in ("torch.float32", "float32"):
        raise TypeError(f"{name} must be float32")
    return _ptr(x)


def stamp_problem_create(desc: stamp_problem_desc, init_poses, goal_poses, max_particles: int,
                         cuda_stream: int | None = None) -> int:
    init = np.ascontiguousarray(init_poses, dtype=np.float32)
    goal = np.ascontiguousarray(goal_poses, dtype=np.float32)
    out = _vp()
    _check(_lib.stamp_problem_create(ctypes.byref(desc), init.ctypes.data, goal.ctypes.data,
                                     max_particles, cuda_stream, ctypes.byref(out)))
    return out.value


def stamp_problem_destroy(prob: int) -> None:
    _lib.stamp_problem_destroy(prob)


def stamp_rollout_fwd(prob, theta, N, seed, iter, hard, cost, final_state=None):
    _check(_lib.stamp_rollout_fwd(prob, _f32(theta, "theta"), N, seed, iter, int(hard),
                                  _f32(cost, "cost"), _f32(final_state, "final_state")))


def stamp_rollout_adjoint(prob, theta, N, seed, iter, grad_logp):
    _check(_lib.stamp_rollout_adjoint(prob, _f32(theta, "theta"), N, seed, iter,
                                      _f32(grad_logp, "grad_logp")))


def stamp_read_tape(prob, N, tape_out):
    _check(_lib.stamp_read_tape(prob, N, _f32(tape_out, "tape_out")))


def stamp_svgd_step(prob, theta, grad_logp, N, adam_m, adam_v, step, lr, sgd_phase=0,
                    h_out=None, phi_out=None):
    _check(_lib.stamp_svgd_step(prob, _f32(theta, "theta"), _f32(grad_logp, "grad_logp"), N,
                                _f32(adam_m, "adam_m"), _f32(adam_v, "adam_v"), step, lr,
                                int(sgd_phase), _f32(h_out, "h_out"), _f32(phi_out, "phi_out")))


def stamp_solve(prob, N, svgd_iters, sgd_iters, seed, lr, theta_init, theta_out, cost_out=None,
                k=0, topk_particle=None, stats_out=None):
    if topk_particle is not None and str(topk_particle.dtype) not in ("int32", "torch.int32"):
        raise TypeError("topk_particle must be int32")
    _check(_lib.stamp_solve(prob, N, svgd_iters, sgd_iters, seed, lr, _f32(theta_init, "theta_init"),
                            _f32(theta_out, "theta_out"), _f32(cost_out, "cost_out"), k,
                            _ptr(topk_particle), _f32(stats_out, "stats_out")))


def stamp_sync(prob):
    _check(_lib.stamp_sync(prob))


def stamp_set_profiling(prob, enable: bool):
    _check(_lib.stamp_set_profiling(prob, int(enable)))


def stamp_get_kernel_times(prob) -> dict:
    ms = np.zeros(STAMP_NKERNELS, dtype=np.float64)
    n = np.zeros(STAMP_NKERNELS, dtype=np.int64)
    _check(_lib.stamp_get_kernel_times(prob, ms.ctypes.data, n.ctypes.data))
    return {k: (float(ms[i]), int(n[i])) for i, k in enumerate(KERNELS)}


def stamp_set_lanes(prob, fwd_lanes: int, adj_lanes: int):
    _check(_lib.stamp_set_lanes(prob, fwd_lanes, adj_lanes))


def stamp_dropped_gradients(prob) -> int:
    n = ctypes.c_longlong()
    _check(_lib.stamp_dropped_gradients(prob, ctypes.byref(n)))
    return n.value


def stamp_svgd_step_noalloc(theta, grad_logp, N, D, adam_m, adam_v, step, lr, sgd_phase=0,
                            h_out=None, phi_out=None, cuda_stream=None):
    """stamp_svgd_step for callers that cannot allocate device memory (its
    scratch is a fixed array inside the library; N <= 1024, D <= 288)."""
    _check(_lib.stamp_svgd_step_noalloc(_f32(theta, "theta"), _f32(grad_logp, "grad_logp"), N, D,
                                        _f32(adam_m, "adam_m"), _f32(adam_v, "adam_v"), step, lr,
                                        int(sgd_phase), _f32(h_out, "h_out"),
                                        _f32(phi_out, "phi_out"), cuda_stream))


def stamp_fp32_fma_peak(launches: int = 20) -> tuple[float, float]:
    """(TFLOP/s, ms per launch): measured FP32 FMA throughput of the current
    device (independent fmaf chains filling every SM)."""
    tf, ms = ctypes.c_double(), ctypes.c_double()
    _check(_lib.stamp_fp32_fma_peak(int(launches), ctypes.byref(tf), ctypes.byref(ms)))
    return tf.value, ms.value


def library_path() -> str:
    return _LIB_PATH


class Problem:
    """Owns a stamp_problem handle; methods forward to the functions above."""

    def __init__(self, params: dict, init_poses, goal_poses, max_particles: int,
                 cuda_stream: int | None = None):
        self.params = dict(params)
        self.M = 4 * params["n_blocks"]
        self.P = self.M + 2
        self.D = params["H"] * self.P
        self.S = 6 * params["n_blocks"]
        self.n_ckpt = params["H"] * params["T"] // params["ckpt_every"]
        self.handle = stamp_problem_create(stamp_problem_desc.from_params(params), init_poses,
                                           goal_poses, max_particles, cuda_stream)

    def close(self):
        if self.handle:
            stamp_problem_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def rollout_fwd(self, theta, N, seed, iter, hard, cost, final_state=None):
        self._tape_owner = None          # the tape now belongs to this call
        stamp_rollout_fwd(self.handle, theta, N, seed, iter, hard, cost, final_state)

    def rollout_fwd_from(self, theta, init_states, N, seed, iter, hard, cost, final_state=None):
        """Forward rollout from per-particle start poses (N x n_blocks x 3)."""
        self._tape_owner = None
        _check(_lib.stamp_rollout_fwd_from(self.handle, _f32(theta, "theta"),
                                           _f32(init_states, "init_states"), N, seed, iter,
                                           int(hard), _f32(cost, "cost"),
                                           _f32(final_state, "final_state")))

    def rollout_adjoint(self, theta, N, seed, iter, grad_logp):
        stamp_rollout_adjoint(self.handle, theta, N, seed, iter, grad_logp)

    def read_tape(self, N, tape_out):
        stamp_read_tape(self.handle, N, tape_out)

    def svgd_step(self, theta, grad_logp, N, adam_m, adam_v, step, lr, sgd_phase=0, h_out=None,
                  phi_out=None):
        stamp_svgd_step(self.handle, theta, grad_logp, N, adam_m, adam_v, step, lr, sgd_phase,
                        h_out, phi_out)

    def solve(self, N, svgd_iters, sgd_iters, seed, lr, theta_init, theta_out, cost_out=None, k=0,
              topk_particle=None, stats_out=None):
        self._tape_owner = None
        stamp_solve(self.handle, N, svgd_iters, sgd_iters, seed, lr, theta_init, theta_out,
                    cost_out, k, topk_particle, stats_out)

    def sync(self):
        stamp_sync(self.handle)

    def set_profiling(self, enable):
        stamp_set_profiling(self.handle, enable)

    def set_profiling_kernels(self, names):
        """Record events only around the named kernels (KERNELS entries)."""
        mask = 0
        for n in names:
            mask |= 1 << KERNELS.index(n)
        _check(_lib.stamp_set_profiling_mask(self.handle, mask))

    def kernel_times(self):
        return stamp_get_kernel_times(self.handle)

    def set_overlap(self, enable):
        """Bandwidth on a second stream beside the rollouts in the solves (default on)."""
        _check(_lib.stamp_set_overlap(self.handle, int(enable)))

    def set_adjoint_mode(self, mode):
        """STAMP_ADJ_AUTO (default), STAMP_ADJ_TIME_PARALLEL, STAMP_ADJ_REPLAY or
        STAMP_ADJ_SEQUENTIAL."""
        _check(_lib.stamp_set_adjoint_mode(self.handle, int(mode)))

    def adjoint_mode(self, N):
        """The reverse sweep a call with N particles uses."""
        m = ctypes.c_int()
        _check(_lib.stamp_get_adjoint_mode(self.handle, int(N), ctypes.byref(m)))
        return m.value

    def adjoint_launches(self, N):
        """Kernel launches of one reverse sweep with N particles (the
        time-parallel sweep: relaxed parameters, Jacobians, recurrence; the
        replay: rebuild, sweep)."""
        return {STAMP_ADJ_TIME_PARALLEL: 3, STAMP_ADJ_REPLAY: 2}.get(self.adjoint_mode(N), 1)

    def set_lanes(self, fwd_lanes, adj_lanes):
        stamp_set_lanes(self.handle, fwd_lanes, adj_lanes)

    def set_replay_lanes(self, lanes):
        """Lanes per (particle, segment) team of the segment replay (0: automatic)."""
        _check(_lib.stamp_set_replay_lanes(self.handle, int(lanes)))

    def set_particle_offset(self, particle0):
        """Later rollouts' row r is particle particle0 + r of a larger set."""
        _check(_lib.stamp_set_particle_offset(self.handle, int(particle0)))

    def svgd_step_rows(self, theta_all, grad_all, N, row0, rows, theta_rows, adam_m, adam_v, step,
                       lr, sgd_phase=0, h_out=None, phi_out=None):
        """The Stein step of rows [row0, row0 + rows) from the gathered particles."""
        _check(_lib.stamp_svgd_step_rows(self.handle, _f32(theta_all, "theta_all"),
                                         _f32(grad_all, "grad_all"), N, row0, rows,
                                         _f32(theta_rows, "theta_rows"), _f32(adam_m, "adam_m"),
                                         _f32(adam_v, "adam_v"), step, lr, int(sgd_phase),
                                         _f32(h_out, "h_out"), _f32(phi_out, "phi_out")))

    def set_trace(self, on: bool):
        """Record every persistent launch's work items (stamp_batch_set_trace)."""
        _check(_lib.stamp_batch_set_trace(self.handle, int(bool(on))))

    def read_trace(self) -> dict:
        """The last persistent launch's items: kind, SM and claim / start /
        end times in ns (from the first claim)."""
        n, kinds = ctypes.c_int(), (ctypes.c_int * 5)()
        _check(_lib.stamp_batch_read_trace(self.handle, None, 0, ctypes.byref(n), kinds))
        raw = np.zeros((n.value, 4), dtype=np.uint64)   # 3 x u64 times, then (item, sm)
        _check(_lib.stamp_batch_read_trace(self.handle, raw.ctypes.data, n.value, None, None))
        t = raw[:, :3].astype(np.int64)
        item_sm = np.ascontiguousarray(raw[:, 3]).view(np.uint32).reshape(-1, 2)
        bounds = np.cumsum([0, kinds[0], kinds[1], kinds[2], kinds[2], kinds[3], kinds[4]])
        names = np.array(["rollout", "pairwise", "median1", "median2", "stein", "adam"])
        kind = names[np.searchsorted(bounds, np.arange(n.value), side="right") - 1]
        t0 = t[t[:, 0] > 0, 0].min() if (t[:, 0] > 0).any() else 0
        return {"kind": kind, "item": item_sm[:, 0], "sm": item_sm[:, 1],
                "claim": t[:, 0] - t0, "start": t[:, 1] - t0, "end": t[:, 2] - t0}

    def inject_wait_timeout(self):
        """Test hook: the next Stein-direction launch's first copy is never
        issued and its bounded wait runs out (STAMP_ETIMEOUT at the next sync)."""
        _check(_lib.stamp_inject_wait_timeout(self.handle))

    def dropped_gradients(self):
        return stamp_dropped_gradients(self.handle)

    def solve_surrogate(self, surrogate, n_candidates, N, surrogate_iters, sim_iters, seed, lr,
                        theta_out, cost_out=None, k=0, topk_particle=None, stats_out=None,
                        sgd_iters=0):
        """Algorithm 1 with screening and surrogate iterations (stamp_solve_surrogate)."""
        if topk_particle is not None and str(topk_particle.dtype) not in ("int32", "torch.int32"):
            raise TypeError("topk_particle must be int32")
        self._tape_owner = None
        _check(_lib.stamp_solve_surrogate(self.handle, surrogate.handle, n_candidates, N,
                                          surrogate_iters, sim_iters, sgd_iters, seed, lr,
                                          _f32(theta_out, "theta_out"), _f32(cost_out, "cost_out"),
                                          k, _ptr(topk_particle), _f32(stats_out, "stats_out")))

    def svgd_step_weighted(self, theta, grad_logp, cost_relaxed, cost_hard, N, adam_m, adam_v,
                           step, lr, h_out=None, phi_out=None):
        """Stein step with the importance weights of Eq. dsvgd from the two costs."""
        _check(_lib.stamp_svgd_step_weighted(self.handle, _f32(theta, "theta"),
                                             _f32(grad_logp, "grad_logp"),
                                             _f32(cost_relaxed, "cost_relaxed"),
                                             _f32(cost_hard, "cost_hard"), N,
                                             _f32(adam_m, "adam_m"), _f32(adam_v, "adam_v"), step,
                                             lr, _f32(h_out, "h_out"), _f32(phi_out, "phi_out")))

    def set_svgd_kernel(self, kind):
        """0: RBF on the whole plan; 1: the structured kernel (per-action RBFs on
        the push parameters and on softmax(a_k))."""
        _check(_lib.stamp_set_svgd_kernel(self.handle, int(kind)))

    def set_dsvgd(self, enable):
        """Eq. dsvgd importance weights in the solves' SVGD iterations."""
        _check(_lib.stamp_set_dsvgd(self.handle, int(enable)))

    def set_target(self, target_cost, check_every):
        """Early stop of the solves on the lowest hard, noise-free simulator cost."""
        _check(_lib.stamp_set_target(self.handle, target_cost, check_every))

    def solve_info(self):
        """(iterations the last solve ran, lowest hard cost of its last check)."""
        it, best = ctypes.c_int(), ctypes.c_float()
        _check(_lib.stamp_solve_info(self.handle, ctypes.byref(it), ctypes.byref(best)))
        return it.value, best.value


class Surrogate:
    """Learned pose-dynamics surrogate of one push (stamp_surrogate_*)."""

    def __init__(self, params: dict, max_rows: int, max_particles: int,
                 cuda_stream: int | None = None):
        out = _vp()
        _check(_lib.stamp_surrogate_create(ctypes.byref(stamp_problem_desc.from_params(params)),
                                           max_rows, max_particles, cuda_stream, ctypes.byref(out)))
        self.handle = out.value
        i, o = ctypes.c_int(), ctypes.c_int()
        self.n_params = _lib.stamp_surrogate_dims(self.handle, ctypes.byref(i), ctypes.byref(o))
        self.in_dim, self.out_dim = i.value, o.value

    def close(self):
        if self.handle:
            _lib.stamp_surrogate_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def init_params(self, seed):
        _check(_lib.stamp_surrogate_init_params(self.handle, seed))

    def set_params(self, params):
        _check(_lib.stamp_surrogate_set_params(self.handle, _f32(params, "params")))

    def get_params(self, params):
        _check(_lib.stamp_surrogate_get_params(self.handle, _f32(params, "params")))

    def transitions(self, n, seed, x_out, y_out):
        _check(_lib.stamp_surrogate_transitions(self.handle, n, seed, _f32(x_out, "x_out"),
                                                _f32(y_out, "y_out")))

    def train(self, x, y, n, epochs, batch, lr):
        """Returns the mean loss of each epoch."""
        losses = np.zeros(epochs, dtype=np.float32)
        _check(_lib.stamp_surrogate_train(self.handle, _f32(x, "x"), _f32(y, "y"), n, epochs,
                                          batch, lr, losses.ctypes.data))
        return losses

    def last_kept(self):
        """Transitions the last train() call kept (blow-ups dropped)."""
        return int(_lib.stamp_surrogate_last_kept(self.handle))

    def rollout(self, problem, theta, N, seed, iter, cost, grad_logp=None):
        _check(_lib.stamp_surrogate_rollout(self.handle, problem.handle, _f32(theta, "theta"), N,
                                            seed, iter, _f32(cost, "cost"),
                                            _f32(grad_logp, "grad_logp")))

    def screen(self, problem, candidates, n_candidates, N, theta_out, index_out=None):
        if index_out is not None and str(index_out.dtype) not in ("int32", "torch.int32"):
            raise TypeError("index_out must be int32")
        _check(_lib.stamp_surrogate_screen(self.handle, problem.handle,
                                           _f32(candidates, "candidates"), n_candidates, N,
                                           _f32(theta_out, "theta_out"), _ptr(index_out)))

    def sync(self):
        _check(_lib.stamp_surrogate_sync(self.handle))


class MLP:
    """The BF16 tensor-core MLP (in_dim -> 256 -> 256 -> 256 -> out_dim, SiLU)."""

    def __init__(self, in_dim: int, out_dim: int, max_rows: int, train_rows: int = 0,
                 cuda_stream: int | None = None):
        self.in_dim, self.out_dim = in_dim, out_dim
        out = _vp()
        _check(_lib.stamp_mlp_create(in_dim, out_dim, max_rows, train_rows, cuda_stream,
                                     ctypes.byref(out)))
        self.handle = out.value
        self.n_params = int(_lib.stamp_mlp_param_count(in_dim, out_dim))

    def close(self):
        if self.handle:
            _lib.stamp_mlp_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def set_params(self, params):
        """params: device float32 vector W1,b1,...,W4,b4 (W as (out, in))."""
        _check(_lib.stamp_mlp_set_params(self.handle, _f32(params, "params")))

    def forward(self, x, rows, y):
        _check(_lib.stamp_mlp_forward(self.handle, _f32(x, "x"), rows, _f32(y, "y")))

    def forward_saved(self, x, rows, y, tile_base=0):
        _check(_lib.stamp_mlp_forward_saved(self.handle, _f32(x, "x"), rows, _f32(y, "y"),
                                            tile_base))

    def backward(self, dy, rows, tile_base=0, dx=None, dparams=None):
        _check(_lib.stamp_mlp_backward(self.handle, _f32(dy, "dy"), rows, tile_base,
                                       _f32(dx, "dx"), _f32(dparams, "dparams")))

    def train(self, params, x, target, rows, epochs, batch, lr):
        """Returns the mean loss of each epoch."""
        losses = np.zeros(epochs, dtype=np.float32)
        _check(_lib.stamp_mlp_train(self.handle, _f32(params, "params"), _f32(x, "x"),
                                    _f32(target, "target"), rows, epochs, batch, lr,
                                    losses.ctypes.data))
        return losses

    def sync(self):
        _check(_lib.stamp_mlp_sync(self.handle))


class Batch:
    """Many planning instances solved together (stamp_batch_*).

    instances: dicts with n_blocks, H, N, seed, init (n_blocks x 3), goal
    (n_blocks x 3); physics: a parameter dict (its n_blocks/H are ignored)."""

    def __init__(self, physics: dict, instances, cuda_stream: int | None = None):
        arr = (stamp_instance_desc * len(instances))()
        for d, inst in zip(arr, instances):
            d.n_blocks, d.H, d.N, d.seed = inst["n_blocks"], inst["H"], inst["N"], inst["seed"]
            init = np.zeros(12, dtype=np.float32)
            goal = np.zeros(12, dtype=np.float32)
            init[:3 * inst["n_blocks"]] = np.asarray(inst["init"], dtype=np.float32).ravel()
            goal[:3 * inst["n_blocks"]] = np.asarray(inst["goal"], dtype=np.float32).ravel()
            d.init[:] = init.tolist()
            d.goal[:] = goal.tolist()
        desc = stamp_problem_desc.from_params(dict(physics, n_blocks=1, H=1, ckpt_every=1))
        out = _vp()
        _check(_lib.stamp_batch_create(ctypes.byref(desc), ctypes.cast(arr, _vp), len(instances),
                                       cuda_stream, ctypes.byref(out)))
        self.handle = out.value
        self.instances = [dict(i) for i in instances]
        self.n = len(instances)

    def close(self):
        if self.handle:
            _lib.stamp_batch_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def set_config(self, n_blocks, lanes, cta, ckpt_every):
        _check(_lib.stamp_batch_set_config(self.handle, n_blocks, lanes, cta, ckpt_every))

    def get_config(self, n_blocks):
        l, c, k = ctypes.c_int(), ctypes.c_int(), ctypes.c_int()
        _check(_lib.stamp_batch_get_config(self.handle, n_blocks, ctypes.byref(l), ctypes.byref(c),
                                           ctypes.byref(k)))
        return l.value, c.value, k.value

    def autotune(self, reps=2):
        _check(_lib.stamp_batch_autotune(self.handle, reps))

    def set_persistent(self, on: bool):
        """One launch per Stein iteration (True) or the per-class launches."""
        _check(_lib.stamp_batch_set_persistent(self.handle, int(bool(on))))

    def persistent(self) -> tuple[bool, float, float]:
        """(launch mode, autotuned ms per iteration per-class, persistent)."""
        on, a, p = ctypes.c_int(), ctypes.c_float(), ctypes.c_float()
        _check(_lib.stamp_batch_get_persistent(self.handle, ctypes.byref(on), ctypes.byref(a),
                                               ctypes.byref(p)))
        return bool(on.value), a.value, p.value

    def set_trace(self, on: bool):
        """Record every persistent launch's work items (stamp_batch_set_trace)."""
        _check(_lib.stamp_batch_set_trace(self.handle, int(bool(on))))

    def read_trace(self) -> dict:
        """The last persistent launch's items: kind, SM and claim / start /
        end times in ns (from the first claim)."""
        n, kinds = ctypes.c_int(), (ctypes.c_int * 5)()
        _check(_lib.stamp_batch_read_trace(self.handle, None, 0, ctypes.byref(n), kinds))
        raw = np.zeros((n.value, 4), dtype=np.uint64)   # 3 x u64 times, then (item, sm)
        _check(_lib.stamp_batch_read_trace(self.handle, raw.ctypes.data, n.value, None, None))
        t = raw[:, :3].astype(np.int64)
        item_sm = np.ascontiguousarray(raw[:, 3]).view(np.uint32).reshape(-1, 2)
        bounds = np.cumsum([0, kinds[0], kinds[1], kinds[2], kinds[2], kinds[3], kinds[4]])
        names = np.array(["rollout", "pairwise", "median1", "median2", "stein", "adam"])
        kind = names[np.searchsorted(bounds, np.arange(n.value), side="right") - 1]
        t0 = t[t[:, 0] > 0, 0].min() if (t[:, 0] > 0).any() else 0
        return {"kind": kind, "item": item_sm[:, 0], "sm": item_sm[:, 1],
                "claim": t[:, 0] - t0, "start": t[:, 1] - t0, "end": t[:, 2] - t0}

    def inject_wait_timeout(self):
        """The next persistent solve's dependency waits run out (error-path test)."""
        _check(_lib.stamp_batch_inject_wait_timeout(self.handle))

    def solve(self, iters, lr, target_cost=0.0, check_every=0, use_graph=True):
        _check(_lib.stamp_batch_solve(self.handle, iters, lr, target_cost, check_every,
                                      int(use_graph)))

    def results(self) -> dict:
        it = np.zeros(self.n, dtype=np.int32)
        best = np.zeros(self.n, dtype=np.float32)
        tts = np.zeros(self.n, dtype=np.float64)
        top3 = np.zeros(3 * self.n, dtype=np.int32)
        units, secs = ctypes.c_longlong(), ctypes.c_double()
        _check(_lib.stamp_batch_results(self.handle, it.ctypes.data, best.ctypes.data,
                                        tts.ctypes.data, top3.ctypes.data, ctypes.byref(units),
                                        ctypes.byref(secs)))
        return {"iterations": it, "best_cost": best, "seconds_to_target": tts,
                "top3": top3.reshape(self.n, 3), "units": units.value, "seconds": secs.value}

    def screen(self, surrogate, instance, n_candidates):
        """Start the instance's next solve from the N of n_candidates draws
        with the lowest surrogate cost (stamp_batch_screen)."""
        _check(_lib.stamp_batch_screen(self.handle, surrogate.handle, int(instance),
                                       int(n_candidates)))

    def read_theta(self, instance, out):
        _check(_lib.stamp_batch_read_theta(self.handle, instance, _f32(out, "theta_out")))

    def read_grad(self, instance, out):
        """grad log rho (N x D) of the instance's last Stein iteration."""
        _check(_lib.stamp_batch_read_grad(self.handle, instance, _f32(out, "grad_out")))
