// C ABI of the STAMP hot path (declared in include/stamp.h): problem
// objects, argument checks, the Algorithm 1 loop and kernel timing.
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

#include "stamp.h"
#include "stamp_internal.cuh"

using stamp::SimConst;

namespace {

thread_local std::string g_err;

stamp_status fail(stamp_status s, const char* fmt, ...) {
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    g_err = buf;
    return s;
}

#define STAMP_CUDA(call)                                                                 \
    do {                                                                                 \
        cudaError_t e_ = (call);                                                         \
        if (e_ != cudaSuccess)                                                           \
            return fail(STAMP_ECUDA, "%s failed: %s", #call, cudaGetErrorString(e_));    \
    } while (0)

constexpr int kMaxParticles = 16384;     // d2 scratch is N^2 floats (1 GiB at the cap)
constexpr long long kMaxStatsIters = 1 << 20;
// the time-parallel reverse sweep keeps 39 coefficients per particle and
// substep; above this it is not set up (the sequential sweep runs)
constexpr size_t kMaxTimeParallelBytes = (size_t)4 << 30;
constexpr int kTimeParallelMaxN = 3072;   // the automatic mode's crossover (see time_parallel)
constexpr unsigned kInjectedWaitLimit = 4096;   // polls of a wait made to run out (test hook)

bool is_device_ptr(const void* p) {
    cudaPointerAttributes at;
    if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return at.type == cudaMemoryTypeDevice || at.type == cudaMemoryTypeManaged;
}

}  // namespace

struct stamp_problem {
    SimConst sc;
    int max_n = 0;
    cudaStream_t stream = nullptr;
    // one device arena, carved into the buffers below
    char* arena = nullptr;
    float *tape = nullptr, *cost = nullptr, *grad = nullptr, *theta = nullptr, *m = nullptr,
          *v = nullptr, *phi = nullptr, *d2 = nullptr, *h = nullptr, *one = nullptr;
    unsigned *hist = nullptr, *stats = nullptr, *sel = nullptr, *counter = nullptr, *stop = nullptr;
    int *flag = nullptr, *topk = nullptr;
    unsigned long long* dropped = nullptr;
    // global index of the first particle of later calls (a shard of a larger set)
    int particle0 = 0;
    // last forward
    bool have_tape = false;
    int last_n = 0, last_iter = 0, last_hard = 0, last_particle0 = 0;
    unsigned long long last_seed = 0;
    const float* last_theta = nullptr;
    int fwd_lanes = 0, adj_lanes = 0, replay_lanes = 0;
    // one-block reverse sweep as a linear recurrence in time (checkpoint
    // interval 1): its scratch exists when the problem qualifies
    int adj_mode = STAMP_ADJ_AUTO;
    float *pit_rel = nullptr, *pit_coef = nullptr;
    bool pit_ok = false;
    // segment replay (checkpoint interval > 1): the per-substep states of the
    // last forward, rebuilt in parallel, then swept at interval 1
    float* full = nullptr;
    float2* full_trig = nullptr;   // the replayed states' yaw (cos, sin)
    bool replay_ok = false;
    // the bandwidth (pairwise distances + median) depends on theta only: the
    // solves run it on a second stream beside the rollouts
    bool overlap = true;
    cudaStream_t side = nullptr;
    cudaEvent_t ev_theta = nullptr, ev_h = nullptr;
    // early stop of the solves, and what the last solve did
    float target = 0.f;
    int check_every = 0;
    bool dsvgd = false;          // Eq. dsvgd importance weights in the solves' SVGD iterations
    float *cost_hard = nullptr, *wn = nullptr;
    // structured kernel (App. D.3 restated): components and a second median scratch
    int kernel_kind = 0;
    char* sk_arena = nullptr;
    float *sk_C = nullptr, *sk_S = nullptr, *sk_d2 = nullptr, *sk_h = nullptr;
    unsigned *sk_hist = nullptr, *sk_sel = nullptr, *sk_counter = nullptr;
    int iters_run = 0;
    float best_hard = 0.f;
    // test hook: the next Stein-direction launch's CTAs arm their first
    // stage without issuing its copy and give up after a short wait
    bool inject_wait_timeout = false;
    // kernel timing
    bool prof = false;
    unsigned prof_mask = ~0u;             // kernel kinds recorded while profiling
    std::vector<cudaEvent_t> ev;          // pairs (start, stop)
    std::vector<int> ev_kind;
    size_t ev_used = 0;
    double ms[STAMP_NKERNELS] = {};
    long long launches[STAMP_NKERNELS] = {};
};

namespace {

template <class F>
stamp_status timed_on(stamp_problem* p, int kind, cudaStream_t st, F&& launch) {
    const bool rec = p->prof && ((p->prof_mask >> kind) & 1u) && p->ev_used < p->ev_kind.size();
    if (rec) STAMP_CUDA(cudaEventRecord(p->ev[2 * p->ev_used], st));
    const cudaError_t e = launch();
    if (e != cudaSuccess) return fail(STAMP_ECUDA, "kernel launch failed: %s", cudaGetErrorString(e));
    if (rec) {
        STAMP_CUDA(cudaEventRecord(p->ev[2 * p->ev_used + 1], st));
        p->ev_kind[p->ev_used++] = kind;
    }
    return STAMP_OK;
}
template <class F>
stamp_status timed(stamp_problem* p, int kind, F&& launch) {
    return timed_on(p, kind, p->stream, launch);
}

// After a stream sync: fold the recorded event pairs into the totals.
stamp_status collect(stamp_problem* p) {
    for (size_t q = 0; q < p->ev_used; ++q) {
        float t = 0.f;
        STAMP_CUDA(cudaEventElapsedTime(&t, p->ev[2 * q], p->ev[2 * q + 1]));
        p->ms[p->ev_kind[q]] += t;
        p->launches[p->ev_kind[q]] += 1;
    }
    p->ev_used = 0;
    return STAMP_OK;
}

stamp_status check_flag(stamp_problem* p) {
    int f = 0;
    STAMP_CUDA(cudaMemcpy(&f, p->flag, sizeof(int), cudaMemcpyDeviceToHost));
    if (f) {
        STAMP_CUDA(cudaMemset(p->flag, 0, sizeof(int)));
        if (f & 2) return fail(STAMP_ETIMEOUT, "a bounded device wait gave up (copy never completed)");
        return fail(STAMP_ENONFINITE, "a non-finite particle or Stein direction was produced");
    }
    return STAMP_OK;
}

int lanes_for(const stamp_problem* p, int N, bool adj) {
    const int want = adj ? p->adj_lanes : p->fwd_lanes;
    return want ? want : stamp::default_lanes(p->sc.nb, N, adj);
}

stamp_status check_n(const stamp_problem* p, int N) {
    if (N < 1 || N > p->max_n) return fail(STAMP_EINVAL, "N=%d outside [1, %d]", N, p->max_n);
    return STAMP_OK;
}

stamp_status check_dev(const void* ptr, const char* name, bool allow_null = false) {
    if (!ptr) return allow_null ? STAMP_OK : fail(STAMP_EINVAL, "%s is NULL", name);
    if (!is_device_ptr(ptr)) return fail(STAMP_EINVAL, "%s is not device memory", name);
    return STAMP_OK;
}

#define STAMP_TRY(x)                      \
    do {                                  \
        stamp_status s_ = (x);            \
        if (s_ != STAMP_OK) return s_;    \
    } while (0)

// The reverse sweep a call with N particles uses: time-parallel where its
// scratch exists and, in the automatic mode, up to kTimeParallelMaxN
// particles -- measured on GB300 (one block, H = 4, T = 100): the
// time-parallel sweep takes half the sequential one's time at 1024
// particles and breaks even near 4096, where the sequential teams fill the
// GPU and the Jacobians' extra arithmetic no longer comes for free.
bool time_parallel(const stamp_problem* p, int N) {
    if (!p->pit_ok || p->adj_mode == STAMP_ADJ_SEQUENTIAL || p->adj_mode == STAMP_ADJ_REPLAY)
        return false;
    return p->adj_mode == STAMP_ADJ_TIME_PARALLEL || N <= kTimeParallelMaxN;
}

// The sweep a call with N particles runs: time-parallel (above), else the
// segment replay where its scratch exists (checkpoint interval > 1) unless
// the sequential sweep was asked for, else sequential.
int adjoint_kind(const stamp_problem* p, int N) {
    if (time_parallel(p, N)) return STAMP_ADJ_TIME_PARALLEL;
    if (p->replay_ok && p->adj_mode != STAMP_ADJ_SEQUENTIAL) return STAMP_ADJ_REPLAY;
    return STAMP_ADJ_SEQUENTIAL;
}

stamp_status fwd(stamp_problem* p, const float* theta, int N, unsigned long long seed, int iter,
                 int hard, float* cost, float* final_state, unsigned* stats_word,
                 const float* init_states = nullptr) {
    stamp::RolloutArgs a{};
    a.theta = theta; a.N = N; a.seed = seed; a.iter = iter; a.hard = hard;
    a.tape = p->tape; a.cost = cost; a.final_state = final_state; a.stats_min = stats_word;
    a.init_states = init_states;
    a.particle0 = p->particle0;
    const int lanes = lanes_for(p, N, false);
    STAMP_TRY(timed(p, STAMP_K_ROLLOUT_FWD,
                    [&] { return stamp::launch_rollout_fwd(p->sc, a, lanes, p->stream); }));
    p->have_tape = true;
    p->last_n = N; p->last_seed = seed; p->last_iter = iter; p->last_hard = hard;
    p->last_particle0 = p->particle0;
    p->last_theta = theta;
    return STAMP_OK;
}

stamp_status adj(stamp_problem* p, const float* theta, int N, float* grad) {
    stamp::RolloutArgs a{};
    a.theta = theta; a.N = N; a.seed = p->last_seed; a.iter = p->last_iter; a.hard = p->last_hard;
    a.tape = p->tape; a.grad = grad; a.dropped = p->dropped; a.particle0 = p->last_particle0;
    const int kind = adjoint_kind(p, N);
    if (kind == STAMP_ADJ_TIME_PARALLEL)
        return timed(p, STAMP_K_ROLLOUT_ADJ, [&] {
            return stamp::launch_adjoint_time(p->sc, a, p->pit_rel, p->pit_coef, p->flag, p->stream);
        });
    const int lanes = lanes_for(p, N, true);
    if (kind == STAMP_ADJ_REPLAY)
        return timed(p, STAMP_K_ROLLOUT_ADJ, [&] {
            stamp::RolloutArgs ar = a;
            ar.trig = p->full_trig;
            const int rl = p->replay_lanes ? p->replay_lanes : stamp::replay_lanes(p->sc.nb);
            cudaError_t e = stamp::launch_replay(p->sc, ar, rl, p->full, p->stream);
            if (e != cudaSuccess) return e;
            SimConst sc1 = p->sc;          // the rebuilt tape has interval 1
            sc1.C = 1;
            sc1.n_ckpt = sc1.H * sc1.T;
            stamp::RolloutArgs a1 = ar;
            a1.tape = p->full;
            return stamp::launch_rollout_adj(sc1, a1, lanes, p->stream);
        });
    return timed(p, STAMP_K_ROLLOUT_ADJ,
                 [&] { return stamp::launch_rollout_adj(p->sc, a, lanes, p->stream); });
}

// RBF bandwidth of theta (pairwise distances, radix-select median) on stream
// st; h lands in p->h (and h_out when given).
stamp_status bandwidth(stamp_problem* p, const float* theta, int N, float* h_out, cudaStream_t st) {
    stamp::SvgdScratch s{p->d2, p->hist, p->sel, p->counter, p->h, p->flag};
    STAMP_CUDA(cudaMemsetAsync(p->hist, 0, (2048 + 2048 + 1024) * sizeof(unsigned), st));
    STAMP_TRY(timed_on(p, STAMP_K_PAIRWISE, st,
                       [&] { return stamp::launch_pairwise(theta, N, p->sc.D, s, st); }));
    if (N >= 2) {
        for (int dg = 1; dg <= 2; ++dg)
            STAMP_TRY(timed_on(p, STAMP_K_MEDIAN, st, [&] {
                return stamp::launch_median_digit(N, dg, s, dg == 2 ? h_out : nullptr, st);
            }));
    } else if (h_out) {
        STAMP_CUDA(cudaMemcpyAsync(h_out, p->one, sizeof(float), cudaMemcpyDeviceToDevice, st));
    }
    return STAMP_OK;
}

// bw_done: the RBF bandwidth of theta is already in p->h (launched beside the
// rollouts and waited for).
stamp_status svgd(stamp_problem* p, float* theta, const float* grad, int N, float* m, float* v,
                  int step, float lr, int sgd_phase, float* h_out, float* phi_out,
                  const float* wn = nullptr, bool bw_done = false) {
    const int D = p->sc.D;
    const float* part = grad;   // SGD phase: phi = grad log rho, one share
    int shares = 1;
    if (!sgd_phase && p->kernel_kind == 1) {
        // structured kernel: bandwidths of the offset/distance and choice components
        const int H = p->sc.H, M = p->sc.M;
        STAMP_CUDA(stamp::launch_struct_prep(theta, N, H, M, p->sk_C, p->sk_S, p->stream));
        stamp::SvgdScratch a{p->d2, p->hist, p->sel, p->counter, p->h, p->flag};
        stamp::SvgdScratch b{p->sk_d2, p->sk_hist, p->sk_sel, p->sk_counter, p->sk_h, p->flag};
        const stamp::SvgdScratch* ss[2] = {&a, &b};
        const float* comp[2] = {p->sk_C, p->sk_S};
        const int width[2] = {2 * H, M * H};
        for (int q = 0; q < 2; ++q) {
            STAMP_CUDA(cudaMemsetAsync(ss[q]->hist, 0, (2048 + 2048 + 1024) * sizeof(unsigned), p->stream));
            STAMP_TRY(timed(p, STAMP_K_PAIRWISE, [&] {
                return stamp::launch_pairwise(comp[q], N, width[q], *ss[q], p->stream);
            }));
            if (N >= 2)
                for (int dg = 1; dg <= 2; ++dg)
                    STAMP_TRY(timed(p, STAMP_K_MEDIAN, [&] {
                        return stamp::launch_median_digit(N, dg, *ss[q], nullptr, p->stream);
                    }));
        }
        if (h_out) STAMP_CUDA(stamp::launch_scale_scalar(p->h, 1.f / (float)H, h_out, p->stream));
        STAMP_TRY(timed(p, STAMP_K_PHI, [&] {
            return stamp::launch_struct_phi(theta, grad, p->sk_C, p->sk_S, N, H, M, p->h, p->sk_h, wn,
                                            p->phi, stamp::kMaxShares, &shares, p->stream);
        }));
        part = p->phi;
    } else if (!sgd_phase) {
        stamp::SvgdScratch s{p->d2, p->hist, p->sel, p->counter, p->h, p->flag};
        if (p->inject_wait_timeout) {
            s.wait_limit = kInjectedWaitLimit;
            s.skip_first_copy = 1;
            p->inject_wait_timeout = false;
        }
        if (!bw_done) STAMP_TRY(bandwidth(p, theta, N, h_out, p->stream));
        STAMP_TRY(timed(p, STAMP_K_PHI, [&] {
            return stamp::launch_phi(theta, grad, N, D, s, p->phi, stamp::kMaxShares, &shares,
                                     p->stream, wn);
        }));
        part = p->phi;
    } else if (h_out) {
        STAMP_CUDA(cudaMemcpyAsync(h_out, p->one, sizeof(float), cudaMemcpyDeviceToDevice,
                                   p->stream));
    }
    return timed(p, STAMP_K_ADAM, [&] {
        return stamp::launch_adam(theta, part, shares, phi_out, m, v, N * D, step, lr, p->flag,
                                  p->stream);
    });
}

// Iterations of one solve: [0, sur) on the surrogate's gradients, then svgd
// Stein iterations and sgd plain-gradient iterations on the simulator.
struct Phases {
    stamp_surrogate* s;
    int n_cand, sur, svgd, sgd;
};

// Events around a multi-launch piece (surrogate rollout, screening).
template <class F>
stamp_status timed_piece(stamp_problem* p, int kind, F&& piece) {
    const bool rec = p->prof && ((p->prof_mask >> kind) & 1u) && p->ev_used < p->ev_kind.size();
    if (rec) STAMP_CUDA(cudaEventRecord(p->ev[2 * p->ev_used], p->stream));
    STAMP_TRY(piece());
    if (rec) {
        STAMP_CUDA(cudaEventRecord(p->ev[2 * p->ev_used + 1], p->stream));
        p->ev_kind[p->ev_used++] = kind;
    }
    return STAMP_OK;
}

// Hard, noise-free rollout of all particles; the lowest cost in *best.
stamp_status hard_min(stamp_problem* p, const float* th, int N, unsigned long long seed, float* cost,
                      float* best) {
    STAMP_CUDA(cudaMemsetAsync(p->stop, 0xFF, sizeof(unsigned), p->stream));
    STAMP_TRY(fwd(p, th, N, seed, -1, 1, cost, nullptr, p->stop));
    unsigned bits = 0;
    STAMP_CUDA(cudaMemcpyAsync(&bits, p->stop, sizeof bits, cudaMemcpyDeviceToHost, p->stream));
    STAMP_CUDA(cudaStreamSynchronize(p->stream));
    std::memcpy(best, &bits, sizeof bits);
    return STAMP_OK;
}

stamp_status run_solve(stamp_problem* p, const Phases& ph, int N, unsigned long long seed, float lr,
                       const float* theta_init, float* theta_out, float* cost_out, int k,
                       int* topk_particle, float* stats_out) {
    STAMP_TRY(check_n(p, N));
    if (ph.svgd < 0 || ph.sgd < 0) return fail(STAMP_EINVAL, "negative iteration count");
    const long long iters = (long long)ph.sur + ph.svgd + ph.sgd;
    if (stats_out && iters > kMaxStatsIters)
        return fail(STAMP_EINVAL, "stats_out supports at most %lld iterations", kMaxStatsIters);
    if (!theta_out) return fail(STAMP_EINVAL, "theta_out is NULL");
    if (k < 0 || (k > 0 && !topk_particle)) return fail(STAMP_EINVAL, "bad k / topk_particle");
    if (k > 0 && N > stamp::kMaxTopkN) return fail(STAMP_EINVAL, "top-k needs N <= %d", stamp::kMaxTopkN);
    if (k > N) return fail(STAMP_EINVAL, "k=%d > N=%d", k, N);
    if (!std::isfinite(lr)) return fail(STAMP_EINVAL, "lr is not finite");
    const int D = p->sc.D;
    const size_t nd = (size_t)N * D;
    const bool out_dev = is_device_ptr(theta_out);
    float* th = out_dev ? theta_out : p->theta;
    if (ph.s && ph.n_cand > N) {
        float* cand = stamp::surrogate_candidates(ph.s);
        STAMP_TRY(timed_piece(p, STAMP_K_SCREEN, [&] {
            const cudaError_t e = stamp::launch_init_theta(cand, ph.n_cand, D, seed, p->stream);
            if (e != cudaSuccess) return fail(STAMP_ECUDA, "candidate launch failed: %s", cudaGetErrorString(e));
            return stamp::surrogate_screen(ph.s, p->sc, cand, ph.n_cand, N, th, nullptr);
        }));
    } else if (theta_init) {
        STAMP_CUDA(cudaMemcpyAsync(th, theta_init, nd * sizeof(float), cudaMemcpyDefault, p->stream));
    } else {
        STAMP_TRY(timed(p, STAMP_K_INIT, [&] { return stamp::launch_init_theta(th, N, D, seed, p->stream); }));
    }
    STAMP_CUDA(cudaMemsetAsync(p->m, 0, nd * sizeof(float), p->stream));
    STAMP_CUDA(cudaMemsetAsync(p->v, 0, nd * sizeof(float), p->stream));
    if (stats_out) STAMP_CUDA(cudaMemsetAsync(p->stats, 0xFF, iters * sizeof(unsigned), p->stream));
    p->iters_run = (int)iters;
    p->best_hard = INFINITY;
    for (long long it = 0; it < iters; ++it) {
        unsigned* sw = stats_out ? p->stats + it : nullptr;
        const bool sgd = it >= (long long)ph.sur + ph.svgd;
        // the bandwidth needs theta only: start it beside this iteration's rollouts
        const bool side_bw = p->overlap && !sgd && p->kernel_kind == 0 && N >= 2;
        if (side_bw) {
            STAMP_CUDA(cudaEventRecord(p->ev_theta, p->stream));
            STAMP_CUDA(cudaStreamWaitEvent(p->side, p->ev_theta, 0));
            STAMP_TRY(bandwidth(p, th, N, nullptr, p->side));
            STAMP_CUDA(cudaEventRecord(p->ev_h, p->side));
        }
        if (it < ph.sur) {
            STAMP_TRY(timed_piece(p, STAMP_K_SURROGATE, [&] {
                return stamp::surrogate_rollout(ph.s, p->sc, th, N, seed, (int)it, p->cost, p->grad, sw);
            }));
        } else {
            STAMP_TRY(fwd(p, th, N, seed, (int)it, 0, p->cost, nullptr, sw));
            STAMP_TRY(adj(p, th, N, p->grad));
        }
        const float* wn = nullptr;
        if (p->dsvgd && !sgd && it >= ph.sur) {
            // Eq. dsvgd: the hard plan of the same Gumbel draws against the relaxed one
            STAMP_TRY(fwd(p, th, N, seed, (int)it, 1, p->cost_hard, nullptr, nullptr));
            STAMP_CUDA(stamp::launch_dsvgd_weights(p->cost, p->cost_hard, N, p->wn, p->stream));
            wn = p->wn;
        }
        if (side_bw) STAMP_CUDA(cudaStreamWaitEvent(p->stream, p->ev_h, 0));
        STAMP_TRY(svgd(p, th, p->grad, N, p->m, p->v, (int)it + 1, lr, sgd ? 1 : 0, nullptr,
                       nullptr, wn, side_bw));
        if (p->check_every > 0 && (it + 1) % p->check_every == 0) {
            STAMP_TRY(hard_min(p, th, N, seed, p->cost, &p->best_hard));
            if (p->best_hard < p->target) {
                p->iters_run = (int)(it + 1);
                break;
            }
        }
    }
    // hard evaluation (Gamma, no noise) and the distinct-plan top-k
    float* ch = (cost_out && is_device_ptr(cost_out)) ? cost_out : p->cost;
    STAMP_CUDA(cudaMemsetAsync(p->stop, 0xFF, sizeof(unsigned), p->stream));
    STAMP_TRY(fwd(p, th, N, seed, -1, 1, ch, nullptr, p->stop));
    if (k > 0)
        STAMP_TRY(timed(p, STAMP_K_TOPK, [&] { return stamp::launch_topk(th, ch, N, p->sc, k, p->topk, p->stream); }));
    if (!out_dev)
        STAMP_CUDA(cudaMemcpyAsync(theta_out, th, nd * sizeof(float), cudaMemcpyDefault, p->stream));
    if (cost_out && ch != cost_out)
        STAMP_CUDA(cudaMemcpyAsync(cost_out, ch, N * sizeof(float), cudaMemcpyDefault, p->stream));
    if (k > 0)
        STAMP_CUDA(cudaMemcpyAsync(topk_particle, p->topk, k * sizeof(int), cudaMemcpyDefault, p->stream));
    if (stats_out)
        STAMP_CUDA(cudaMemcpyAsync(stats_out, p->stats, iters * sizeof(float), cudaMemcpyDefault, p->stream));
    unsigned bits = 0;
    STAMP_CUDA(cudaMemcpyAsync(&bits, p->stop, sizeof bits, cudaMemcpyDeviceToHost, p->stream));
    STAMP_CUDA(cudaStreamSynchronize(p->stream));
    std::memcpy(&p->best_hard, &bits, sizeof bits);
    STAMP_TRY(collect(p));
    return check_flag(p);
}

bool finite_pos(float x) { return std::isfinite(x) && x > 0.f; }
bool finite_nonneg(float x) { return std::isfinite(x) && x >= 0.f; }

}  // namespace

namespace stamp {

void set_last_error(const char* msg) { g_err = msg; }

int sm_count() {
    constexpr int kDevices = 64;
    static int cached[kDevices] = {};
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kDevices) {
        cudaGetLastError();
        return 152;
    }
    if (!cached[dev]) {
        int n = 0;
        if (cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || n < 1) {
            cudaGetLastError();
            n = 152;
        }
        cached[dev] = n;
    }
    return cached[dev];
}

SimConst problem_const(const stamp_problem* p) { return p->sc; }

stamp_status rollout_from(stamp_problem* p, const float* theta, const float* init_states, int N,
                          uint64_t seed, int iter, float* cost, float* final_state) {
    STAMP_TRY(check_n(p, N));
    return fwd(p, theta, N, seed, iter, 0, cost, final_state, nullptr, init_states);
}

bool lanes_supported(int nb, int lanes) {
    switch (nb) {
        case 1: return lanes == 1 || lanes == 2 || lanes == 4;
        case 2: return lanes == 2 || lanes == 4 || lanes == 8 || lanes == 16;
        case 3: case 4: return lanes == 8 || lanes == 16 || lanes == 32;
    }
    return false;
}

// Lanes per particle, from sweeps on GB300 at 2048 particles (H = 6, C = 25,
// segment replay): one block 4/4; two blocks forward 8 (0.28 ms; 0.38 at 4,
// 0.40 at 16), sweep 8 (0.50 ms; 0.60 at 16); three blocks forward 8
// (0.75 ms; 0.82 at 16, 0.90 at 32), sweep 8 (1.28 ms; 1.38 at 16, 2.11 at
// 32); four blocks forward 16 (1.28 ms; 1.39 at 8, 1.46 at 32), sweep 16
// (2.37 ms; 3.09 at 8, 2.82 at 32).
int default_lanes(int nb, int N, bool adjoint) {
    (void)N;
    if (nb == 1) return 4;
    if (nb == 2 || nb == 3) return 8;
    return 16;
}

cudaError_t launch_rollout_fwd(const SimConst& sc, const RolloutArgs& a, int lanes, cudaStream_t st) {
    switch (sc.nb) {
        case 1: return launch_rollout_nb1(sc, a, lanes, false, st);
        case 2: return launch_rollout_nb2(sc, a, lanes, false, st);
        case 3: return launch_rollout_nb3(sc, a, lanes, false, st);
        case 4: return launch_rollout_nb4(sc, a, lanes, false, st);
    }
    return cudaErrorInvalidValue;
}

// The fewest lanes each block count supports: the replay is throughput
// bound, and fewer lanes integrate the state less redundantly.
int replay_lanes(int nb) { return nb == 1 ? 1 : nb == 2 ? 2 : nb == 3 ? 4 : 8; }

cudaError_t launch_replay(const SimConst& sc, const RolloutArgs& a, int lanes, float* full,
                          cudaStream_t st) {
    switch (sc.nb) {
        case 1: return launch_replay_nb1(sc, a, lanes, full, st);
        case 2: return launch_replay_nb2(sc, a, lanes, full, st);
        case 3: return launch_replay_nb3(sc, a, lanes, full, st);
        case 4: return launch_replay_nb4(sc, a, lanes, full, st);
    }
    return cudaErrorInvalidValue;
}

cudaError_t launch_rollout_adj(const SimConst& sc, const RolloutArgs& a, int lanes, cudaStream_t st) {
    switch (sc.nb) {
        case 1: return launch_rollout_nb1(sc, a, lanes, true, st);
        case 2: return launch_rollout_nb2(sc, a, lanes, true, st);
        case 3: return launch_rollout_nb3(sc, a, lanes, true, st);
        case 4: return launch_rollout_nb4(sc, a, lanes, true, st);
    }
    return cudaErrorInvalidValue;
}

}  // namespace stamp

extern "C" {

const char* stamp_status_str(stamp_status s) {
    switch (s) {
        case STAMP_OK: return "ok";
        case STAMP_EINVAL: return "invalid argument";
        case STAMP_ENOMEM: return "out of memory";
        case STAMP_ECUDA: return "CUDA error";
        case STAMP_ENONFINITE: return "non-finite value";
        case STAMP_ETIMEOUT: return "device wait timed out";
    }
    return "unknown status";
}

const char* stamp_last_error(void) { return g_err.c_str(); }

stamp_status stamp_problem_create(const stamp_problem_desc* d, const float* init_poses,
                                  const float* goal_poses, int max_particles, void* cuda_stream,
                                  stamp_problem** out) {
    if (!out) return fail(STAMP_EINVAL, "out is NULL");
    *out = nullptr;
    if (!d || !init_poses || !goal_poses) return fail(STAMP_EINVAL, "NULL description or poses");
    if (d->n_blocks < 1 || d->n_blocks > stamp::kMaxBlocks)
        return fail(STAMP_EINVAL, "n_blocks=%d outside [1, %d]", d->n_blocks, stamp::kMaxBlocks);
    if (d->H < 1 || d->H > stamp::kMaxH) return fail(STAMP_EINVAL, "H=%d outside [1, %d]", d->H, stamp::kMaxH);
    if (d->T < 1 || d->ckpt_every < 1 || d->T % d->ckpt_every)
        return fail(STAMP_EINVAL, "need T >= 1, ckpt_every >= 1 and T %% ckpt_every == 0");
    if (max_particles < 1 || max_particles > kMaxParticles)
        return fail(STAMP_EINVAL, "max_particles=%d outside [1, %d]", max_particles, kMaxParticles);
    const float pos[] = {d->half_size, d->mass, d->pusher_r, d->eps_v, d->eps_w, d->eps_t, d->dt, d->tau};
    for (float x : pos)
        if (!finite_pos(x)) return fail(STAMP_EINVAL, "a size, mass, smoothing, dt or tau is not > 0");
    const float nonneg[] = {d->mu, d->mu_c, d->g, d->k_contact, d->c_contact, d->w_yaw, d->w_push,
                            d->offset_max, d->dist_max};
    for (float x : nonneg)
        if (!finite_nonneg(x)) return fail(STAMP_EINVAL, "a coefficient or range is negative or not finite");
    for (int q = 0; q < 3 * d->n_blocks; ++q)
        if (!std::isfinite(init_poses[q]) || !std::isfinite(goal_poses[q]))
            return fail(STAMP_EINVAL, "non-finite pose");

    stamp_problem* p = new stamp_problem();
    SimConst& sc = p->sc;
    std::memset(&sc, 0, sizeof sc);
    sc.nb = d->n_blocks; sc.H = d->H; sc.T = d->T; sc.C = d->ckpt_every;
    sc.M = 4 * sc.nb; sc.P = sc.M + 2; sc.D = sc.H * sc.P; sc.S = 6 * sc.nb;
    sc.n_ckpt = sc.H * sc.T / sc.C;
    const double a = 2.0 * d->half_size;
    const double inertia = d->mass * (a * a + a * a) / 12.0;                   // uniform square
    const double r_eff = a / 6.0 * (std::sqrt(2.0) + std::log(1.0 + std::sqrt(2.0)));
    sc.hs = d->half_size; sc.r = d->pusher_r; sc.k = d->k_contact; sc.c = d->c_contact;
    sc.mu_c = d->mu_c; sc.dt = d->dt; sc.inv_dt = (float)(1.0 / d->dt);
    sc.inv_m = (float)(1.0 / d->mass); sc.inv_I = (float)(1.0 / inertia);
    sc.fric_lin = (float)((double)d->mu * d->mass * d->g);
    sc.fric_ang = (float)((double)d->mu * d->mass * d->g * r_eff);
    sc.eps_v2 = d->eps_v * d->eps_v; sc.eps_w2 = d->eps_w * d->eps_w; sc.eps_t2 = d->eps_t * d->eps_t;
    {
        const double circ = std::sqrt(2.0) * d->half_size;   // circumscribed radius of a block
        const double dr = 1.001 * (circ + d->pusher_r), cr = 1.001 * circ;
        sc.disk_reach2 = (float)(dr * dr);
        sc.corner_reach2 = (float)(cr * cr);
    }
    sc.inv_tau = (float)(1.0 / d->tau); sc.w_yaw = d->w_yaw; sc.w_push = d->w_push;
    sc.off_max = d->offset_max; sc.dist_max = d->dist_max;
    for (int b = 0; b < sc.nb; ++b)
        for (int q = 0; q < 3; ++q) {
            sc.init[b][q] = init_poses[3 * b + q];
            sc.goal[b][q] = goal_poses[3 * b + q];
        }
    const int D = sc.D;
    // a checkpoint segment must fit in shared memory for one team
    if ((size_t)(sc.C * (sc.S / 2) + 1) * 8 > 200 * 1024) {
        delete p;
        return fail(STAMP_EINVAL, "ckpt_every=%d too large for on-chip segment replay", sc.C);
    }
    p->max_n = max_particles;
    p->stream = (cudaStream_t)cuda_stream;

    // carve the arena
    const size_t n = (size_t)max_particles;
    const size_t pit_coef_bytes = stamp::adjoint_time_coef_floats(max_particles, sc.H, sc.T) * sizeof(float);
    const bool pit = sc.nb == 1 && sc.C == 1 && pit_coef_bytes <= kMaxTimeParallelBytes;
    const size_t full_bytes = (size_t)(sc.H * sc.T + 1) * n * sc.S * sizeof(float);
    const bool replay = sc.C > 1 && full_bytes <= kMaxTimeParallelBytes;
    struct Part { void** dst; size_t bytes; };
    const Part parts[] = {
        {(void**)&p->tape, (size_t)(sc.n_ckpt + 1) * n * sc.S * sizeof(float)},
        {(void**)&p->cost, n * sizeof(float)},
        {(void**)&p->grad, n * D * sizeof(float)},
        {(void**)&p->theta, n * D * sizeof(float)},
        {(void**)&p->m, n * D * sizeof(float)},
        {(void**)&p->v, n * D * sizeof(float)},
        {(void**)&p->phi, (size_t)stamp::kMaxShares * n * D * sizeof(float)},
        {(void**)&p->d2, n * n * sizeof(float)},
        {(void**)&p->h, sizeof(float)},
        {(void**)&p->one, sizeof(float)},
        {(void**)&p->hist, (2048 + 2048 + 1024) * sizeof(unsigned)},
        {(void**)&p->stats, kMaxStatsIters * sizeof(unsigned)},
        {(void**)&p->flag, sizeof(int)},
        {(void**)&p->topk, n * sizeof(int)},
        {(void**)&p->dropped, sizeof(unsigned long long)},
        {(void**)&p->sel, 4 * sizeof(unsigned)},
        {(void**)&p->counter, 3 * sizeof(unsigned)},
        {(void**)&p->stop, sizeof(unsigned)},
        {(void**)&p->cost_hard, n * sizeof(float)},
        {(void**)&p->wn, n * sizeof(float)},
        {(void**)&p->pit_rel, pit ? stamp::adjoint_time_rel_floats(max_particles, sc.H) * sizeof(float) : 0},
        {(void**)&p->pit_coef, pit ? pit_coef_bytes : 0},
        {(void**)&p->full, replay ? full_bytes : 0},
        {(void**)&p->full_trig, replay ? (size_t)sc.H * sc.T * n * sc.nb * sizeof(float2) : 0},
    };
    p->pit_ok = pit;
    p->replay_ok = replay;
    size_t total = 0;
    for (const Part& q : parts) total += (q.bytes + 255) / 256 * 256;
    cudaError_t e = cudaMalloc(&p->arena, total);
    if (e != cudaSuccess) {
        cudaGetLastError();
        delete p;
        return fail(STAMP_ENOMEM, "cudaMalloc of %zu bytes failed: %s", total, cudaGetErrorString(e));
    }
    size_t off = 0;
    for (const Part& q : parts) {
        *q.dst = p->arena + off;
        off += (q.bytes + 255) / 256 * 256;
    }
    const float one = 1.f;
    e = cudaStreamCreateWithFlags(&p->side, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&p->ev_theta, cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&p->ev_h, cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaMemcpy(p->one, &one, sizeof one, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemset(p->flag, 0, sizeof(int));
    if (e == cudaSuccess) e = cudaMemset(p->dropped, 0, sizeof(unsigned long long));
    if (e == cudaSuccess) e = cudaMemset(p->counter, 0, 3 * sizeof(unsigned));
    if (e != cudaSuccess) {
        cudaGetLastError();
        if (p->ev_h) cudaEventDestroy(p->ev_h);
        if (p->ev_theta) cudaEventDestroy(p->ev_theta);
        if (p->side) cudaStreamDestroy(p->side);
        cudaFree(p->arena);
        delete p;
        return fail(STAMP_ECUDA, "problem set-up failed: %s", cudaGetErrorString(e));
    }
    *out = p;
    return STAMP_OK;
}

void stamp_problem_destroy(stamp_problem* p) {
    if (!p) return;
    cudaStreamSynchronize(p->stream);
    if (p->side) cudaStreamSynchronize(p->side);
    for (cudaEvent_t e : p->ev) cudaEventDestroy(e);
    if (p->ev_h) cudaEventDestroy(p->ev_h);
    if (p->ev_theta) cudaEventDestroy(p->ev_theta);
    if (p->side) cudaStreamDestroy(p->side);
    cudaFree(p->sk_arena);
    cudaFree(p->arena);
    delete p;
}

stamp_status stamp_set_lanes(stamp_problem* p, int fwd_lanes, int adj_lanes) {
    if (!p) return fail(STAMP_EINVAL, "NULL problem");
    if ((fwd_lanes && !stamp::lanes_supported(p->sc.nb, fwd_lanes)) ||
        (adj_lanes && !stamp::lanes_supported(p->sc.nb, adj_lanes)))
        return fail(STAMP_EINVAL, "unsupported lane count for n_blocks=%d", p->sc.nb);
    p->fwd_lanes = fwd_lanes;
    p->adj_lanes = adj_lanes;
    return STAMP_OK;
}

stamp_status stamp_set_replay_lanes(stamp_problem* p, int lanes) {
    if (!p) return fail(STAMP_EINVAL, "NULL problem");
    // the replay's instantiations: one block 1-4, two 2-16, three 2-32, four 4-32 lanes
    const int lo = p->sc.nb == 1 ? 1 : p->sc.nb == 4 ? 4 : 2, hi = p->sc.nb == 1 ? 4 : p->sc.nb == 2 ? 16 : 32;
    const bool pow2 = lanes > 0 && (lanes & (lanes - 1)) == 0;
    if (lanes != 0 && !(pow2 && lanes >= lo && lanes <= hi))
        return fail(STAMP_EINVAL, "unsupported replay lane count %d for n_blocks=%d", lanes, p->sc.nb);
    p->replay_lanes = lanes;
    return STAMP_OK;
}

stamp_status stamp_rollout_fwd(stamp_problem* p, const float* theta, int N, unsigned long long seed,
                               int iter, int hard, float* cost, float* final_state) {
    if (!p) return fail(STAMP_EINVAL, "NULL problem");
    STAMP_TRY(check_n(p, N));
    STAMP_TRY(check_dev(theta, "theta"));
    STAMP_TRY(check_dev(cost, "cost"));
    STAMP_TRY(check_dev(final_state, "final_state", true));
    return fwd(p, theta, N, seed, iter, hard ? 1 : 0, cost, final_state, nullptr);
}

stamp_status stamp_rollout_fwd_from(stamp_problem* p, const float* theta, const float* init_states,
                                    int N, unsigned long long seed, int iter, int hard, float* cost,
                                    float* final_state) {
    if (!p) return fail(STAMP_EINVAL, "NULL problem");
    STAMP_TRY(check_n(p, N));
    STAMP_TRY(check_dev(theta, "theta"));
    STAMP_TRY(check_dev(init_states, "init_states"));
    STAMP_TRY(check_dev(cost, "cost"));
    STAMP_TRY(check_dev(final_state, "final_state", true));
    return fwd(p, theta, N, seed, iter, hard ? 1 : 0, cost, final_state, nullptr, init_states);
}

stamp_status stamp_rollout_adjoint(stamp_problem* p, const float* theta, int N,
                                   unsigned long long seed, int iter, float* grad_logp) {
    if (!p) return fail(STAMP_EINVAL, "NULL problem");
    STAMP_TRY(check_n(p, N));
    STAMP_TRY(check_dev(theta, "theta"));
    STAMP_TRY(check_dev(grad_logp, "grad_logp"));
    if (!p->have_tape || N != p->last_n || seed != p->last_seed || iter != p->last_iter)
        return fail(STAMP_EINVAL, "adjoint must follow stamp_rollout_fwd with the same N, seed and iter");
    return adj(p, theta, N, grad_logp);
}

stamp_status stamp_read_tape(stamp_problem* p, int N, float* tape_out) {
    if (!p) return fail(STAMP_EINVAL, "NULL problem");
    STAMP_TRY(check_dev(tape_out, "tape_out"));
    if (!p->have_tape || N != p->last_n) return fail(STAMP_EINVAL, "no tape for N=%d", N);
    STAMP_CUDA(cudaMemcpyAsync(tape_out, p->tape,
                               (size_t)(p->sc.n_ckpt + 1) * N * p->sc.S * sizeof(float),
                               cudaMemcpyDeviceToDevice, p->stream));
    return STAMP_OK;
}

stamp_status stamp_svgd_step(stamp_problem* p, float* theta, const float* grad_logp, int N,
                             float* adam_m, float* adam_v, int step, float lr, int sgd_phase,
                             float* h_out, float* phi_out) {
    if (!p) return fail(STAMP_EINVAL, "NULL problem");
    STAMP_TRY(check_n(p, N));
    STAMP_TRY(check_dev(theta, "theta"));
    STAMP_TRY(check_dev(grad_logp, "grad_logp"));
    STAMP_TRY(check_dev(adam_m, "adam_m"));
    STAMP_TRY(check_dev(adam_v, "adam_v"));
    STAMP_TRY(check_dev(h_out, "h_out", true));
    STAMP_TRY(check_dev(phi_out, "phi_out", true));
    if (step < 1) return fail(STAMP_EINVAL, "step must be >= 1");
    if ((reinterpret_cast<uintptr_t>(theta) | reinterpret_cast<uintptr_t>(grad_logp)) & 15u)
        return fail(STAMP_EINVAL, "theta and grad_logp must be 16-byte aligned");
    if (!std::isfinite(lr)) return fail(STAMP_EINVAL, "lr is not finite");
    return svgd(p, theta, grad_logp, N, adam_m, adam_v, step, lr, sgd_phase, h_out, phi_out);
}

stamp_status stamp_set_particle_offset(stamp_problem* p, int particle0) {
    if (!p) return fail(STAMP_EINVAL, "NULL problem");
    if (particle0 < 0) return fail(STAMP_EINVAL, "particle0 must be >= 0");
    p->particle0 = particle0;
    return STAMP_OK;
}

stamp_status stamp_svgd_step_rows(stamp_problem* p, const float* theta_all, const float* grad_all,
                                  int N, int row0, int rows, float* theta_rows, float* adam_m,
                                  float* adam_v, int step, float lr, int sgd_phase, float* h_out,
                                  float* phi_out) {
    if (!p) return fail(STAMP_EINVAL, "NULL problem");
    STAMP_TRY(check_n(p, N));
    if (row0 < 0 || rows < 1 || row0 + rows > N)
        return fail(STAMP_EINVAL, "rows [%d, %d) outside [0, %d)", row0, row0 + rows, N);
    STAMP_TRY(check_dev(theta_all, "theta_all"));
    STAMP_TRY(check_dev(grad_all, "grad_all"));
    STAMP_TRY(check_dev(theta_rows, "theta_rows"));
    STAMP_TRY(check_dev(adam_m, "adam_m"));
    STAMP_TRY(check_dev(adam_v, "adam_v"));
    STAMP_TRY(check_dev(h_out, "h_out", true));
    STAMP_TRY(check_dev(phi_out, "phi_out", true));
    if (step < 1) return fail(STAMP_EINVAL, "step must be >= 1");
    if ((reinterpret_cast<uintptr_t>(theta_all) | reinterpret_cast<uintptr_t>(grad_all)) & 15u)
        return fail(STAMP_EINVAL, "theta_all and grad_all must be 16-byte aligned");
    if (!std::isfinite(lr)) return fail(STAMP_EINVAL, "lr is not finite");
    if (p->kernel_kind != 0) return fail(STAMP_EINVAL, "row steps use the RBF kernel (kind 0)");
    const int D = p->sc.D;
    const float* part = grad_all + (size_t)row0 * D;   // SGD phase: phi = grad log rho
    int shares = 1;
    if (!sgd_phase) {
        // the bandwidth from every particle (replicated on each shard), phi
        // for this shard's rows, the sum over j split as for all N rows
        stamp::SvgdScratch sc{p->d2, p->hist, p->sel, p->counter, p->h, p->flag};
        STAMP_TRY(bandwidth(p, theta_all, N, h_out, p->stream));
        STAMP_TRY(timed(p, STAMP_K_PHI, [&] {
            return stamp::launch_phi_rows(theta_all, grad_all, N, D, row0, rows, sc, p->phi,
                                          stamp::kMaxShares, &shares, p->stream);
        }));
        part = p->phi;
    } else if (h_out) {
        STAMP_CUDA(cudaMemcpyAsync(h_out, p->one, sizeof(float), cudaMemcpyDeviceToDevice, p->stream));
    }
    return timed(p, STAMP_K_ADAM, [&] {
        return stamp::launch_adam(theta_rows, part, shares, phi_out, adam_m, adam_v, rows * D, step,
                                  lr, p->flag, p->stream);
    });
}

stamp_status stamp_solve(stamp_problem* p, int N, int svgd_iters, int sgd_iters,
                         unsigned long long seed, float lr, const float* theta_init,
                         float* theta_out, float* cost_out, int k, int* topk_particle,
                         float* stats_out) {
    if (!p) return fail(STAMP_EINVAL, "NULL problem");
    Phases ph{nullptr, 0, 0, svgd_iters, sgd_iters};
    return run_solve(p, ph, N, seed, lr, theta_init, theta_out, cost_out, k, topk_particle, stats_out);
}

stamp_status stamp_solve_surrogate(stamp_problem* p, stamp_surrogate* s, int n_candidates, int N,
                                   int surrogate_iters, int sim_iters, int sgd_iters,
                                   unsigned long long seed, float lr, float* theta_out,
                                   float* cost_out, int k, int* topk_particle, float* stats_out) {
    if (!p || !s) return fail(STAMP_EINVAL, "NULL problem or surrogate");
    if (stamp::surrogate_stream(s) != p->stream)
        return fail(STAMP_EINVAL, "the problem and the surrogate must share one stream");
    if (N > stamp::surrogate_max_particles(s))
        return fail(STAMP_EINVAL, "N=%d exceeds the surrogate's max_particles", N);
    if (n_candidates < N || n_candidates > stamp::surrogate_max_rows(s))
        return fail(STAMP_EINVAL, "need N <= n_candidates <= the surrogate's max_rows");
    if (n_candidates > N && N > stamp::kMaxScreenN)
        return fail(STAMP_EINVAL, "screening keeps at most %d particles", stamp::kMaxScreenN);
    if (surrogate_iters < 0 || sim_iters < 0 || sgd_iters < 0)
        return fail(STAMP_EINVAL, "negative iteration count");
    Phases ph{s, n_candidates, surrogate_iters, sim_iters, sgd_iters};
    return run_solve(p, ph, N, seed, lr, nullptr, theta_out, cost_out, k, topk_particle, stats_out);
}

stamp_status stamp_set_adjoint_mode(stamp_problem* p, int mode) {
    if (!p) return fail(STAMP_EINVAL, "NULL problem");
    if (mode != STAMP_ADJ_SEQUENTIAL && mode != STAMP_ADJ_TIME_PARALLEL && mode != STAMP_ADJ_AUTO &&
        mode != STAMP_ADJ_REPLAY)
        return fail(STAMP_EINVAL, "unknown adjoint mode %d", mode);
    p->adj_mode = mode;
    return STAMP_OK;
}

stamp_status stamp_get_adjoint_mode(stamp_problem* p, int N, int* mode) {
    if (!p || !mode) return fail(STAMP_EINVAL, "NULL problem or mode");
    STAMP_TRY(check_n(p, N));
    *mode = adjoint_kind(p, N);
    return STAMP_OK;
}

stamp_status stamp_set_overlap(stamp_problem* p, int enable) {
    if (!p) return fail(STAMP_EINVAL, "NULL problem");
    p->overlap = enable != 0;
    return STAMP_OK;
}

stamp_status stamp_set_svgd_kernel(stamp_problem* p, int kind) {
    if (!p) return fail(STAMP_EINVAL, "NULL problem");
    if (kind != 0 && kind != 1) return fail(STAMP_EINVAL, "kernel kind must be 0 (RBF) or 1 (structured)");
    if (kind == 1 && !p->sk_arena) {
        const size_t n = (size_t)p->max_n, H = p->sc.H, M = p->sc.M;
        const size_t bytes[] = {n * 2 * H * 4, n * M * H * 4, n * n * 4, 4,
                                (2048 + 2048 + 1024) * 4, 4 * 4, 3 * 4};
        size_t total = 0;
        for (size_t b : bytes) total += (b + 255) / 256 * 256;
        if (cudaMalloc(&p->sk_arena, total) != cudaSuccess) {
            cudaGetLastError();
            p->sk_arena = nullptr;
            return fail(STAMP_ENOMEM, "cudaMalloc of %zu bytes for the structured kernel failed", total);
        }
        void** dst[] = {(void**)&p->sk_C, (void**)&p->sk_S, (void**)&p->sk_d2, (void**)&p->sk_h,
                        (void**)&p->sk_hist, (void**)&p->sk_sel, (void**)&p->sk_counter};
        char* q = p->sk_arena;
        for (size_t k = 0; k < sizeof bytes / sizeof bytes[0]; ++k) {
            *dst[k] = q;
            q += (bytes[k] + 255) / 256 * 256;
        }
        STAMP_CUDA(cudaMemset(p->sk_arena, 0, total));
    }
    p->kernel_kind = kind;
    return STAMP_OK;
}

stamp_status stamp_set_dsvgd(stamp_problem* p, int enable) {
    if (!p) return fail(STAMP_EINVAL, "NULL problem");
    p->dsvgd = enable != 0;
    return STAMP_OK;
}

stamp_status stamp_svgd_step_weighted(stamp_problem* p, float* theta, const float* grad_logp,
                                      const float* cost_relaxed, const float* cost_hard, int N,
                                      float* adam_m, float* adam_v, int step, float lr,
                                      float* h_out, float* phi_out) {
    if (!p) return fail(STAMP_EINVAL, "NULL problem");
    STAMP_TRY(check_n(p, N));
    STAMP_TRY(check_dev(theta, "theta"));
    STAMP_TRY(check_dev(grad_logp, "grad_logp"));
    STAMP_TRY(check_dev(cost_relaxed, "cost_relaxed"));
    STAMP_TRY(check_dev(cost_hard, "cost_hard"));
    STAMP_TRY(check_dev(adam_m, "adam_m"));
    STAMP_TRY(check_dev(adam_v, "adam_v"));
    STAMP_TRY(check_dev(h_out, "h_out", true));
    STAMP_TRY(check_dev(phi_out, "phi_out", true));
    if (step < 1) return fail(STAMP_EINVAL, "step must be >= 1");
    if ((reinterpret_cast<uintptr_t>(theta) | reinterpret_cast<uintptr_t>(grad_logp)) & 15u)
        return fail(STAMP_EINVAL, "theta and grad_logp must be 16-byte aligned");
    if (!std::isfinite(lr)) return fail(STAMP_EINVAL, "lr is not finite");
    STAMP_CUDA(stamp::launch_dsvgd_weights(cost_relaxed, cost_hard, N, p->wn, p->stream));
    return svgd(p, theta, grad_logp, N, adam_m, adam_v, step, lr, 0, h_out, phi_out, p->wn);
}

stamp_status stamp_inject_wait_timeout(stamp_problem* p) {
    if (!p) return fail(STAMP_EINVAL, "NULL problem");
    p->inject_wait_timeout = true;
    return STAMP_OK;
}

stamp_status stamp_set_target(stamp_problem* p, float target_cost, int check_every) {
    if (!p) return fail(STAMP_EINVAL, "NULL problem");
    if (check_every < 0 || !std::isfinite(target_cost)) return fail(STAMP_EINVAL, "bad target or interval");
    p->target = target_cost;
    p->check_every = check_every;
    return STAMP_OK;
}

stamp_status stamp_solve_info(stamp_problem* p, int* iterations_run, float* best_hard_cost) {
    if (!p) return fail(STAMP_EINVAL, "NULL problem");
    if (iterations_run) *iterations_run = p->iters_run;
    if (best_hard_cost) *best_hard_cost = p->best_hard;
    return STAMP_OK;
}

stamp_status stamp_sync(stamp_problem* p) {
    if (!p) return fail(STAMP_EINVAL, "NULL problem");
    STAMP_CUDA(cudaStreamSynchronize(p->stream));
    STAMP_TRY(collect(p));
    return check_flag(p);
}

stamp_status stamp_dropped_gradients(stamp_problem* p, long long* count) {
    if (!p || !count) return fail(STAMP_EINVAL, "NULL problem or count");
    STAMP_CUDA(cudaStreamSynchronize(p->stream));
    unsigned long long n = 0;
    STAMP_CUDA(cudaMemcpy(&n, p->dropped, sizeof n, cudaMemcpyDeviceToHost));
    *count = (long long)n;
    return STAMP_OK;
}

stamp_status stamp_set_profiling(stamp_problem* p, int enable) {
    return stamp_set_profiling_mask(p, enable ? ~0u : 0u);
}

stamp_status stamp_set_profiling_mask(stamp_problem* p, unsigned mask) {
    if (!p) return fail(STAMP_EINVAL, "NULL problem");
    STAMP_CUDA(cudaStreamSynchronize(p->stream));
    if (p->side) STAMP_CUDA(cudaStreamSynchronize(p->side));
    p->ev_used = 0;
    for (int q = 0; q < STAMP_NKERNELS; ++q) { p->ms[q] = 0.0; p->launches[q] = 0; }
    p->prof = mask != 0;
    p->prof_mask = mask;
    if (p->prof && p->ev.empty()) {
        constexpr size_t kPairs = 1 << 15;
        p->ev.resize(2 * kPairs);
        for (cudaEvent_t& e : p->ev) STAMP_CUDA(cudaEventCreate(&e));
        p->ev_kind.resize(kPairs);
    }
    return STAMP_OK;
}

stamp_status stamp_get_kernel_times(stamp_problem* p, double* ms_out, long long* launches_out) {
    if (!p) return fail(STAMP_EINVAL, "NULL problem");
    for (int q = 0; q < STAMP_NKERNELS; ++q) {
        if (ms_out) ms_out[q] = p->ms[q];
        if (launches_out) launches_out[q] = p->launches[q];
    }
    return STAMP_OK;
}

}  // extern "C"
