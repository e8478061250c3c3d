// Learned pose-dynamics surrogate of the pushing simulator.
//
// One push maps the blocks' poses at the push start and the push's relaxed
// parameters (choice weights z~, offset, distance; Eq. gamma_map) to the pose
// change after the push.  The surrogate replaces the T simulated substeps of
// that map by one evaluation of the BF16 tensor-core MLP of mlp.cu:
//   f_k = [x_b, y_b, cos phi_b, sin phi_b]_b ++ z~_k ++ [tanh u_k, sigmoid v_k]
//   q_{k+1} = q_k + MLP(f_k)                            (deltas, world frame)
// and the plan's cost C (the simulator's cost on q_H) is differentiated
// through the H chained evaluations back to theta.  It is trained on
// simulator transitions from random non-overlapping poses and random actions.
#include <algorithm>
#include <cmath>
#include <cstdint>
#include <cstdio>
#include <cstring>
#include <vector>

#include "mlp.cuh"
#include "rollout.cuh"
#include "stamp.h"
#include "stamp_internal.cuh"

namespace stamp {
namespace surrogate {

constexpr uint64_t kStreamPoses = 2, kStreamActions = 3;
constexpr int kChunk = 4096;         // transitions per chunk (one key each)
constexpr int kTrainRows = 16384;    // largest training minibatch
constexpr int kAttempts = 32;        // rejection-sampling attempts per start scene
constexpr int kSelectChunk = 8192;   // keys sorted by one CTA of the screening selection

// Features of push k (and the stored relaxation).  Pose source: the scene's
// start poses (src NULL), else src (+ delta when given); the pose used is
// written to pose_out when given.
template <int NB>
__global__ void __launch_bounds__(128)
features_kernel(const SimConst sc, const float* __restrict__ theta, int N, int k, uint64_t seed,
                int iter, const float* __restrict__ src, const float* __restrict__ delta,
                float* __restrict__ pose_out, float* __restrict__ x, float* __restrict__ relax) {
    constexpr int M = rollout::Dims<NB>::M, P = M + 2, IN = 8 * NB + 2;
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= N) return;
    float q[3 * NB];
#pragma unroll
    for (int t = 0; t < 3 * NB; ++t) {
        q[t] = src ? src[(size_t)i * 3 * NB + t] : sc.init[t / 3][t % 3];
        if (delta) q[t] += delta[(size_t)i * 3 * NB + t];
        if (pose_out) pose_out[(size_t)i * 3 * NB + t] = q[t];
    }
    const bool noise = iter >= 0;
    const uint64_t gkey = noise ? sm64(sm64(seed, kStreamGumbel), (uint64_t)iter) : 0ull;
    float z[M], uu, vv;
    rollout::relax_action<NB>(sc, theta + (size_t)i * sc.D, k, i, gkey, noise, false, z, uu, vv);
    const float tu = tanhf(uu), sv = rollout::sigmoidf_(vv);
    float* xi = x + (size_t)i * IN;
#pragma unroll
    for (int b = 0; b < NB; ++b) {
        float sn, cs;
        sincosf(q[3 * b + 2], &sn, &cs);
        xi[4 * b] = q[3 * b];
        xi[4 * b + 1] = q[3 * b + 1];
        xi[4 * b + 2] = cs;
        xi[4 * b + 3] = sn;
    }
    float* ri = relax + ((size_t)i * sc.H + k) * P;
#pragma unroll
    for (int c = 0; c < M; ++c) xi[4 * NB + c] = ri[c] = z[c];
    xi[4 * NB + M] = ri[M] = tu;
    xi[4 * NB + M + 1] = ri[M + 1] = sv;
}

// q_H = q_{H-1} + delta; C = sum_b |p_b - g_b|^2 + w_yaw wrap(phi_b - phi_gb)^2
// + w_push sum_k dist_k^2 and, when apose is given, dC/dq_H.
template <int NB>
__global__ void __launch_bounds__(128)
cost_kernel(const SimConst sc, int N, const float* __restrict__ src, const float* __restrict__ delta,
            const float* __restrict__ relax, float* __restrict__ cost, float* __restrict__ apose,
            unsigned* __restrict__ stats_min) {
    constexpr int M = rollout::Dims<NB>::M, P = M + 2;
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= N) return;
    float c = 0.f;
    for (int k = 0; k < sc.H; ++k) {
        const float d = sc.dist_max * relax[((size_t)i * sc.H + k) * P + M + 1];
        c += d * d;
    }
    c *= sc.w_push;
#pragma unroll
    for (int b = 0; b < NB; ++b) {
        const size_t o = (size_t)i * 3 * NB + 3 * b;
        const float ex = src[o] + delta[o] - sc.goal[b][0];
        const float ey = src[o + 1] + delta[o + 1] - sc.goal[b][1];
        const float ew = rollout::wrapf(src[o + 2] + delta[o + 2] - sc.goal[b][2]);
        c += ex * ex + ey * ey + sc.w_yaw * ew * ew;
        if (apose) {
            apose[o] = 2.f * ex;
            apose[o + 1] = 2.f * ey;
            apose[o + 2] = 2.f * sc.w_yaw * ew;
        }
    }
    cost[i] = c;
    if (stats_min) atomicMin(stats_min, __float_as_uint(c));
}

// Reverse of push k's features: dx (N x F, dC/df_k) is added into the pose
// adjoint (which holds dC/dq_{k+1} on entry and dC/dq_k on exit) and gives
// grad log rho = -dC/dtheta for push k's parameters (with the w_push term).
template <int NB>
__global__ void __launch_bounds__(128)
features_bwd_kernel(const SimConst sc, int N, int k, const float* __restrict__ pose,
                    const float* __restrict__ relax, const float* __restrict__ dx,
                    float* __restrict__ apose, float* __restrict__ grad) {
    constexpr int M = rollout::Dims<NB>::M, P = M + 2, IN = 8 * NB + 2;
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= N) return;
    const float* di = dx + (size_t)i * IN;
    const float* pi = pose + (size_t)i * 3 * NB;
    float* ai = apose + (size_t)i * 3 * NB;
#pragma unroll
    for (int b = 0; b < NB; ++b) {
        float sn, cs;
        sincosf(pi[3 * b + 2], &sn, &cs);
        ai[3 * b] += di[4 * b];
        ai[3 * b + 1] += di[4 * b + 1];
        ai[3 * b + 2] += cs * di[4 * b + 3] - sn * di[4 * b + 2];
    }
    const float* ri = relax + ((size_t)i * sc.H + k) * P;
    float zg = 0.f;
#pragma unroll
    for (int c = 0; c < M; ++c) zg += ri[c] * di[4 * NB + c];
    float* gi = grad + (size_t)i * sc.D + k * P;
    // softmax((a+g)/tau): dC/da_j = z_j (dC/dz_j - sum_c z_c dC/dz_c) / tau
#pragma unroll
    for (int c = 0; c < M; ++c) gi[c] = -(ri[c] * (di[4 * NB + c] - zg) * sc.inv_tau);
    const float tu = ri[M], sv = ri[M + 1];
    gi[M] = -(di[4 * NB + M] * (1.f - tu * tu));
    const float dist = sc.dist_max * sv;
    gi[M + 1] = -((di[4 * NB + M + 1] + 2.f * sc.w_push * dist * sc.dist_max) * sv * (1.f - sv));
}

// Random start scenes: the first of kAttempts counter-based draws whose block
// centres are all more than 0.16 m apart; products and sums in float32 with
// explicit rounding so that the accept decision is reproducible.
__global__ void sample_poses_kernel(int m, int nb, uint64_t cs, float* __restrict__ poses) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= m) return;
    const uint64_t key = sm64(cs, kStreamPoses);
    const float thr = 0.16f * 0.16f;
    float p[kMaxBlocks][3];
    bool ok = false;
    for (int att = 0; att < kAttempts && !ok; ++att) {
        const uint64_t base = ((uint64_t)i * kAttempts + att) * 3 * kMaxBlocks;
        for (int b = 0; b < nb; ++b) {
            p[b][0] = __fsub_rn(u23(sm64(key, base + 3 * b)), 0.5f);
            p[b][1] = __fsub_rn(u23(sm64(key, base + 3 * b + 1)), 0.5f);
            p[b][2] = __fmul_rn(__fsub_rn(u23(sm64(key, base + 3 * b + 2)), 0.5f), 3.14159265f);
        }
        ok = true;
        for (int a = 0; a < nb; ++a)
            for (int b = a + 1; b < nb; ++b) {
                const float dx = __fsub_rn(p[a][0], p[b][0]), dy = __fsub_rn(p[a][1], p[b][1]);
                ok = ok && __fadd_rn(__fmul_rn(dx, dx), __fmul_rn(dy, dy)) > thr;
            }
    }
    if (!ok) {
        const float den = (float)max(nb - 1, 1);
        for (int b = 0; b < nb; ++b) p[b][0] = __fadd_rn(-0.4f, __fdiv_rn(__fmul_rn(0.8f, (float)b), den));
    }
    for (int b = 0; b < nb; ++b)
        for (int q = 0; q < 3; ++q) poses[(size_t)i * 3 * nb + 3 * b + q] = p[b][q];
}

// Random action parameters: row i draws u_0..u_{P-1} and w (counter
// i (P+1) + j, w last); theta_j = (u_j - 1/2) * 6, the M logits further
// scaled by w so that the choice weights range from nearly uniform to nearly
// one-hot.  Each product rounded once.
__global__ void sample_actions_kernel(int m, int M, uint64_t cs, float* __restrict__ theta) {
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    const int P = M + 2;
    if (t >= m * P) return;
    const int i = t / P, j = t % P;
    const uint64_t key = sm64(cs, kStreamActions);
    float v = __fmul_rn(__fsub_rn(u23(sm64(key, (uint64_t)i * (P + 1) + j)), 0.5f), 6.f);
    if (j < M) v = __fmul_rn(v, u23(sm64(key, (uint64_t)i * (P + 1) + P)));
    theta[t] = v;
}

// Transition targets: each block's pose change over the push.
__global__ void delta_kernel(int m, int nb, const float* __restrict__ start,
                             const float* __restrict__ final_state, float* __restrict__ y) {
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= m * 3 * nb) return;
    const int i = t / (3 * nb), r = t % (3 * nb), b = r / 3, q = r % 3;
    y[t] = final_state[(size_t)i * 6 * nb + 6 * b + q] - start[t];
}

// Sort keys (cost bits << 32 | index; a negative or NaN cost sorts last).
__global__ void keys_kernel(const float* __restrict__ cost, int n, unsigned long long* __restrict__ keys) {
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= n) return;
    unsigned cb = __float_as_uint(cost[t]);
    if (cb >= 0x7F800001u) cb = 0xFFFFFFFFu;
    keys[t] = ((unsigned long long)cb << 32) | (unsigned)t;
}

// Each CTA bitonic-sorts one chunk of kSelectChunk keys in shared memory
// (missing keys padded with the largest key) and writes its `keep` smallest.
__global__ void __launch_bounds__(1024)
select_kernel(const unsigned long long* __restrict__ in, int n, int keep,
              unsigned long long* __restrict__ out) {
    extern __shared__ unsigned long long key[];
    const int c0 = blockIdx.x * kSelectChunk, m = min(kSelectChunk, n - c0);
    for (int t = threadIdx.x; t < kSelectChunk; t += blockDim.x) key[t] = t < m ? in[c0 + t] : ~0ull;
    __syncthreads();
    for (int size = 2; size <= kSelectChunk; size <<= 1)
        for (int stride = size >> 1; stride > 0; stride >>= 1) {
            for (int t = threadIdx.x; t < kSelectChunk / 2; t += blockDim.x) {
                const int lo = 2 * t - (t & (stride - 1)), hi = lo + stride;
                const bool up = (lo & size) == 0;
                const unsigned long long a = key[lo], b = key[hi];
                if ((a > b) == up) { key[lo] = b; key[hi] = a; }
            }
            __syncthreads();
        }
    for (int t = threadIdx.x; t < keep; t += blockDim.x) out[(size_t)blockIdx.x * keep + t] = key[t];
}

__global__ void gather_kernel(const unsigned long long* __restrict__ keys, int N, int D,
                              const float* __restrict__ cand, float* __restrict__ theta,
                              int* __restrict__ index) {
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= N * D) return;
    const int i = t / D, d = t % D;
    const int src = (int)(keys[i] & 0xFFFFFFFFull);
    theta[t] = cand[(size_t)src * D + d];
    if (index && d == 0) index[i] = src;
}

// Uniform(-1/sqrt(fan_in), 1/sqrt(fan_in)) parameters; draw t of key `seed`.
__global__ void init_params_kernel(float* __restrict__ params, int in_dim, int out_dim, uint64_t seed) {
    const size_t t = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= mlp::param_count(in_dim, out_dim)) return;
    const int fan_in = t < mlp::param_offset(1, in_dim, out_dim) ? in_dim : mlp::kHidden;
    params[t] = (2.f * u23(sm64(seed, t)) - 1.f) * rsqrtf((float)fan_in);
}

// ---- training-set preparation ------------------------------------------------
constexpr int kPrepRows = 256;        // rows per CTA of the compaction
constexpr int kMomentCtas = 256;      // CTAs of the target-moment reduction

// A transition is kept when every block moved at most 0.5 m and turned at
// most pi: larger changes from one push of at most dist_max are blow-ups of
// the explicit contact integration, not dynamics to learn.
__device__ __forceinline__ bool keep_row(const float* y, int out) {
    bool ok = true;
    for (int c = 0; c < out; ++c) {
        const float v = y[c];
        ok = ok && isfinite(v) && fabsf(v) <= ((c % 3 == 2) ? 3.14159265f : 0.5f);
    }
    return ok;
}

__global__ void __launch_bounds__(kPrepRows)
count_kept_kernel(const float* __restrict__ y, int n, int out, int* __restrict__ counts) {
    const int i = blockIdx.x * kPrepRows + threadIdx.x;
    const int k = __syncthreads_count(i < n && keep_row(y + (size_t)i * out, out));
    if (threadIdx.x == 0) counts[blockIdx.x] = k;
}

// Stable compaction: row i goes to offsets[block] + (kept rows before it in its block).
__global__ void __launch_bounds__(kPrepRows)
compact_kernel(const float* __restrict__ x, const float* __restrict__ y, int n, int in, int out,
               const int* __restrict__ offsets, float* __restrict__ xs, float* __restrict__ ys) {
    __shared__ int warp_tot[kPrepRows / 32];
    const int i = blockIdx.x * kPrepRows + threadIdx.x;
    const bool k = i < n && keep_row(y + (size_t)i * out, out);
    const unsigned ballot = __ballot_sync(0xffffffffu, k);
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    if (lane == 0) warp_tot[w] = __popc(ballot);
    __syncthreads();
    int before = __popc(ballot & ((1u << lane) - 1u));
    for (int q = 0; q < w; ++q) before += warp_tot[q];
    if (!k) return;
    const size_t dst = (size_t)offsets[blockIdx.x] + before;
    for (int c = 0; c < in; ++c) xs[dst * in + c] = x[(size_t)i * in + c];
    for (int c = 0; c < out; ++c) ys[dst * out + c] = y[(size_t)i * out + c];
}

// Per-CTA partial sums (double) of y_c and y_c^2 over a strided share of rows.
__global__ void __launch_bounds__(256)
moments_kernel(const float* __restrict__ y, int m, int out, double* __restrict__ partial) {
    __shared__ double red[2][256];
    for (int c = 0; c < out; ++c) {
        double s1 = 0.0, s2 = 0.0;
        for (int i = blockIdx.x * 256 + threadIdx.x; i < m; i += kMomentCtas * 256) {
            const double v = y[(size_t)i * out + c];
            s1 += v;
            s2 += v * v;
        }
        red[0][threadIdx.x] = s1;
        red[1][threadIdx.x] = s2;
        __syncthreads();
        for (int o = 128; o > 0; o >>= 1) {
            if (threadIdx.x < o) {
                red[0][threadIdx.x] += red[0][threadIdx.x + o];
                red[1][threadIdx.x] += red[1][threadIdx.x + o];
            }
            __syncthreads();
        }
        if (threadIdx.x == 0) {
            partial[((size_t)blockIdx.x * out + c) * 2] = red[0][0];
            partial[((size_t)blockIdx.x * out + c) * 2 + 1] = red[1][0];
        }
        __syncthreads();
    }
}

__global__ void standardize_kernel(float* __restrict__ ys, int m, int out, const float* __restrict__ mu,
                                   const float* __restrict__ sd) {
    const size_t t = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= (size_t)m * out) return;
    const int c = (int)(t % out);
    ys[t] = (ys[t] - mu[c]) / sd[c];
}

// Head of the network in target units (fold = 1) or in standardized units
// (fold = 0): W4 row c and b4_c scaled by sd_c, mu_c added to the bias, or
// the inverse.  src and dst may be the same vector.
__global__ void head_scale_kernel(const float* __restrict__ src, float* __restrict__ dst, int in_dim,
                                  int out_dim, const float* __restrict__ mu, const float* __restrict__ sd,
                                  int fold) {
    const size_t n = mlp::param_count(in_dim, out_dim), h = mlp::param_offset(3, in_dim, out_dim);
    const size_t t = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= n) return;
    float v = src[t];
    if (t >= h) {
        const size_t r = t - h, wsz = (size_t)out_dim * mlp::kHidden;
        const int c = r < wsz ? (int)(r / mlp::kHidden) : (int)(r - wsz);
        if (fold) v = v * sd[c] + (r < wsz ? 0.f : mu[c]);
        else v = r < wsz ? v / sd[c] : (v - mu[c]) / sd[c];
    }
    dst[t] = v;
}

template <int NB>
cudaError_t features(const SimConst& sc, const float* theta, int N, int k, uint64_t seed, int iter,
                     const float* src, const float* delta, float* pose_out, float* x, float* relax,
                     cudaStream_t st) {
    features_kernel<NB><<<(N + 127) / 128, 128, 0, st>>>(sc, theta, N, k, seed, iter, src, delta,
                                                         pose_out, x, relax);
    return cudaGetLastError();
}
template <int NB>
cudaError_t cost(const SimConst& sc, int N, const float* src, const float* delta, const float* relax,
                 float* c, float* apose, unsigned* stats, cudaStream_t st) {
    cost_kernel<NB><<<(N + 127) / 128, 128, 0, st>>>(sc, N, src, delta, relax, c, apose, stats);
    return cudaGetLastError();
}
template <int NB>
cudaError_t features_bwd(const SimConst& sc, int N, int k, const float* pose, const float* relax,
                         const float* dx, float* apose, float* grad, cudaStream_t st) {
    features_bwd_kernel<NB><<<(N + 127) / 128, 128, 0, st>>>(sc, N, k, pose, relax, dx, apose, grad);
    return cudaGetLastError();
}

cudaError_t features_nb(const SimConst& sc, const float* theta, int N, int k, uint64_t seed, int iter,
                        const float* src, const float* delta, float* pose_out, float* x, float* relax,
                        cudaStream_t st) {
    switch (sc.nb) {
        case 1: return features<1>(sc, theta, N, k, seed, iter, src, delta, pose_out, x, relax, st);
        case 2: return features<2>(sc, theta, N, k, seed, iter, src, delta, pose_out, x, relax, st);
        case 3: return features<3>(sc, theta, N, k, seed, iter, src, delta, pose_out, x, relax, st);
    }
    return cudaErrorInvalidValue;
}
cudaError_t cost_nb(const SimConst& sc, int N, const float* src, const float* delta, const float* relax,
                    float* c, float* apose, unsigned* stats, cudaStream_t st) {
    switch (sc.nb) {
        case 1: return cost<1>(sc, N, src, delta, relax, c, apose, stats, st);
        case 2: return cost<2>(sc, N, src, delta, relax, c, apose, stats, st);
        case 3: return cost<3>(sc, N, src, delta, relax, c, apose, stats, st);
    }
    return cudaErrorInvalidValue;
}
cudaError_t features_bwd_nb(const SimConst& sc, int N, int k, const float* pose, const float* relax,
                            const float* dx, float* apose, float* grad, cudaStream_t st) {
    switch (sc.nb) {
        case 1: return features_bwd<1>(sc, N, k, pose, relax, dx, apose, grad, st);
        case 2: return features_bwd<2>(sc, N, k, pose, relax, dx, apose, grad, st);
        case 3: return features_bwd<3>(sc, N, k, pose, relax, dx, apose, grad, st);
    }
    return cudaErrorInvalidValue;
}

}  // namespace surrogate
}  // namespace stamp

// ------------------------------- object ----------------------------------------
struct stamp_surrogate {
    int nb = 0, max_H = 0, M = 0, in_dim = 0, out_dim = 0, max_rows = 0, max_n = 0;
    int last_kept = 0;   // transitions the last training call kept
    size_t n_params = 0;
    cudaStream_t stream = nullptr;
    stamp_mlp* mlp = nullptr;
    stamp_problem* trans = nullptr;   // one-push simulator (H = 1) for transitions
    char* arena = nullptr;
    float *params = nullptr, *pose = nullptr, *x = nullptr, *y = nullptr, *relax = nullptr,
          *apose = nullptr, *dx = nullptr, *cost = nullptr, *cand = nullptr, *tstart = nullptr,
          *tfinal = nullptr, *taction = nullptr, *tcost = nullptr;
    unsigned long long *keys = nullptr, *keys2 = nullptr;
};

namespace {

stamp_status sur_fail(stamp_status s, const char* msg, cudaError_t e = cudaSuccess) {
    char buf[320];
    std::snprintf(buf, sizeof buf, "%s%s%s", msg, e != cudaSuccess ? ": " : "",
                  e != cudaSuccess ? cudaGetErrorString(e) : "");
    if (e != cudaSuccess) cudaGetLastError();
    stamp::set_last_error(buf);
    return s;
}
#define SUR_CUDA(call, what)                                           \
    do {                                                               \
        cudaError_t e_ = (call);                                       \
        if (e_ != cudaSuccess) return sur_fail(STAMP_ECUDA, what, e_); \
    } while (0)
#define SUR_TRY(x)                     \
    do {                               \
        stamp_status s_ = (x);         \
        if (s_ != STAMP_OK) return s_; \
    } while (0)

bool dev_ptr(const void* p) {
    if (!p) return false;
    cudaPointerAttributes at;
    if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return at.type == cudaMemoryTypeDevice || at.type == cudaMemoryTypeManaged;
}

stamp_status check_problem(const stamp_surrogate* s, const stamp::SimConst& sc) {
    if (sc.nb != s->nb) return sur_fail(STAMP_EINVAL, "the problem's block count differs from the surrogate's");
    if (sc.H > s->max_H) return sur_fail(STAMP_EINVAL, "the problem's horizon exceeds the surrogate's");
    return STAMP_OK;
}

}  // namespace

namespace stamp {

stamp_status surrogate_rollout(stamp_surrogate* s, const SimConst& sc, const float* theta, int N,
                               uint64_t seed, int iter, float* cost, float* grad, unsigned* stats_word) {
    SUR_TRY(check_problem(s, sc));
    const bool rev = grad != nullptr;
    if (N < 1 || N > (rev ? s->max_n : s->max_rows))
        return sur_fail(STAMP_EINVAL, "N outside the surrogate's capacity");
    const int S3 = 3 * s->nb, tiles = (N + 127) / 128;
    cudaStream_t st = s->stream;
    for (int k = 0; k < sc.H; ++k) {
        const float* prev = k ? s->pose + (size_t)(k - 1) * N * S3 : nullptr;
        SUR_CUDA(surrogate::features_nb(sc, theta, N, k, seed, iter, prev, k ? s->y : nullptr,
                                        s->pose + (size_t)k * N * S3, s->x, s->relax, st),
                 "feature launch failed");
        SUR_TRY(rev ? stamp_mlp_forward_saved(s->mlp, s->x, N, s->y, k * tiles)
                    : stamp_mlp_forward(s->mlp, s->x, N, s->y));
    }
    SUR_CUDA(surrogate::cost_nb(sc, N, s->pose + (size_t)(sc.H - 1) * N * S3, s->y, s->relax, cost,
                                rev ? s->apose : nullptr, stats_word, st),
             "cost launch failed");
    if (!rev) return STAMP_OK;
    for (int k = sc.H - 1; k >= 0; --k) {
        // q_{k+1} = q_k + y_k: dC/dy_k = dC/dq_{k+1}
        SUR_TRY(stamp_mlp_backward(s->mlp, s->apose, N, k * tiles, s->dx, nullptr));
        SUR_CUDA(surrogate::features_bwd_nb(sc, N, k, s->pose + (size_t)k * N * S3, s->relax, s->dx,
                                            s->apose, grad, st),
                 "feature backward failed");
    }
    return STAMP_OK;
}

stamp_status surrogate_screen(stamp_surrogate* s, const SimConst& sc, const float* cand, int n_cand,
                              int N, float* theta_out, int* index_out) {
    SUR_TRY(check_problem(s, sc));
    if (N < 1 || N > n_cand || N > kMaxScreenN || n_cand > s->max_rows)
        return sur_fail(STAMP_EINVAL, "need 1 <= N <= min(n_candidates, 4096) and n_candidates <= max_rows");
    SUR_TRY(surrogate_rollout(s, sc, cand, n_cand, 0, -1, s->cost, nullptr, nullptr));
    using surrogate::kSelectChunk;
    const size_t smem = kSelectChunk * sizeof(unsigned long long);
    SUR_CUDA(cudaFuncSetAttribute(surrogate::select_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                  (int)smem), "shared-memory opt-in failed");
    surrogate::keys_kernel<<<(n_cand + 255) / 256, 256, 0, s->stream>>>(s->cost, n_cand, s->keys);
    unsigned long long *a = s->keys, *b = s->keys2;
    int n = n_cand;
    while (n > kSelectChunk) {   // N <= 4096 keeps at most half of every full chunk: n shrinks
        const int chunks = (n + kSelectChunk - 1) / kSelectChunk;
        surrogate::select_kernel<<<chunks, 1024, smem, s->stream>>>(a, n, N, b);
        n = chunks * N;
        std::swap(a, b);
    }
    surrogate::select_kernel<<<1, 1024, smem, s->stream>>>(a, n, N, b);
    const int D = sc.D;
    surrogate::gather_kernel<<<(N * D + 255) / 256, 256, 0, s->stream>>>(b, N, D, cand, theta_out, index_out);
    SUR_CUDA(cudaGetLastError(), "selection launch failed");
    return STAMP_OK;
}

float* surrogate_candidates(stamp_surrogate* s) { return s->cand; }
int surrogate_max_rows(const stamp_surrogate* s) { return s->max_rows; }
int surrogate_max_particles(const stamp_surrogate* s) { return s->max_n; }
cudaStream_t surrogate_stream(const stamp_surrogate* s) { return s->stream; }

}  // namespace stamp

extern "C" {

stamp_status stamp_surrogate_create(const stamp_problem_desc* desc, int max_rows, int max_particles,
                                    void* cuda_stream, stamp_surrogate** out) {
    if (!out) return sur_fail(STAMP_EINVAL, "out is NULL");
    *out = nullptr;
    if (!desc) return sur_fail(STAMP_EINVAL, "NULL description");
    if (desc->n_blocks < 1 || desc->n_blocks > 3) return sur_fail(STAMP_EINVAL, "the surrogate takes 1 to 3 blocks");
    if (desc->H < 1 || desc->H > stamp::kMaxH) return sur_fail(STAMP_EINVAL, "H outside [1, 16]");
    if (max_particles < 1 || max_particles > max_rows || max_rows > (1 << 20))
        return sur_fail(STAMP_EINVAL, "need 1 <= max_particles <= max_rows <= 2^20");
    // the one-push simulator that generates transitions (start poses per particle)
    stamp_problem_desc d1 = *desc;
    d1.H = 1;
    d1.ckpt_every = d1.T;
    const float zeros[3 * stamp::kMaxBlocks] = {};
    stamp_problem* trans = nullptr;
    SUR_TRY(stamp_problem_create(&d1, zeros, zeros, stamp::surrogate::kChunk, cuda_stream, &trans));
    stamp_surrogate* s = new stamp_surrogate();
    s->trans = trans;
    s->nb = desc->n_blocks; s->max_H = desc->H; s->M = 4 * s->nb;
    s->in_dim = 8 * s->nb + 2; s->out_dim = 3 * s->nb;
    s->max_rows = max_rows; s->max_n = max_particles;
    s->n_params = stamp_mlp_param_count(s->in_dim, s->out_dim);
    s->stream = static_cast<cudaStream_t>(cuda_stream);
    const size_t R = std::max(max_rows, stamp::surrogate::kChunk), S3 = 3 * s->nb, P = s->M + 2;
    const int train_rows = std::max(stamp::surrogate::kTrainRows, s->max_H * ((max_particles + 127) / 128) * 128);
    stamp_status r = stamp_mlp_create(s->in_dim, s->out_dim, (int)R, train_rows, cuda_stream, &s->mlp);
    if (r != STAMP_OK) { stamp_problem_destroy(trans); delete s; return r; }
    const size_t C = stamp::surrogate::kChunk;
    const size_t bytes[] = {s->n_params * 4, (size_t)s->max_H * R * S3 * 4, R * s->in_dim * 4,
                            R * s->out_dim * 4, R * s->max_H * P * 4, (size_t)max_particles * S3 * 4,
                            (size_t)max_particles * s->in_dim * 4, R * 4, R * s->max_H * P * 4,
                            C * S3 * 4, C * 6 * s->nb * 4, C * P * 4, C * 4, R * 8, R * 8};
    void** dst[] = {(void**)&s->params, (void**)&s->pose, (void**)&s->x, (void**)&s->y,
                    (void**)&s->relax, (void**)&s->apose, (void**)&s->dx, (void**)&s->cost,
                    (void**)&s->cand, (void**)&s->tstart, (void**)&s->tfinal, (void**)&s->taction,
                    (void**)&s->tcost, (void**)&s->keys, (void**)&s->keys2};
    size_t total = 0;
    for (size_t b : bytes) total += (b + 255) / 256 * 256;
    cudaError_t e = cudaMalloc(&s->arena, total);
    if (e != cudaSuccess) {
        stamp_mlp_destroy(s->mlp); stamp_problem_destroy(trans); delete s;
        return sur_fail(STAMP_ENOMEM, "cudaMalloc failed", e);
    }
    char* p = s->arena;
    for (size_t q = 0; q < sizeof bytes / sizeof bytes[0]; ++q) {
        *dst[q] = p;
        p += (bytes[q] + 255) / 256 * 256;
    }
    e = cudaMemset(s->arena, 0, total);
    if (e != cudaSuccess) {
        stamp_surrogate_destroy(s);
        return sur_fail(STAMP_ECUDA, "memset failed", e);
    }
    *out = s;
    return STAMP_OK;
}

void stamp_surrogate_destroy(stamp_surrogate* s) {
    if (!s) return;
    cudaStreamSynchronize(s->stream);
    stamp_mlp_destroy(s->mlp);
    stamp_problem_destroy(s->trans);
    cudaFree(s->arena);
    delete s;
}

int stamp_surrogate_dims(const stamp_surrogate* s, int* in_dim, int* out_dim) {
    if (!s) return 0;
    if (in_dim) *in_dim = s->in_dim;
    if (out_dim) *out_dim = s->out_dim;
    return (int)s->n_params;
}

stamp_status stamp_surrogate_init_params(stamp_surrogate* s, unsigned long long seed) {
    if (!s) return sur_fail(STAMP_EINVAL, "NULL surrogate");
    stamp::surrogate::init_params_kernel<<<(unsigned)((s->n_params + 255) / 256), 256, 0, s->stream>>>(
        s->params, s->in_dim, s->out_dim, seed);
    SUR_CUDA(cudaGetLastError(), "parameter initialisation failed");
    return stamp_mlp_set_params(s->mlp, s->params);
}

stamp_status stamp_surrogate_set_params(stamp_surrogate* s, const float* params) {
    if (!s || !dev_ptr(params)) return sur_fail(STAMP_EINVAL, "NULL surrogate or non-device params");
    SUR_CUDA(cudaMemcpyAsync(s->params, params, s->n_params * 4, cudaMemcpyDeviceToDevice, s->stream),
             "parameter copy failed");
    return stamp_mlp_set_params(s->mlp, s->params);
}

stamp_status stamp_surrogate_get_params(stamp_surrogate* s, float* params) {
    if (!s || !dev_ptr(params)) return sur_fail(STAMP_EINVAL, "NULL surrogate or non-device params");
    SUR_CUDA(cudaMemcpyAsync(params, s->params, s->n_params * 4, cudaMemcpyDeviceToDevice, s->stream),
             "parameter copy failed");
    return STAMP_OK;
}

stamp_status stamp_surrogate_transitions(stamp_surrogate* s, int n, unsigned long long seed,
                                         float* x_out, float* y_out) {
    if (!s || n < 1 || !dev_ptr(x_out) || !dev_ptr(y_out))
        return sur_fail(STAMP_EINVAL, "NULL surrogate, n < 1 or non-device output");
    using stamp::surrogate::kChunk;
    const int nb = s->nb, S3 = 3 * nb, P = s->M + 2;
    const stamp::SimConst sc1 = stamp::problem_const(s->trans);
    for (int c0 = 0; c0 < n; c0 += kChunk) {
        const int m = std::min(kChunk, n - c0);
        const uint64_t cs = stamp::sm64(seed, (uint64_t)c0);
        stamp::surrogate::sample_poses_kernel<<<(m + 127) / 128, 128, 0, s->stream>>>(m, nb, cs, s->tstart);
        stamp::surrogate::sample_actions_kernel<<<(m * P + 255) / 256, 256, 0, s->stream>>>(m, s->M, cs, s->taction);
        SUR_CUDA(cudaGetLastError(), "sampling launch failed");
        SUR_TRY(stamp::rollout_from(s->trans, s->taction, s->tstart, m, cs, 0, s->tcost, s->tfinal));
        SUR_CUDA(stamp::surrogate::features_nb(sc1, s->taction, m, 0, cs, 0, s->tstart, nullptr, nullptr,
                                               x_out + (size_t)c0 * s->in_dim, s->relax, s->stream),
                 "feature launch failed");
        stamp::surrogate::delta_kernel<<<(m * S3 + 255) / 256, 256, 0, s->stream>>>(
            m, nb, s->tstart, s->tfinal, y_out + (size_t)c0 * S3);
        SUR_CUDA(cudaGetLastError(), "target launch failed");
    }
    return STAMP_OK;
}

stamp_status stamp_surrogate_train(stamp_surrogate* s, const float* x, const float* y, int n,
                                   int epochs, int batch, float lr, float* loss_out) {
    using namespace stamp::surrogate;
    if (!s || n < 1 || !dev_ptr(x) || !dev_ptr(y)) return sur_fail(STAMP_EINVAL, "NULL surrogate, n < 1 or non-device data");
    if (epochs < 1 || batch < 1 || !std::isfinite(lr)) return sur_fail(STAMP_EINVAL, "bad epochs, batch or lr");
    const int in = s->in_dim, out = s->out_dim, blocks = (n + kPrepRows - 1) / kPrepRows;
    cudaStream_t st = s->stream;
    // scratch of this call: the kept rows, standardized targets, block offsets, moments
    const size_t bytes[] = {(size_t)n * in * 4, (size_t)n * out * 4, (size_t)blocks * 4,
                            (size_t)kMomentCtas * out * 2 * 8, (size_t)2 * out * 4, s->n_params * 4};
    size_t total = 0;
    for (size_t b : bytes) total += (b + 255) / 256 * 256;
    char* arena = nullptr;
    SUR_CUDA(cudaMalloc(&arena, total), "training scratch allocation failed");
    char* q = arena;
    float* xs = reinterpret_cast<float*>(q); q += (bytes[0] + 255) / 256 * 256;
    float* ys = reinterpret_cast<float*>(q); q += (bytes[1] + 255) / 256 * 256;
    int* offs = reinterpret_cast<int*>(q); q += (bytes[2] + 255) / 256 * 256;
    double* partial = reinterpret_cast<double*>(q); q += (bytes[3] + 255) / 256 * 256;
    float* musd = reinterpret_cast<float*>(q); q += (bytes[4] + 255) / 256 * 256;
    float* pn = reinterpret_cast<float*>(q);
    auto body = [&]() -> stamp_status {
        count_kept_kernel<<<blocks, kPrepRows, 0, st>>>(y, n, out, offs);
        SUR_CUDA(cudaGetLastError(), "count launch failed");
        std::vector<int> h(blocks);
        SUR_CUDA(cudaMemcpyAsync(h.data(), offs, blocks * sizeof(int), cudaMemcpyDeviceToHost, st), "copy failed");
        SUR_CUDA(cudaStreamSynchronize(st), "synchronisation failed");
        int m = 0;
        for (int b = 0; b < blocks; ++b) { const int c = h[b]; h[b] = m; m += c; }
        if (m < 1) return sur_fail(STAMP_EINVAL, "no usable transition (all blew up)");
        SUR_CUDA(cudaMemcpyAsync(offs, h.data(), blocks * sizeof(int), cudaMemcpyHostToDevice, st), "copy failed");
        compact_kernel<<<blocks, kPrepRows, 0, st>>>(x, y, n, in, out, offs, xs, ys);
        moments_kernel<<<kMomentCtas, 256, 0, st>>>(ys, m, out, partial);
        SUR_CUDA(cudaGetLastError(), "compaction launch failed");
        std::vector<double> pt((size_t)kMomentCtas * out * 2);
        SUR_CUDA(cudaMemcpyAsync(pt.data(), partial, pt.size() * 8, cudaMemcpyDeviceToHost, st), "copy failed");
        SUR_CUDA(cudaStreamSynchronize(st), "synchronisation failed");
        std::vector<float> hm(2 * out);
        for (int c = 0; c < out; ++c) {
            double s1 = 0.0, s2 = 0.0;
            for (int b = 0; b < kMomentCtas; ++b) {
                s1 += pt[((size_t)b * out + c) * 2];
                s2 += pt[((size_t)b * out + c) * 2 + 1];
            }
            const double mean = s1 / m, var = std::max(s2 / m - mean * mean, 0.0);
            hm[c] = (float)mean;
            hm[out + c] = (float)std::max(std::sqrt(var), 1e-6);
        }
        SUR_CUDA(cudaMemcpyAsync(musd, hm.data(), 2 * out * sizeof(float), cudaMemcpyHostToDevice, st), "copy failed");
        standardize_kernel<<<(unsigned)(((size_t)m * out + 255) / 256), 256, 0, st>>>(ys, m, out, musd, musd + out);
        const unsigned pg = (unsigned)((s->n_params + 255) / 256);
        head_scale_kernel<<<pg, 256, 0, st>>>(s->params, pn, in, out, musd, musd + out, 0);
        SUR_CUDA(cudaGetLastError(), "standardisation launch failed");
        SUR_TRY(stamp_mlp_train(s->mlp, pn, xs, ys, m, epochs, std::min(batch, m), lr, loss_out));
        head_scale_kernel<<<pg, 256, 0, st>>>(pn, s->params, in, out, musd, musd + out, 1);
        SUR_CUDA(cudaGetLastError(), "fold launch failed");
        SUR_TRY(stamp_mlp_set_params(s->mlp, s->params));
        SUR_CUDA(cudaStreamSynchronize(st), "synchronisation failed");
        s->last_kept = m;
        return STAMP_OK;
    };
    const stamp_status r = body();
    cudaStreamSynchronize(st);
    cudaFree(arena);
    return r;
}

int stamp_surrogate_last_kept(const stamp_surrogate* s) { return s ? s->last_kept : 0; }

stamp_status stamp_surrogate_rollout(stamp_surrogate* s, stamp_problem* p, const float* theta, int N,
                                     unsigned long long seed, int iter, float* cost, float* grad_logp) {
    if (!s || !p || !dev_ptr(theta) || !dev_ptr(cost) || (grad_logp && !dev_ptr(grad_logp)))
        return sur_fail(STAMP_EINVAL, "NULL object or non-device argument");
    return stamp::surrogate_rollout(s, stamp::problem_const(p), theta, N, seed, iter, cost, grad_logp,
                                    nullptr);
}

stamp_status stamp_surrogate_screen(stamp_surrogate* s, stamp_problem* p, const float* candidates,
                                    int n_candidates, int N, float* theta_out, int* index_out) {
    if (!s || !p || !dev_ptr(candidates) || !dev_ptr(theta_out) || (index_out && !dev_ptr(index_out)))
        return sur_fail(STAMP_EINVAL, "NULL object or non-device argument");
    return stamp::surrogate_screen(s, stamp::problem_const(p), candidates, n_candidates, N, theta_out,
                                   index_out);
}

stamp_status stamp_surrogate_sync(stamp_surrogate* s) {
    if (!s) return sur_fail(STAMP_EINVAL, "NULL surrogate");
    SUR_CUDA(cudaStreamSynchronize(s->stream), "stream synchronisation failed");
    return stamp_mlp_sync(s->mlp);
}

}  // extern "C"
