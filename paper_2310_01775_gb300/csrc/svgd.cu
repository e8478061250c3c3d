// Stein update of Algorithm 1 (Eq. svgd with unit weights), its median
// bandwidth, Adam, the initial particles and the final distinct-plan top-k.
//
// Bandwidth: h = med/ln(N+1), med the lower median (rank floor((M-1)/2)) of
// the M = N(N-1)/2 squared distances d2_ij, i<j -- the median heuristic the
// paper uses for its RBF kernels (App. C.3).  It is selected exactly by a
// three-digit radix select on the float bits (11 + 11 + 10 bits; the bits of
// non-negative floats order like the floats) over the d2 matrix, which stays
// in L2 (4 MB at N = 1024).  Each pass histograms one digit; the last CTA of
// the pass to finish (a device-scope counter, no waiting) picks the digit for
// the next pass, and the last pass writes h.
#include "svgd_bodies.cuh"

namespace stamp {
namespace {

__global__ void __launch_bounds__(256) pairwise_kernel(const float* __restrict__ theta, int N,
                                                       int D, float* __restrict__ d2,
                                                       unsigned* __restrict__ hist,
                                                       unsigned* __restrict__ sel,
                                                       unsigned* __restrict__ counter,
                                                       float* __restrict__ h_dev) {
    if (blockIdx.y > blockIdx.x) return;
    pairwise_body(theta, N, D, d2, hist, sel, counter, h_dev, blockIdx.y, blockIdx.x, gridDim.x);
}

// Batched: one CTA per work item (instance, tile row bi, tile column bj >= bi).
__global__ void __launch_bounds__(256) pairwise_batch_kernel(const SvgdInst* __restrict__ inst,
                                                             const int4* __restrict__ items,
                                                             const int* __restrict__ active) {
    const int4 it = items[blockIdx.x];
    const SvgdInst& g = inst[it.x];
    if (!active[g.gid]) return;
    pairwise_body(g.theta, g.N, g.D, g.d2, g.hist, g.sel, g.counter, g.h, it.y, it.z, g.nt);
}


__global__ void __launch_bounds__(256) median_digit_kernel(int N, int dg,
                                                           const float* __restrict__ d2,
                                                           unsigned* __restrict__ hist,
                                                           unsigned* __restrict__ sel,
                                                           unsigned* __restrict__ counter,
                                                           float* __restrict__ h_dev,
                                                           float* __restrict__ h_out) {
    median_digit_body(N, dg, d2, hist, sel, counter, h_dev, h_out, blockIdx.x, gridDim.x);
}

// Batched: work item (instance, CTA index) of the instance's med_ctas CTAs.
__global__ void __launch_bounds__(256) median_digit_batch_kernel(const SvgdInst* __restrict__ inst,
                                                                 const int2* __restrict__ items,
                                                                 const int* __restrict__ active,
                                                                 int dg) {
    const int2 it = items[blockIdx.x];
    const SvgdInst& g = inst[it.x];
    if (!active[g.gid] || g.N < 2) return;
    median_digit_body(g.N, dg, g.d2, g.hist, g.sel, g.counter + dg, g.h, nullptr, it.y, g.med_ctas);
}


template <int DP>
__global__ void __launch_bounds__(kW * 32) phi_kernel(const float* __restrict__ theta,
                                                      const float* __restrict__ grad, int N, int D,
                                                      const float* __restrict__ d2,
                                                      const float* __restrict__ h_dev,
                                                      float* __restrict__ part, int j_chunk,
                                                      int* err, const float* __restrict__ wn,
                                                      unsigned wait_limit, int skip_first, int row0,
                                                      int rows) {
    phi_body<DP>(theta, grad, N, D, d2, h_dev, part, j_chunk, err, blockIdx.x, blockIdx.y, wn,
                 wait_limit, skip_first != 0, row0, rows);
}

// Batched: work item (instance, row block, j-share); DP covers the batch's largest D.
template <int DP>
__global__ void __launch_bounds__(kW * 32) phi_batch_kernel(const SvgdInst* __restrict__ inst,
                                                            const int4* __restrict__ items,
                                                            const int* __restrict__ active,
                                                            int* err) {
    const int4 it = items[blockIdx.x];
    const SvgdInst& g = inst[it.x];
    if (!active[g.gid]) return;
    phi_body<DP>(g.theta, g.grad, g.N, g.D, g.d2, g.h, g.part, g.j_chunk, err, it.y, it.z, nullptr,
                 kWaitLimit, false, 0, g.N);
}

// Adam (Kingma & Ba 2015) with gradient -phi, phi the in-order sum of the
// `shares` partial directions (stride n); optionally stores phi.  Flags
// non-finite inputs/results.
__global__ void adam_kernel(float* __restrict__ theta, const float* __restrict__ part, int shares,
                            float* __restrict__ phi_out, float* __restrict__ m,
                            float* __restrict__ v, int n, float lr, float bc1, float bc2,
                            int* flag) {
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= n) return;
    float phi = part[t];
    for (int q = 1; q < shares; ++q) phi += part[(size_t)q * n + t];
    if (phi_out) phi_out[t] = phi;
    const float g = -phi;
    const float mt = 0.9f * m[t] + 0.1f * g;
    const float vt = 0.999f * v[t] + 0.001f * g * g;
    const float th = theta[t] - lr * (mt / bc1) / (sqrtf(vt / bc2) + 1e-8f);
    m[t] = mt;
    v[t] = vt;
    theta[t] = th;
    if (!isfinite(th) || !isfinite(g)) atomicOr(flag, 1);
}

// Batched Adam over the concatenated particles of all instances: element t
// belongs to the last instance whose first element is <= t; its phi is the
// in-order sum of that instance's shares.  step is read on the device.
__global__ void adam_batch_kernel(float* __restrict__ theta, float* __restrict__ m,
                                  float* __restrict__ v, long long n, const SvgdInst* __restrict__ inst,
                                  int n_inst, const int* __restrict__ active,
                                  const int* __restrict__ step_dev, const float2* __restrict__ bc,
                                  float lr, int* flag) {
    const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= n) return;
    int lo = 0, hi = n_inst - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (__ldg(&inst[mid].elem0) <= t) lo = mid; else hi = mid - 1;
    }
    const SvgdInst& g = inst[lo];
    const long long loc = t - g.elem0, ne = (long long)g.N * g.D;
    if (loc >= ne || !active[g.gid]) return;
    const float* part = g.part;
    float phi = part[loc];
    for (int q = 1; q < g.shares; ++q) phi += part[(size_t)q * ne + loc];
    const float2 b12 = bc[*step_dev + 1];
    const float bc1 = b12.x, bc2 = b12.y;
    const float gr = -phi;
    const float mt = 0.9f * m[t] + 0.1f * gr;
    const float vt = 0.999f * v[t] + 0.001f * gr * gr;
    const float th = theta[t] - lr * (mt / bc1) / (sqrtf(vt / bc2) + 1e-8f);
    m[t] = mt;
    v[t] = vt;
    theta[t] = th;
    if (!isfinite(th) || !isfinite(gr)) atomicOr(flag, 1);
}

// Eq. dsvgd weights, normalised: w_j = exp(C_j - C~_j - max) / sum, C the hard
// and C~ the relaxed cost of particle j; a non-finite difference weighs 0.
// One CTA; fixed per-thread strides and a fixed tree: deterministic.
__global__ void __launch_bounds__(1024) dsvgd_weights_kernel(const float* __restrict__ c_relaxed,
                                                            const float* __restrict__ c_hard, int N,
                                                            float* __restrict__ wn) {
    __shared__ float red[1024];
    float mx = -INFINITY;
    for (int j = threadIdx.x; j < N; j += 1024) {
        const float d = c_hard[j] - c_relaxed[j];
        if (isfinite(d)) mx = fmaxf(mx, d);
    }
    red[threadIdx.x] = mx;
    __syncthreads();
    for (int o = 512; o > 0; o >>= 1) {
        if (threadIdx.x < o) red[threadIdx.x] = fmaxf(red[threadIdx.x], red[threadIdx.x + o]);
        __syncthreads();
    }
    mx = red[0];
    __syncthreads();
    float sum = 0.f;
    for (int j = threadIdx.x; j < N; j += 1024) {
        const float d = c_hard[j] - c_relaxed[j];
        const float e = isfinite(d) ? expf(d - mx) : 0.f;
        wn[j] = e;
        sum += e;
    }
    red[threadIdx.x] = sum;
    __syncthreads();
    for (int o = 512; o > 0; o >>= 1) {
        if (threadIdx.x < o) red[threadIdx.x] += red[threadIdx.x + o];
        __syncthreads();
    }
    const float inv = red[0] > 0.f ? 1.f / red[0] : 0.f;
    for (int j = threadIdx.x; j < N; j += 1024) wn[j] *= inv;
}

__global__ void init_theta_kernel(float* theta, int n, uint64_t key) {
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t < n) theta[t] = 2.f * u23(sm64(key, (uint64_t)t)) - 1.f;
}

// Distinct-plan top-k: sort (cost bits, index) ascending, then keep the first
// k distinct argmax sequences (Gamma, Eq. gamma_map; ties to the lowest index).
__global__ void __launch_bounds__(1024) topk_kernel(const float* __restrict__ theta,
                                                    const float* __restrict__ cost, int N, int H,
                                                    int M, int P, int k, int* out) {
    extern __shared__ unsigned long long sk[];
    int n2 = 1;
    while (n2 < N) n2 <<= 1;
    unsigned long long* key = sk;
    unsigned long long* code = sk + n2;
    for (int t = threadIdx.x; t < n2; t += blockDim.x) {
        if (t < N) {
            unsigned cb = __float_as_uint(cost[t]);
            if (cb & 0x80000000u) cb = 0xFFFFFFFFu;   // costs are >= 0; anything else last
            key[t] = ((unsigned long long)cb << 32) | (unsigned)t;
            unsigned long long cd = 0;
            for (int a = 0; a < H; ++a) {
                const float* lg = theta + (size_t)t * H * P + a * P;
                int best = 0;
                float bv = lg[0];
                for (int c = 1; c < M; ++c)
                    if (lg[c] > bv) { bv = lg[c]; best = c; }
                cd |= (unsigned long long)best << (4 * a);
            }
            code[t] = cd;
        } else {
            key[t] = ~0ull;
        }
    }
    __syncthreads();
    for (int size = 2; size <= n2; size <<= 1)
        for (int stride = size >> 1; stride > 0; stride >>= 1) {
            for (int t = threadIdx.x; t < n2; t += blockDim.x) {
                const int p = t ^ stride;
                if (p > t) {
                    const bool up = (t & size) == 0;
                    const unsigned long long a = key[t], b = key[p];
                    if ((a > b) == up) { key[t] = b; key[p] = a; }
                }
            }
            __syncthreads();
        }
    if (threadIdx.x == 0) {
        int got = 0;
        for (int r = 0; r < N && got < k; ++r) {
            const int idx = (int)(key[r] & 0xFFFFFFFFu);
            const unsigned long long cd = code[idx];
            bool dup = false;
            for (int q = 0; q < got; ++q) dup |= code[out[q]] == cd;
            if (!dup) out[got++] = idx;
        }
        for (int q = got; q < k; ++q) out[q] = -1;
    }
}

template <int DP>
cudaError_t phi_launch(const float* theta, const float* grad, int N, int D, const float* d2,
                       const float* h_dev, float* part, int shares, int j_chunk, int* err,
                       const float* wn, unsigned wait_limit, int skip_first, int row0, int rows,
                       cudaStream_t st) {
    const size_t smem = (size_t)4 * phi_stage_floats(D, DP) * sizeof(float) +
                        (size_t)kW * kTJ * sizeof(float4) + 2 * sizeof(uint64_t);
    if (smem > 48 * 1024) {
        cudaError_t e = cudaFuncSetAttribute(phi_kernel<DP>,
                                             cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
    }
    const int per_cta = kW * kR;
    phi_kernel<DP><<<dim3((rows + per_cta - 1) / per_cta, shares), kW * 32, smem, st>>>(
        theta, grad, N, D, d2, h_dev, part, j_chunk, err, wn, wait_limit, skip_first, row0, rows);
    return cudaGetLastError();
}

}  // namespace

cudaError_t launch_pairwise(const float* theta, int N, int D, const SvgdScratch& s,
                            cudaStream_t st) {
    const int nt = (N + kTile - 1) / kTile;
    const size_t smem = 2 * kTile * (D + 1) * sizeof(float);
    if (smem + kPairwiseStatic > 48 * 1024) {   // static + dynamic above the default limit
        cudaError_t e = cudaFuncSetAttribute(pairwise_kernel,
                                             cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
    }
    pairwise_kernel<<<dim3(nt, nt), 256, smem, st>>>(theta, N, D, s.d2, s.hist, s.sel, s.counter,
                                                     s.h);
    return cudaGetLastError();
}

cudaError_t launch_median_digit(int N, int digit, const SvgdScratch& s, float* h_out,
                                cudaStream_t st) {
    const int cap = 2 * sm_count();
    int grid = N - 1 < cap ? N - 1 : cap;
    if (grid < 1) grid = 1;
    median_digit_kernel<<<grid, 256, 0, st>>>(N, digit, s.d2, s.hist, s.sel, s.counter + digit,
                                              s.h, h_out);
    return cudaGetLastError();
}

cudaError_t launch_phi_rows(const float* theta, const float* grad, int N, int D, int row0,
                            int rows, const SvgdScratch& s, float* part, int max_shares, int* shares,
                            cudaStream_t st, const float* wn) {
    // TMA bulk copies need 16-byte aligned sources
    if ((reinterpret_cast<uintptr_t>(theta) | reinterpret_cast<uintptr_t>(grad)) & 15u)
        return cudaErrorMisalignedAddress;
    // split the sum over j so that about four CTAs per SM are in flight; the
    // shares start on kTJ-row boundaries (16-byte aligned TMA sources)
    const int row_blocks = (N + kW * kR - 1) / (kW * kR);
    int want = (4 * sm_count() + row_blocks - 1) / row_blocks;
    want = want < 1 ? 1 : (want > max_shares ? max_shares : want);
    const int j_chunk = ((N + want - 1) / want + kTJ - 1) / kTJ * kTJ;
    *shares = (N + j_chunk - 1) / j_chunk;
    const unsigned limit = s.wait_limit ? s.wait_limit : kWaitLimit;
    const int dp = (D + 31) / 32;
    switch (dp) {
        case 1: return phi_launch<1>(theta, grad, N, D, s.d2, s.h, part, *shares, j_chunk, s.err, wn, limit, s.skip_first_copy, row0, rows, st);
        case 2: return phi_launch<2>(theta, grad, N, D, s.d2, s.h, part, *shares, j_chunk, s.err, wn, limit, s.skip_first_copy, row0, rows, st);
        case 3: return phi_launch<3>(theta, grad, N, D, s.d2, s.h, part, *shares, j_chunk, s.err, wn, limit, s.skip_first_copy, row0, rows, st);
        case 4: return phi_launch<4>(theta, grad, N, D, s.d2, s.h, part, *shares, j_chunk, s.err, wn, limit, s.skip_first_copy, row0, rows, st);
        case 5: case 6:
            return phi_launch<6>(theta, grad, N, D, s.d2, s.h, part, *shares, j_chunk, s.err, wn, limit, s.skip_first_copy, row0, rows, st);
        case 7: case 8: case 9:
            return phi_launch<9>(theta, grad, N, D, s.d2, s.h, part, *shares, j_chunk, s.err, wn, limit, s.skip_first_copy, row0, rows, st);
    }
    return cudaErrorInvalidValue;
}

cudaError_t launch_phi(const float* theta, const float* grad, int N, int D, const SvgdScratch& s,
                       float* part, int max_shares, int* shares, cudaStream_t st, const float* wn) {
    return launch_phi_rows(theta, grad, N, D, 0, N, s, part, max_shares, shares, st, wn);
}

cudaError_t launch_adam(float* theta, const float* part, int shares, float* phi_out, float* m,
                        float* v, int n, int step, float lr, int* flag, cudaStream_t st) {
    const float bc1 = 1.f - powf(0.9f, (float)step);
    const float bc2 = 1.f - powf(0.999f, (float)step);
    adam_kernel<<<(n + 255) / 256, 256, 0, st>>>(theta, part, shares, phi_out, m, v, n, lr, bc1,
                                                 bc2, flag);
    return cudaGetLastError();
}

cudaError_t launch_pairwise_batch(const SvgdInst* inst, const int4* items, int n_items, int max_D,
                                  const int* active, cudaStream_t st) {
    const size_t smem = 2 * kTile * (max_D + 1) * sizeof(float);
    if (smem + kPairwiseStatic > 48 * 1024) {
        cudaError_t e = cudaFuncSetAttribute(pairwise_batch_kernel,
                                             cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
    }
    pairwise_batch_kernel<<<n_items, 256, smem, st>>>(inst, items, active);
    return cudaGetLastError();
}

cudaError_t launch_median_digit_batch(const SvgdInst* inst, const int2* items, int n_items,
                                      const int* active, int digit, cudaStream_t st) {
    median_digit_batch_kernel<<<n_items, 256, 0, st>>>(inst, items, active, digit);
    return cudaGetLastError();
}

void phi_batch_plan(int N, int* shares, int* j_chunk) {
    const int row_blocks = (N + kW * kR - 1) / (kW * kR);
    int want = (4 * sm_count() + row_blocks - 1) / row_blocks;
    want = want < 1 ? 1 : (want > kMaxShares ? kMaxShares : want);
    *j_chunk = ((N + want - 1) / want + kTJ - 1) / kTJ * kTJ;
    *shares = (N + *j_chunk - 1) / *j_chunk;
}
int phi_rows_per_block() { return kW * kR; }

template <int DP>
cudaError_t phi_batch_launch(const SvgdInst* inst, const int4* items, int n_items, int max_D,
                             const int* active, int* err, cudaStream_t st) {
    const size_t smem = (size_t)4 * phi_stage_floats(max_D, DP) * sizeof(float) +
                        (size_t)kW * kTJ * sizeof(float4) + 2 * sizeof(uint64_t);
    if (smem > 48 * 1024) {
        cudaError_t e = cudaFuncSetAttribute(phi_batch_kernel<DP>,
                                             cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
    }
    phi_batch_kernel<DP><<<n_items, kW * 32, smem, st>>>(inst, items, active, err);
    return cudaGetLastError();
}

cudaError_t launch_phi_batch(const SvgdInst* inst, const int4* items, int n_items, int max_D,
                             const int* active, int* err, cudaStream_t st) {
    switch ((max_D + 31) / 32) {
        case 1: return phi_batch_launch<1>(inst, items, n_items, max_D, active, err, st);
        case 2: return phi_batch_launch<2>(inst, items, n_items, max_D, active, err, st);
        case 3: return phi_batch_launch<3>(inst, items, n_items, max_D, active, err, st);
        case 4: return phi_batch_launch<4>(inst, items, n_items, max_D, active, err, st);
        case 5: case 6: return phi_batch_launch<6>(inst, items, n_items, max_D, active, err, st);
        case 7: case 8: case 9: return phi_batch_launch<9>(inst, items, n_items, max_D, active, err, st);
    }
    return cudaErrorInvalidValue;
}

cudaError_t launch_adam_batch(float* theta, float* m, float* v, long long n, const SvgdInst* inst,
                              int n_inst, const int* active, const int* step_dev, const float2* bc,
                              float lr, int* flag, cudaStream_t st) {
    adam_batch_kernel<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(theta, m, v, n, inst, n_inst, active,
                                                                   step_dev, bc, lr, flag);
    return cudaGetLastError();
}

cudaError_t launch_dsvgd_weights(const float* c_relaxed, const float* c_hard, int N, float* wn,
                                 cudaStream_t st) {
    dsvgd_weights_kernel<<<1, 1024, 0, st>>>(c_relaxed, c_hard, N, wn);
    return cudaGetLastError();
}

cudaError_t launch_init_theta(float* theta, int N, int D, uint64_t seed, cudaStream_t st) {
    const int n = N * D;
    init_theta_kernel<<<(n + 255) / 256, 256, 0, st>>>(theta, n, sm64(seed, kStreamInit));
    return cudaGetLastError();
}

cudaError_t launch_topk(const float* theta, const float* cost, int N, const SimConst& sc, int k,
                        int* topk_out, cudaStream_t st) {
    int n2 = 1;
    while (n2 < N) n2 <<= 1;
    const size_t smem = (size_t)2 * n2 * sizeof(unsigned long long);
    if (smem > 48 * 1024) {
        cudaError_t e = cudaFuncSetAttribute(topk_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             (int)smem);
        if (e != cudaSuccess) return e;
    }
    topk_kernel<<<1, 1024, smem, st>>>(theta, cost, N, sc.H, sc.M, sc.P, k, topk_out);
    return cudaGetLastError();
}

}  // namespace stamp
