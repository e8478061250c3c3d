// Stein update of Algorithm 1 (Eq. svgd with unit weights), its median
// bandwidth, Adam, the initial particles and the final distinct-plan top-k.
//
// Bandwidth: h = med/ln(N+1), med the lower median (rank floor((M-1)/2)) of
// the M = N(N-1)/2 squared distances d2_ij, i<j -- the median heuristic the
// paper uses for its RBF kernels (App. C.3).  It is selected exactly with a
// three-digit radix select on the float bits (11 + 11 + 10 bits; the bits of
// non-negative floats order like the floats), over a d2 matrix kept in HBM
// (16 MB at N = 2048, L2-resident).  Every digit is picked by each CTA of the
// next kernel from the previous histogram, so no kernel waits on another CTA.
#include <cfloat>
#include <cstdint>

#include "stamp_internal.cuh"

namespace stamp {
namespace {

constexpr int kTile = 32;     // pairwise tile edge
constexpr int kBins0 = 2048, kBins1 = 2048, kBins2 = 1024;

__device__ __forceinline__ unsigned digit_of(unsigned bits, int d) {
    return d == 0 ? (bits >> 21) : d == 1 ? ((bits >> 10) & 2047u) : (bits & 1023u);
}

// d2 for one kTile x kTile tile of (i, j); histogram of digit 0 over i < j.
__global__ void __launch_bounds__(256) pairwise_kernel(const float* __restrict__ theta, int N,
                                                       int D, float* __restrict__ d2,
                                                       unsigned* __restrict__ hist) {
    extern __shared__ float sm[];
    const int ld = D + 1;                        // padded row: conflict-free column walks
    float* A = sm;
    float* B = sm + kTile * ld;
    __shared__ unsigned h0[kBins0];
    const int bi = blockIdx.y, bj = blockIdx.x;
    const int i0 = bi * kTile, j0 = bj * kTile;
    for (int t = threadIdx.x; t < kBins0; t += blockDim.x) h0[t] = 0u;
    for (int t = threadIdx.x; t < kTile * D; t += blockDim.x) {
        const int r = t / D, d = t % D;
        A[r * ld + d] = (i0 + r < N) ? theta[(size_t)(i0 + r) * D + d] : 0.f;
        B[r * ld + d] = (j0 + r < N) ? theta[(size_t)(j0 + r) * D + d] : 0.f;
    }
    __syncthreads();
    const int r = threadIdx.x / 8, c0 = threadIdx.x % 8;
    float acc[4] = {0.f, 0.f, 0.f, 0.f};
    for (int d = 0; d < D; ++d) {
        const float a = A[r * ld + d];
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            const float e = a - B[(c0 + 8 * q) * ld + d];
            acc[q] = fmaf(e, e, acc[q]);
        }
    }
    const int i = i0 + r;
#pragma unroll
    for (int q = 0; q < 4; ++q) {
        const int j = j0 + c0 + 8 * q;
        if (i < N && j < N) {
            d2[(size_t)i * N + j] = acc[q];
            if (i < j) atomicAdd(&h0[digit_of(__float_as_uint(acc[q]), 0)], 1u);
        }
    }
    __syncthreads();
    for (int t = threadIdx.x; t < kBins0; t += blockDim.x)
        if (h0[t]) atomicAdd(&hist[t], h0[t]);
}

// Find the bin of `hist` (nbins) holding rank `rank`; returns the bin and the
// rank inside it.  256 threads.
__device__ void find_bin(const unsigned* hist, int nbins, unsigned rank, unsigned& bin,
                         unsigned& rem) {
    __shared__ unsigned part[256];
    __shared__ unsigned res[2];
    const int per = nbins / 256;
    unsigned s = 0;
    for (int q = 0; q < per; ++q) s += hist[threadIdx.x * per + q];
    part[threadIdx.x] = s;
    __syncthreads();
    if (threadIdx.x == 0) {
        unsigned run = 0;
        int t = 0;
        while (t < 255 && run + part[t] <= rank) run += part[t++];
        int b = t * per;
        for (int q = 0; q < per; ++q, ++b) {
            const unsigned hb = hist[b];
            if (run + hb > rank || q == per - 1) break;
            run += hb;
        }
        res[0] = (unsigned)b;
        res[1] = rank - run;
    }
    __syncthreads();
    bin = res[0];
    rem = res[1];
    __syncthreads();
}

__device__ __forceinline__ unsigned median_rank(int N) {
    const unsigned long long m = (unsigned long long)N * (N - 1) / 2;
    return (unsigned)((m - 1) / 2);
}

// Histogram of digit `dg` (1 or 2) over the i<j entries whose higher digits
// match the prefix selected so far.
__global__ void __launch_bounds__(256) median_digit_kernel(int N, int dg, const float* __restrict__ d2,
                                                           unsigned* __restrict__ hist) {
    __shared__ unsigned hloc[kBins1];
    unsigned b0, r0, b1 = 0, r1;
    find_bin(hist, kBins0, median_rank(N), b0, r0);
    if (dg == 2) find_bin(hist + kBins0, kBins1, r0, b1, r1);
    const int nb = dg == 1 ? kBins1 : kBins2;
    for (int t = threadIdx.x; t < nb; t += blockDim.x) hloc[t] = 0u;
    __syncthreads();
    const size_t total = (size_t)N * N;
    for (size_t e = (size_t)blockIdx.x * blockDim.x + threadIdx.x; e < total;
         e += (size_t)gridDim.x * blockDim.x) {
        const int i = (int)(e / N), j = (int)(e % N);
        if (j <= i) continue;
        const unsigned bits = __float_as_uint(d2[e]);
        const bool match = dg == 1 ? (bits >> 21) == b0 : (bits >> 10) == ((b0 << 11) | b1);
        if (match) atomicAdd(&hloc[digit_of(bits, dg)], 1u);
    }
    __syncthreads();
    unsigned* out = hist + (dg == 1 ? kBins0 : kBins0 + kBins1);
    for (int t = threadIdx.x; t < nb; t += blockDim.x)
        if (hloc[t]) atomicAdd(&out[t], hloc[t]);
}

// h from the three digit histograms (each CTA recomputes it).
__device__ float bandwidth(int N, const unsigned* hist) {
    if (N < 2) return 1.f;
    unsigned b0, r0, b1, r1, b2, r2;
    find_bin(hist, kBins0, median_rank(N), b0, r0);
    find_bin(hist + kBins0, kBins1, r0, b1, r1);
    find_bin(hist + kBins0 + kBins1, kBins2, r1, b2, r2);
    const float med = __uint_as_float((b0 << 21) | (b1 << 10) | b2);
    const float h = med / logf((float)N + 1.f);
    return (h >= 1e-12f) ? h : 1.f;
}

// phi_i = (1/N) sum_j [k_ij g_j + (2/h) k_ij (theta_i - theta_j)], k_ij = exp(-d2_ij/h).
constexpr int kRows = 8, kCols = 64;
__global__ void __launch_bounds__(256) phi_kernel(const float* __restrict__ theta,
                                                  const float* __restrict__ grad, int N, int D,
                                                  const float* __restrict__ d2,
                                                  const unsigned* __restrict__ hist,
                                                  float* __restrict__ phi, float* h_dev,
                                                  float* h_out) {
    extern __shared__ float sm[];
    float* Tj = sm;                       // kCols x D
    float* Gj = Tj + kCols * D;           // kCols x D
    float* Kij = Gj + kCols * D;          // kRows x kCols
    float* Ti = Kij + kRows * kCols;      // kRows x D
    const float h = bandwidth(N, hist);
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        if (h_dev) *h_dev = h;
        if (h_out) *h_out = h;
    }
    const float inv_h = 1.f / h;
    const int i0 = blockIdx.x * kRows;
    const int nout = kRows * D;
    for (int t = threadIdx.x; t < nout; t += blockDim.x) {
        const int r = t / D, d = t % D;
        Ti[t] = (i0 + r < N) ? theta[(size_t)(i0 + r) * D + d] : 0.f;
    }
    constexpr int kMaxOut = 9;            // outputs per thread: kRows*D <= 9*256 (D <= 288)
    float acc_a[kMaxOut], acc_r[kMaxOut];
#pragma unroll
    for (int q = 0; q < kMaxOut; ++q) acc_a[q] = acc_r[q] = 0.f;
    for (int j0 = 0; j0 < N; j0 += kCols) {
        __syncthreads();
        const int nj = min(kCols, N - j0);
        for (int t = threadIdx.x; t < nj * D; t += blockDim.x) {
            Tj[t] = theta[(size_t)j0 * D + t];
            Gj[t] = grad[(size_t)j0 * D + t];
        }
        for (int t = threadIdx.x; t < kRows * kCols; t += blockDim.x) {
            const int r = t / kCols, c = t % kCols;
            const int i = i0 + r, j = j0 + c;
            Kij[t] = (i < N && c < nj) ? expf(-d2[(size_t)i * N + j] * inv_h) : 0.f;
        }
        __syncthreads();
#pragma unroll
        for (int q = 0; q < kMaxOut; ++q) {
            const int o = threadIdx.x + q * 256;
            if (o >= nout) break;
            const int r = o / D, d = o % D;
            const float ti = Ti[o];
            float sa = acc_a[q], sr = acc_r[q];
            for (int c = 0; c < nj; ++c) {
                const float kk = Kij[r * kCols + c];
                sa = fmaf(kk, Gj[c * D + d], sa);
                sr = fmaf(kk, ti - Tj[c * D + d], sr);
            }
            acc_a[q] = sa;
            acc_r[q] = sr;
        }
    }
    const float inv_n = 1.f / (float)N;
#pragma unroll
    for (int q = 0; q < kMaxOut; ++q) {
        const int o = threadIdx.x + q * 256;
        if (o >= nout) break;
        const int r = o / D, d = o % D;
        if (i0 + r < N)
            phi[(size_t)(i0 + r) * D + d] = (acc_a[q] + 2.f * inv_h * acc_r[q]) * inv_n;
    }
}

// Adam (Kingma & Ba 2015) with gradient -phi; flags non-finite inputs/results.
__global__ void adam_kernel(float* __restrict__ theta, const float* __restrict__ phi,
                            float* __restrict__ m, float* __restrict__ v, int n, float lr,
                            float bc1, float bc2, int* flag) {
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= n) return;
    const float g = -phi[t];
    const float mt = 0.9f * m[t] + 0.1f * g;
    const float vt = 0.999f * v[t] + 0.001f * g * g;
    const float th = theta[t] - lr * (mt / bc1) / (sqrtf(vt / bc2) + 1e-8f);
    m[t] = mt;
    v[t] = vt;
    theta[t] = th;
    if (!isfinite(th) || !isfinite(g)) atomicOr(flag, 1);
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

}  // namespace

cudaError_t launch_pairwise(const float* theta, int N, int D, const SvgdScratch& s,
                            cudaStream_t st) {
    const int nt = (N + kTile - 1) / kTile;
    const size_t smem = 2 * kTile * (D + 1) * sizeof(float);
    if (smem > 48 * 1024) {
        cudaError_t e = cudaFuncSetAttribute(pairwise_kernel,
                                             cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
    }
    pairwise_kernel<<<dim3(nt, nt), 256, smem, st>>>(theta, N, D, s.d2, s.hist);
    return cudaGetLastError();
}

cudaError_t launch_median_digit(int N, int digit, const SvgdScratch& s, cudaStream_t st) {
    const long long total = (long long)N * N;
    int grid = (int)((total + 255) / 256);
    if (grid > 152 * 8) grid = 152 * 8;
    median_digit_kernel<<<grid, 256, 0, st>>>(N, digit, s.d2, s.hist);
    return cudaGetLastError();
}

cudaError_t launch_phi(const float* theta, const float* grad, int N, int D, const SvgdScratch& s,
                       float* phi, float* h_out, cudaStream_t st) {
    const size_t smem = (size_t)(2 * kCols * D + kRows * kCols + kRows * D) * sizeof(float);
    if (smem > 48 * 1024) {
        cudaError_t e = cudaFuncSetAttribute(phi_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             (int)smem);
        if (e != cudaSuccess) return e;
    }
    phi_kernel<<<(N + kRows - 1) / kRows, 256, smem, st>>>(theta, grad, N, D, s.d2, s.hist, phi,
                                                           s.h, h_out);
    return cudaGetLastError();
}

cudaError_t launch_adam(float* theta, const float* phi, float* m, float* v, int n, int step,
                        float lr, int* flag, cudaStream_t st) {
    const float bc1 = 1.f - powf(0.9f, (float)step);
    const float bc2 = 1.f - powf(0.999f, (float)step);
    adam_kernel<<<(n + 255) / 256, 256, 0, st>>>(theta, phi, m, v, n, lr, bc1, bc2, flag);
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
