// Device bodies of the Stein update shared by the launch-per-piece kernels
// (svgd.cu) and the persistent batched iteration (batch_persist.cu): the
// pairwise distances with the first radix digit of their median, the two
// further median digits, and the Stein direction.  Internal linkage: each
// translation unit that includes this gets its own copy.
#pragma once

#include <cfloat>
#include <cstdint>

#include "async_copy.cuh"
#include "stamp_internal.cuh"

namespace stamp {
namespace {
constexpr int kTile = 32;                      // pairwise tile edge
constexpr int kBins0 = 2048, kBins1 = 2048, kBins2 = 1024;
// static shared memory of the pairwise kernel (digit-0 histogram, mirror
// tile, the bin search's scratch), with margin
constexpr size_t kPairwiseStatic = kBins0 * 4 + kTile * (kTile + 1) * 4 + 256;

__device__ __forceinline__ unsigned digit_of(unsigned bits, int d) {
    return d == 0 ? (bits >> 21) : d == 1 ? ((bits >> 10) & 2047u) : (bits & 1023u);
}

// Bin of `hist` (BINS bins) holding rank `rank`, and the rank inside it.
// NT threads (128 or 256); parallel prefix sum over the per-thread bin groups.
template <int BINS, int NT>
__device__ void find_bin(const unsigned* hist, unsigned rank, unsigned& bin, unsigned& rem) {
    constexpr int PER = BINS / NT, NW = NT / 32;
    __shared__ unsigned wsum[NW];
    __shared__ unsigned res[2];
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    unsigned loc[PER], s = 0;
#pragma unroll
    for (int q = 0; q < PER; ++q) {
        loc[q] = __ldcg(hist + tid * PER + q);
        s += loc[q];
    }
    unsigned x = s;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const unsigned y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
    }
    if (tid == 0) { res[0] = BINS - 1; res[1] = 0; }
    if (lane == 31) wsum[warp] = x;
    __syncthreads();
    if (warp == 0) {
        unsigned w = lane < NW ? wsum[lane] : 0u, v = w;
#pragma unroll
        for (int o = 1; o < NW; o <<= 1) {
            const unsigned y = __shfl_up_sync(0xffffffffu, v, o);
            if (lane >= o) v += y;
        }
        if (lane < NW) wsum[lane] = v - w;     // exclusive prefix of the warps
    }
    __syncthreads();
    const unsigned incl = x + wsum[warp], excl = incl - s;
    if (excl <= rank && rank < incl) {
        unsigned run = excl;
#pragma unroll
        for (int q = 0; q < PER; ++q) {
            if (run + loc[q] > rank) { res[0] = tid * PER + q; res[1] = rank - run; break; }
            run += loc[q];
        }
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

// True in exactly one thread block: the last of `total` to get here.
__device__ bool last_block(unsigned* counter, unsigned total) {
    __shared__ bool last;
    __threadfence();            // this thread's histogram atomics are visible device-wide
    __syncthreads();
    if (threadIdx.x == 0) last = atomicAdd(counter, 1u) == total - 1;
    __syncthreads();
    if (last && threadIdx.x == 0) *counter = 0u;   // ready for the next launch
    return last;
}

// d2 for the upper-triangle tile pairs (bi, bj), bj0 <= bj < bj1 (bi <= bj0),
// mirrored into the lower triangle; histogram of digit 0 over i < j.  The
// last of the instance's `items` CTAs to finish picks digit 0.  NT threads
// (128 or 256): each owns 32*32/NT entries of one tile row.  A strip of
// several tiles reuses the row tile A and flushes the histogram once.
template <int NT = 256>
__device__ __forceinline__ void pairwise_strip_body(const float* __restrict__ theta, int N, int D,
                                                    float* __restrict__ d2,
                                                    unsigned* __restrict__ hist,
                                                    unsigned* __restrict__ sel,
                                                    unsigned* __restrict__ counter,
                                                    float* __restrict__ h_dev, int bi, int bj0,
                                                    int bj1, unsigned items) {
    extern __shared__ float sm[];
    const int ld = D + 1;                        // padded rows: conflict-free column walks
    float* A = sm;
    float* B = sm + kTile * ld;
    __shared__ unsigned h0[kBins0];
    __shared__ float tile[kTile][kTile + 1];
    const int i0 = bi * kTile;
    for (int t = threadIdx.x; t < kBins0; t += blockDim.x) h0[t] = 0u;
    for (int t = threadIdx.x; t < kTile * D; t += blockDim.x) {
        const int r = t / D, d = t % D;
        A[r * ld + d] = (i0 + r < N) ? theta[(size_t)(i0 + r) * D + d] : 0.f;
    }
    constexpr int TPR = NT / kTile, CPT = kTile / TPR;   // threads per row, columns per thread
    const int r = threadIdx.x / TPR, c0 = threadIdx.x % TPR;
    for (int bj = bj0; bj < bj1; ++bj) {
        const int j0 = bj * kTile;
        // the previous tile's compute is done (barrier before its mirror)
        for (int t = threadIdx.x; t < kTile * D; t += blockDim.x) {
            const int rr = t / D, d = t % D;
            B[rr * ld + d] = (j0 + rr < N) ? theta[(size_t)(j0 + rr) * D + d] : 0.f;
        }
        __syncthreads();
        float acc[CPT];
#pragma unroll
        for (int q = 0; q < CPT; ++q) acc[q] = 0.f;
        for (int d = 0; d < D; ++d) {
            const float a = A[r * ld + d];
#pragma unroll
            for (int q = 0; q < CPT; ++q) {
                const float e = a - B[(c0 + TPR * q) * ld + d];
                acc[q] = fmaf(e, e, acc[q]);
            }
        }
        const int i = i0 + r;
#pragma unroll
        for (int q = 0; q < CPT; ++q) {
            const int c = c0 + TPR * q, j = j0 + c;
            tile[r][c] = acc[q];
            if (i < N && j < N) {
                d2[(size_t)i * N + j] = acc[q];
                if (i < j) atomicAdd(&h0[digit_of(__float_as_uint(acc[q]), 0)], 1u);
            }
        }
        __syncthreads();
        if (bi != bj)   // mirror: coalesced rows of the lower triangle
            for (int t = threadIdx.x; t < kTile * kTile; t += blockDim.x) {
                const int rr = t / kTile, cc = t % kTile;   // rr indexes j, cc indexes i
                if (j0 + rr < N && i0 + cc < N) d2[(size_t)(j0 + rr) * N + i0 + cc] = tile[cc][rr];
            }
        __syncthreads();   // tile and B are free for the next pair
    }
    for (int t = threadIdx.x; t < kBins0; t += blockDim.x)
        if (h0[t]) atomicAdd(&hist[t], h0[t]);
    if (last_block(counter, items)) {
        if (N < 2) {
            if (threadIdx.x == 0) *h_dev = 1.f;
            return;
        }
        unsigned b0, r0;
        find_bin<kBins0, NT>(hist, median_rank(N), b0, r0);
        if (threadIdx.x == 0) { sel[0] = b0; sel[1] = r0; }
    }
}

// One tile pair per CTA: the nt(nt+1)/2 CTAs of an instance.
template <int NT = 256>
__device__ __forceinline__ void pairwise_body(const float* __restrict__ theta, int N, int D,
                                              float* __restrict__ d2, unsigned* __restrict__ hist,
                                              unsigned* __restrict__ sel,
                                              unsigned* __restrict__ counter,
                                              float* __restrict__ h_dev, int bi, int bj, int nt) {
    pairwise_strip_body<NT>(theta, N, D, d2, hist, sel, counter, h_dev, bi, bj, bj + 1,
                            (unsigned)(nt * (nt + 1) / 2));
}

// Histogram of digit `dg` (1 or 2) over the i<j entries whose higher digits
// match the prefix chosen so far; rows of the upper triangle, grid-strided.
// NT threads (128 or 256).
template <int NT = 256>
__device__ __forceinline__ void median_digit_body(int N, int dg, const float* __restrict__ d2,
                                                  unsigned* __restrict__ hist,
                                                  unsigned* __restrict__ sel,
                                                  unsigned* __restrict__ counter,
                                                  float* __restrict__ h_dev,
                                                  float* __restrict__ h_out, int cta, int ctas) {
    __shared__ unsigned hloc[kBins1];
    const unsigned b0 = __ldcg(sel), b1 = dg == 2 ? __ldcg(sel + 2) : 0u;
    const unsigned prefix = dg == 1 ? b0 : ((b0 << 11) | b1);
    const int shift = dg == 1 ? 21 : 10;
    const int nb = dg == 1 ? kBins1 : kBins2;
    for (int t = threadIdx.x; t < nb; t += blockDim.x) hloc[t] = 0u;
    __syncthreads();
    // two of the CTA's rows at a time, four entries of each per thread: the
    // eight loads are in flight together (the row i2 > i is the shorter)
    constexpr int U = 4;
    for (int i = cta; i < N - 1; i += 2 * ctas) {
        const int i2 = i + ctas;
        const float* row = d2 + (size_t)i * N;
        const float* row2 = d2 + (size_t)(i2 < N - 1 ? i2 : i) * N;
        for (int j0 = threadIdx.x; i + 1 + j0 < N; j0 += U * NT) {
            unsigned bits[2 * U];
            bool ok[2 * U];
#pragma unroll
            for (int u = 0; u < U; ++u) {
                const int j = i + 1 + j0 + u * NT, k = i2 + 1 + j0 + u * NT;
                ok[u] = j < N;
                ok[U + u] = i2 < N - 1 && k < N;
                bits[u] = ok[u] ? __float_as_uint(row[j]) : 0u;
                bits[U + u] = ok[U + u] ? __float_as_uint(row2[k]) : 0u;
            }
#pragma unroll
            for (int u = 0; u < 2 * U; ++u)
                if (ok[u] && (bits[u] >> shift) == prefix) atomicAdd(&hloc[digit_of(bits[u], dg)], 1u);
        }
    }
    __syncthreads();
    unsigned* out = hist + (dg == 1 ? kBins0 : kBins0 + kBins1);
    for (int t = threadIdx.x; t < nb; t += blockDim.x)
        if (hloc[t]) atomicAdd(&out[t], hloc[t]);
    if (last_block(counter, (unsigned)ctas)) {
        if (dg == 1) {
            unsigned b1n, r1;
            find_bin<kBins1, NT>(out, __ldcg(sel + 1), b1n, r1);
            if (threadIdx.x == 0) { sel[2] = b1n; sel[3] = r1; }
        } else {
            unsigned b2, r2;
            find_bin<kBins2, NT>(out, __ldcg(sel + 3), b2, r2);
            if (threadIdx.x == 0) {
                const float med = __uint_as_float((b0 << 21) | (b1 << 10) | b2);
                float h = med / logf((float)N + 1.f);
                h = (h >= 1e-12f) ? h : 1.f;
                *h_dev = h;
                if (h_out) *h_out = h;
            }
        }
    }
}

// TMA bulk copies and mbarriers: the shared helpers of async_copy.cuh, whose
// kWaitLimit bounds every wait (then the error flag).
using async::fence_async_shared;
using async::kWaitLimit;
using async::mbar_expect_tx;
using async::mbar_init;
using async::mbar_inval;
using async::mbar_try_wait;
using async::tma_load_1d;

// phi_i = (1/N) sum_j [k_ij g_j + (2/h) k_ij (theta_i - theta_j)], k_ij = exp(-d2_ij/h).
// A warp owns kR rows; lane l owns columns l, l+32, ...  (DP slots).  The j
// range is walked in tiles of kTJ rows of theta and grad, which are
// contiguous in HBM: one thread streams each tile into one of two shared
// memory stages with 1-D TMA bulk copies (mbarrier completion), one tile
// ahead of the compute.  The d2 values of the next tile are prefetched into
// registers; k_ij for the warp's rows is one float4 per j (a broadcast load).
constexpr int kR = 4, kW = 8, kTJ = 32;   // rows per warp, warps per CTA, j rows per tile
__host__ __device__ constexpr int phi_stage_floats(int D, int DP) {
    return ((kTJ * D + 32 * DP) + 3) / 4 * 4;   // per array, 16-byte multiple
}
// KW warps per CTA (kW in the per-piece kernels), the j loop unrolled
// UNROLL times; false if a copy never
// landed (error bit 2 set).  A CTA that goes on to other work may reuse the
// shared memory: the mbarriers are invalidated on the way out.
template <int DP, int KW = kW, int UNROLL = 4>
__device__ __forceinline__ bool phi_body(const float* __restrict__ theta,
                                         const float* __restrict__ grad, int N, int D,
                                         const float* __restrict__ d2,
                                         const float* __restrict__ h_dev, float* __restrict__ part,
                                         int j_chunk, int* err, int rblock, int share,
                                         const float* __restrict__ wn, unsigned wait_limit,
                                         bool skip_first, int row0, int rows) {
    extern __shared__ __align__(128) float sm[];
    const int sf = phi_stage_floats(D, DP);
    // stage s: theta tile at sm + 2*s*sf, grad tile right after it
    float4* Ks = reinterpret_cast<float4*>(sm + 4 * sf);             // KW x kTJ
    uint64_t* bar = reinterpret_cast<uint64_t*>(Ks + KW * kTJ);       // 2 stages
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    // rows [row0, row0 + rows) of phi (all N: row0 = 0, rows = N)
    const int ib = row0 + (rblock * KW + warp) * kR, re = row0 + rows;
    // this CTA's share of the sum over j: rows [jb, je) of theta and grad
    const int jb = share * j_chunk, je = min(N, jb + j_chunk);
    const int ntiles = (je - jb + kTJ - 1) / kTJ;
    const float inv_h = 1.f / __ldcg(h_dev);

    if (tid == 0) {
        mbar_init(&bar[0], 1);
        mbar_init(&bar[1], 1);
        fence_async_shared();
    }
    __syncthreads();
    // thread 0 streams tile t into stage t&1: the 16-byte-aligned bulk of the
    // contiguous rows by TMA, a ragged tail (< 16 bytes) by plain copies
    auto issue = [&](int t) {
        const int s = t & 1, j0 = jb + t * kTJ, n = min(kTJ, je - j0) * D;
        const unsigned bulk = (unsigned)(n * 4) & ~15u;
        mbar_expect_tx(&bar[s], 2 * bulk);
        float* Ts = sm + 2 * s * sf;
        float* Gs = Ts + sf;
        if (bulk && !(skip_first && t == 0)) {
            tma_load_1d(Ts, theta + (size_t)j0 * D, bulk, &bar[s]);
            tma_load_1d(Gs, grad + (size_t)j0 * D, bulk, &bar[s]);
        }
        for (int f = bulk / 4; f < n; ++f) {
            Ts[f] = theta[(size_t)j0 * D + f];
            Gs[f] = grad[(size_t)j0 * D + f];
        }
    };
    if (tid == 0) {
        issue(0);
        if (ntiles > 1) issue(1);
    }
    float ti[kR][DP], ag[kR][DP], ar[kR][DP], dv[kR];
#pragma unroll
    for (int r = 0; r < kR; ++r) {
#pragma unroll
        for (int q = 0; q < DP; ++q) {
            const int d = lane + 32 * q;
            ti[r][q] = (ib + r < re && d < D) ? theta[(size_t)(ib + r) * D + d] : 0.f;
            ag[r][q] = ar[r][q] = 0.f;
        }
        dv[r] = (ib + r < re && jb + lane < je) ? d2[(size_t)(ib + r) * N + jb + lane] : 0.f;
    }
    unsigned phases = 0u;                       // bit s: parity of stage s
    for (int t = 0; t < ntiles; ++t) {
        const int s = t & 1, j0 = jb + t * kTJ, nj = min(kTJ, je - j0);
        {
            float kv[kR];
#pragma unroll
            for (int r = 0; r < kR; ++r) kv[r] = (ib + r < re && lane < nj) ? expf(-dv[r] * inv_h) : 0.f;
            if (wn) {   // Eq. dsvgd: k_ij scaled by w_j / w
                const float wj = lane < nj ? wn[j0 + lane] : 0.f;
#pragma unroll
                for (int r = 0; r < kR; ++r) kv[r] *= wj;
            }
            Ks[warp * kTJ + lane] = make_float4(kv[0], kv[1], kv[2], kv[3]);
        }
        if (t + 1 < ntiles) {   // next tile's distances, consumed one iteration later
            const int jn = j0 + kTJ + lane;
#pragma unroll
            for (int r = 0; r < kR; ++r) dv[r] = (ib + r < re && jn < je) ? d2[(size_t)(ib + r) * N + jn] : 0.f;
        }
        const unsigned par = (phases >> s) & 1u;
        unsigned spins = 0;
        while (!mbar_try_wait(&bar[s], par) && ++spins < wait_limit) {
        }
        if (__syncthreads_or(spins >= wait_limit)) {   // a copy never landed: report, stop
            if (tid == 0) {
                atomicOr(err, 2);
                // a last bounded wait for the copies still in flight (this
                // stage and, if issued, the next) before the CTA exits
                for (unsigned w = 0; w < wait_limit && !mbar_try_wait(&bar[s], par); ++w) {
                }
                const unsigned pn = (phases >> (s ^ 1)) & 1u;
                if (t + 1 < ntiles)
                    for (unsigned w = 0; w < wait_limit && !mbar_try_wait(&bar[s ^ 1], pn); ++w) {
                    }
            }
            return false;
        }
        phases ^= 1u << s;
        const float* Tj = sm + 2 * s * sf;
        const float* Gj = Tj + sf;
#pragma unroll (UNROLL)
        for (int jj = 0; jj < nj; ++jj) {   // several j's shared-memory loads in flight
            const float4 k4 = Ks[warp * kTJ + jj];
            const float kk[kR] = {k4.x, k4.y, k4.z, k4.w};
#pragma unroll
            for (int q = 0; q < DP; ++q) {
                const float g = Gj[jj * D + lane + 32 * q];
                const float tv = Tj[jj * D + lane + 32 * q];
#pragma unroll
                for (int r = 0; r < kR; ++r) {
                    ag[r][q] = fmaf(kk[r], g, ag[r][q]);
                    ar[r][q] = fmaf(kk[r], ti[r][q] - tv, ar[r][q]);
                }
            }
        }
        __syncthreads();                       // stage s and Ks fully read
        if (tid == 0 && t + 2 < ntiles) {
            fence_async_shared();
            issue(t + 2);
        }
    }
    // partial phi of this j-share; the Adam kernel sums the shares in order
    const float inv_n = wn ? 1.f : 1.f / (float)N, two_h = 2.f * inv_h;
    float* out = part + (size_t)share * rows * D;
#pragma unroll
    for (int r = 0; r < kR; ++r)
#pragma unroll
        for (int q = 0; q < DP; ++q) {
            const int d = lane + 32 * q;
            if (ib + r < re && d < D)
                out[(size_t)(ib - row0 + r) * D + d] = (ag[r][q] + two_h * ar[r][q]) * inv_n;
        }
    if (tid == 0) {   // every wait has completed and the loop's last barrier passed
        mbar_inval(&bar[0]);
        mbar_inval(&bar[1]);
    }
    return true;
}

}  // namespace
}  // namespace stamp
