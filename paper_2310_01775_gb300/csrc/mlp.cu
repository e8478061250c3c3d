// BF16 tensor-core MLP for the pose-dynamics surrogate (tcgen05 + TMEM + TMA).
//
// Network: in (<= 32, zero-padded to 32) -> 256 -> 256 -> 256 -> out (<= 16,
// padded to 16), SiLU between layers, linear head; BF16 weights and
// activations, FP32 accumulation in tensor memory.
//
// Operand layout (tcgen05 K-major, no swizzle): a tile of R rows x K columns
// of BF16 is stored as 8x8 "core matrices" of 128 contiguous bytes (8 rows of
// 16 bytes); core matrix (i, j) -- rows 8i..8i+7, columns 8j..8j+7 -- sits at
// byte i*SBO + j*128 with SBO = (K/8)*128.  The matrix descriptor of a 16-wide
// K slice then has leading-dimension offset 128 B (next core matrix along K)
// and stride-dimension offset SBO (next 8-row group).  Weights are packed once
// into this layout in HBM and streamed per layer with 1-D TMA bulk copies;
// each layer's epilogue writes the next layer's A operand straight into it.
#include <cstdint>
#include <cstring>
#include <vector>

#include "async_copy.cuh"
#include "mlp.cuh"
#include "stamp.h"
#include "stamp_internal.cuh"

namespace stamp {
namespace mlp {
namespace {

using async::fence_async_shared;
using async::kWaitLimit;
using async::mbar_expect_tx;
using async::mbar_init;
using async::mbar_try_wait;
using async::smem_u32;
using async::tma_load_1d;

// ---------------- tcgen05 ---------------------------------------------------
__device__ __forceinline__ void tmem_alloc(unsigned* slot, unsigned ncols) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;"
                 ::"r"(smem_u32(slot)), "r"(ncols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
}
__device__ __forceinline__ void tmem_dealloc(unsigned taddr, unsigned ncols) {
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(ncols)
                 : "memory");
}
__device__ __forceinline__ void tc_fence_before() {
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
}
__device__ __forceinline__ void tc_fence_after() {
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
}
// Shared-memory matrix descriptor: start address, LBO, SBO (all >> 4), the
// descriptor version bits (0b01 at bit 46), no swizzle.
__device__ __forceinline__ uint64_t smem_desc(const void* p, unsigned lbo, unsigned sbo) {
    const uint64_t a = (smem_u32(p) & 0x3FFFFu) >> 4;
    return a | ((uint64_t)((lbo >> 4) & 0x3FFFu) << 16) | ((uint64_t)((sbo >> 4) & 0x3FFFu) << 32) |
           (1ull << 46);
}
// Instruction descriptor, kind::f16: D = F32 (bits 4-5 = 1), A = B = BF16
// (bits 7-9 and 10-12 = 1), both K-major, N >> 3 at bit 17, M >> 4 at bit 24.
__host__ __device__ constexpr uint32_t idesc_bf16(int M, int N) {
    return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(N >> 3) << 17) |
           ((uint32_t)(M >> 4) << 24);
}
__device__ __forceinline__ void mma_bf16(unsigned tmem_d, uint64_t adesc, uint64_t bdesc,
                                        uint32_t idesc, unsigned accumulate) {
    asm volatile(
        "{\n .reg .pred p;\n setp.ne.u32 p, %4, 0;\n"
        " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}" ::"r"(tmem_d),
        "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accumulate)
        : "memory");
}
__device__ __forceinline__ void mma_commit(uint64_t* bar) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];"
                 ::"r"(smem_u32(bar))
                 : "memory");
}
// 32 consecutive FP32 columns of this warp's 32 TMEM lanes (one lane per thread).
__device__ __forceinline__ void tmem_ld32(unsigned taddr, float (&v)[32]) {
    unsigned r[32];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,"
        "%14,%15,%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
          "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]),
          "=r"(r[14]), "=r"(r[15]), "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]),
          "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]), "=r"(r[24]), "=r"(r[25]),
          "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
        : "r"(taddr)
        : "memory");
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
    for (int i = 0; i < 32; ++i) v[i] = __uint_as_float(r[i]);
}
__device__ __forceinline__ void tmem_ld16(unsigned taddr, float (&v)[16]) {
    unsigned r[16];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,"
        "%14,%15}, [%16];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
          "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]),
          "=r"(r[14]), "=r"(r[15])
        : "r"(taddr)
        : "memory");
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
    for (int i = 0; i < 16; ++i) v[i] = __uint_as_float(r[i]);
}

__device__ __forceinline__ unsigned pack_bf16(float a, float b) {
    const __nv_bfloat162 h = __floats2bfloat162_rn(a, b);
    return *reinterpret_cast<const unsigned*>(&h);
}
// z sigmoid(z) with the fast reciprocal (its error, a few float ulps, is far
// below the bfloat16 rounding of the result)
__device__ __forceinline__ float silu(float z) { return __fdividef(z, 1.f + __expf(-z)); }

// Byte offset of element (row, col) in a K-major core-matrix tile of K columns.
__host__ __device__ __forceinline__ unsigned tile_off(int row, int col, int K) {
    return (unsigned)((row >> 3) * (K / 8) * 128 + (col >> 3) * 128 + (row & 7) * 16 + (col & 7) * 2);
}

constexpr int kRows = 128;                        // rows per tile (MMA M)
// 16 warps: warp w reads TMEM lane quarter w % 4 (rows 32 (w % 4) ...) and
// takes part w / 4 of the four column parts in the epilogues
constexpr int kThreads = 512;
constexpr int kParts = kThreads / 128;
constexpr unsigned kTmemCols = 256;
constexpr unsigned kActBytes = kRows * kHidden * 2;            // 64 KB
constexpr unsigned kWBytes = kHidden * kHidden * 2;            // 128 KB
constexpr unsigned kInBytes = kRows * kIn * 2;                 // 8 KB per input tile

struct FwdSmem {
    alignas(128) unsigned char act[kActBytes];
    alignas(128) unsigned char w[kWBytes];
    uint64_t tma_bar, mma_bar;
    unsigned tmem_slot;
};

// Layer l: K (inputs), N (outputs), packed forward weight bytes.
__host__ __device__ constexpr int layer_k(int l) { return l == 0 ? kIn : kHidden; }
__host__ __device__ constexpr int layer_n(int l) { return l == 3 ? kOut : kHidden; }

// Forward of all four layers for 128-row tiles; y: rows x kOut FP32.
// Optionally stores, for the backward pass, the input activations a_1..a_3 and
// the pre-activations z_0..z_2 (BF16 tiles): slot (l, tile_base + tile) of
// buffers holding tile_cap tiles per layer.
__global__ void __launch_bounds__(kThreads, 1)
mlp_fwd_kernel(const unsigned char* __restrict__ x_tiled, int n_tiles,
               const unsigned char* __restrict__ w_tiled, const float* __restrict__ bias,
               float* __restrict__ y, int rows, unsigned char* __restrict__ saved,
               unsigned char* __restrict__ zsave, int tile_base, int tile_cap,
               int* __restrict__ err) {
    extern __shared__ __align__(1024) unsigned char smem_raw[];
    FwdSmem& sm = *reinterpret_cast<FwdSmem*>(smem_raw);
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    if (tid == 0) {
        mbar_init(&sm.tma_bar, 1);
        mbar_init(&sm.mma_bar, 1);
        fence_async_shared();
    }
    if (warp == 0) tmem_alloc(&sm.tmem_slot, kTmemCols);
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const unsigned tmem = sm.tmem_slot;
    unsigned tma_phase = 0, mma_phase = 0;
    bool failed = false, tma_pending = false, mma_pending = false;
    // weights of layer l (and, for l = 0, the tile's input) into shared memory
    auto issue_load = [&](int l, int tile) {
        const unsigned wbytes = (unsigned)(layer_n(l) * layer_k(l) * 2);
        mbar_expect_tx(&sm.tma_bar, wbytes + (l == 0 ? kInBytes : 0u));
        tma_load_1d(sm.w, w_tiled + layer_w_offset(l), wbytes, &sm.tma_bar);
        if (l == 0) tma_load_1d(sm.act, x_tiled + (size_t)tile * kInBytes, kInBytes, &sm.tma_bar);
    };
    if (blockIdx.x < n_tiles) {
        if (tid == 0) issue_load(0, blockIdx.x);
        tma_pending = true;
    }
    for (int tile = blockIdx.x; tile < n_tiles && !failed; tile += gridDim.x) {
        for (int l = 0; l < 4 && !failed; ++l) {
            const int K = layer_k(l), N = layer_n(l);
            unsigned spins = 0;
            bool ok = true;
            while (!(ok = mbar_try_wait(&sm.tma_bar, tma_phase)) && ++spins < kWaitLimit) {
            }
            if (__syncthreads_or(!ok)) { failed = true; break; }   // the copy stays pending
            tma_phase ^= 1u;
            tma_pending = false;
            if (tid == 0) {
                tc_fence_after();
                const uint32_t idesc = idesc_bf16(kRows, N);
                for (int kk = 0; kk < K / 16; ++kk)
                    mma_bf16(tmem, smem_desc(sm.act + kk * 256, 128, (K / 8) * 128),
                             smem_desc(sm.w + kk * 256, 128, (K / 8) * 128), idesc, kk > 0);
                mma_commit(&sm.mma_bar);
            }
            mma_pending = true;
            if (saved && l > 0) {   // this layer's input activation, for the backward pass
                // (read beside the MMA, which only reads it too)
                unsigned char* dst = saved + ((size_t)l * tile_cap + tile_base + tile) * kActBytes;
                for (int b = tid * 16; b < (int)kActBytes; b += kThreads * 16)
                    *reinterpret_cast<uint4*>(dst + b) = *reinterpret_cast<const uint4*>(sm.act + b);
            }
            spins = 0;
            while (!(ok = mbar_try_wait(&sm.mma_bar, mma_phase)) && ++spins < kWaitLimit) {
            }
            if (__syncthreads_or(!ok)) { failed = true; break; }   // the MMA stays pending
            mma_phase ^= 1u;
            mma_pending = false;
            tc_fence_after();
            // the weight buffer is free (and, after the last layer, the input
            // buffer): start the next layer's (or next tile's) copy now, so it
            // runs beside this epilogue
            const int next_l = l < 3 ? l + 1 : 0, next_tile = l < 3 ? tile : tile + gridDim.x;
            if (next_tile < n_tiles) {
                if (tid == 0) {
                    fence_async_shared();
                    issue_load(next_l, next_tile);
                }
                tma_pending = true;
            }
            // epilogue: this warp's 32 rows, its part of the N columns
            const int quarter = warp & 3, half = warp >> 2;
            const int row = quarter * 32 + lane;
            const unsigned lane_base = tmem + ((unsigned)(quarter * 32) << 16);
            const float* bl = bias + l * kHidden;
            if (l < 3) {
                for (int c0 = half * (N / kParts); c0 < (half + 1) * (N / kParts); c0 += 32) {
                    float v[32];
                    tmem_ld32(lane_base + c0, v);
#pragma unroll
                    for (int q = 0; q < 4; ++q) {
                        uint4 pk;
                        unsigned* pw = reinterpret_cast<unsigned*>(&pk);
                        uint4 pz;
                        unsigned* pzw = reinterpret_cast<unsigned*>(&pz);
#pragma unroll
                        for (int e = 0; e < 4; ++e) {
                            const int c = c0 + q * 8 + 2 * e;
                            const float z0 = v[q * 8 + 2 * e] + __ldg(bl + c);
                            const float z1 = v[q * 8 + 2 * e + 1] + __ldg(bl + c + 1);
                            pw[e] = pack_bf16(silu(z0), silu(z1));
                            pzw[e] = pack_bf16(z0, z1);
                        }
                        const unsigned off = tile_off(row, c0 + q * 8, kHidden);
                        *reinterpret_cast<uint4*>(sm.act + off) = pk;
                        if (zsave)   // pre-activation of layer l, for the backward pass
                            *reinterpret_cast<uint4*>(
                                zsave + ((size_t)l * tile_cap + tile_base + tile) * kActBytes + off) = pz;
                    }
                }
            } else if (half == 0) {
                float v[16];
                tmem_ld16(lane_base, v);
                const int r = tile * kRows + row;
                if (r < rows) {
                    float4* dst = reinterpret_cast<float4*>(y + (size_t)r * kOut);
#pragma unroll
                    for (int q = 0; q < 4; ++q)
                        dst[q] = make_float4(v[4 * q] + __ldg(bl + 4 * q), v[4 * q + 1] + __ldg(bl + 4 * q + 1),
                                             v[4 * q + 2] + __ldg(bl + 4 * q + 2),
                                             v[4 * q + 3] + __ldg(bl + 4 * q + 3));
                }
            }
            // the next MMA reads act (written here) and overwrites TMEM (read here)
            fence_async_shared();
            tc_fence_before();
            __syncthreads();
        }
    }
    if (failed && tid == 0) {
        atomicOr(err, 2);
        // a last bounded wait for the copy / MMA still in flight before the
        // tensor memory is released
        if (tma_pending)
            for (unsigned w = 0; w < kWaitLimit && !mbar_try_wait(&sm.tma_bar, tma_phase); ++w) {
            }
        if (mma_pending)
            for (unsigned w = 0; w < kWaitLimit && !mbar_try_wait(&sm.mma_bar, mma_phase); ++w) {
            }
    }
    __syncthreads();
    if (warp == 0) tmem_dealloc(tmem, kTmemCols);
}

// x (rows x in_dim FP32) -> zero-padded BF16 K-major tiles of 128 x kIn.
__global__ void pack_input_kernel(const float* __restrict__ x, int rows, int in_dim,
                                  unsigned char* __restrict__ out, int n_tiles) {
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    const int total = n_tiles * kRows * kIn;
    if (t >= total) return;
    const int tile = t / (kRows * kIn), rem = t % (kRows * kIn);
    const int r = rem / kIn, c = rem % kIn;
    const int gr = tile * kRows + r;
    const float v = (gr < rows && c < in_dim) ? x[(size_t)gr * in_dim + c] : 0.f;
    *reinterpret_cast<__nv_bfloat16*>(out + (size_t)tile * kInBytes + tile_off(r, c, kIn)) =
        __float2bfloat16_rn(v);
}

// Master FP32 parameters (W_l as (n_l, k_l) real sizes, then b_l) -> packed BF16
// K-major weight tiles (zero-padded to the kernel's sizes) and FP32 biases.
__global__ void pack_weights_kernel(const float* __restrict__ params, int in_dim, int out_dim,
                                    unsigned char* __restrict__ w_tiled,
                                    unsigned char* __restrict__ wt_tiled, float* __restrict__ bias) {
    const int l = blockIdx.y;
    const int K = layer_k(l), N = layer_n(l);
    const int kr = l == 0 ? in_dim : kHidden, nr = l == 3 ? out_dim : kHidden;
    const float* W = params + param_offset(l, in_dim, out_dim);
    for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < N * K; t += gridDim.x * blockDim.x) {
        const int n = t / K, k = t % K;
        const __nv_bfloat16 v = __float2bfloat16_rn((n < nr && k < kr) ? W[n * kr + k] : 0.f);
        // forward operand: (N = out, K = in); backward operand W^T: (N = in, K = out)
        *reinterpret_cast<__nv_bfloat16*>(w_tiled + layer_w_offset(l) + tile_off(n, k, K)) = v;
        *reinterpret_cast<__nv_bfloat16*>(wt_tiled + layer_w_offset(l) + tile_off(k, n, N)) = v;
    }
    if (blockIdx.x == 0)
        for (int n = threadIdx.x; n < kHidden; n += blockDim.x)
            bias[l * kHidden + n] = (n < nr) ? W[nr * kr + n] : 0.f;
}

__global__ void unpack_output_kernel(const float* __restrict__ ypad, int rows, int out_dim,
                                     float* __restrict__ y) {
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t < rows * out_dim) y[t] = ypad[(size_t)(t / out_dim) * kOut + t % out_dim];
}

__device__ __forceinline__ float silu_grad(float z) {
    const float sg = __fdividef(1.f, 1.f + __expf(-z));
    return sg * (1.f + z * (1.f - sg));
}
__device__ __forceinline__ float bf_lo(unsigned w) { return __uint_as_float(w << 16); }
__device__ __forceinline__ float bf_hi(unsigned w) { return __uint_as_float(w & 0xFFFF0000u); }

// Reverse sweep through the four layers for 128-row tiles:
//   dz_3 = dy;  da_m = dz_m W_m (MMA, B = W_m^T tiles);  dz_{m-1} = da_m * SiLU'(z_{m-1});
//   dx = da_0.
// dz_m (BF16 tiles) go to dzsave slot (m, tile_base + tile) for the weight
// gradients; zsave holds the forward's pre-activations.
__global__ void __launch_bounds__(kThreads, 1)
mlp_bwd_kernel(const float* __restrict__ dy, int rows, int out_dim, int n_tiles,
               const unsigned char* __restrict__ wt_tiled, const unsigned char* __restrict__ zsave,
               unsigned char* __restrict__ dzsave, int tile_base, int tile_cap,
               float* __restrict__ dx, int in_dim, int* __restrict__ err) {
    extern __shared__ __align__(1024) unsigned char smem_raw[];
    FwdSmem& sm = *reinterpret_cast<FwdSmem*>(smem_raw);
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    if (tid == 0) {
        mbar_init(&sm.tma_bar, 1);
        mbar_init(&sm.mma_bar, 1);
        fence_async_shared();
    }
    if (warp == 0) tmem_alloc(&sm.tmem_slot, kTmemCols);
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const unsigned tmem = sm.tmem_slot;
    const int quarter = warp & 3, half = warp >> 2;
    const int row = quarter * 32 + lane;
    unsigned tma_phase = 0, mma_phase = 0;
    bool failed = false, tma_pending = false, mma_pending = false;
    auto issue_load = [&](int m) {   // W_m^T into shared memory
        const unsigned wbytes = (unsigned)(layer_k(m) * layer_n(m) * 2);
        mbar_expect_tx(&sm.tma_bar, wbytes);
        tma_load_1d(sm.w, wt_tiled + layer_w_offset(m), wbytes, &sm.tma_bar);
    };
    if (blockIdx.x < n_tiles) {
        if (tid == 0) issue_load(3);
        tma_pending = true;
    }
    for (int tile = blockIdx.x; tile < n_tiles && !failed; tile += gridDim.x) {
        const int r = tile * kRows + row;
        const size_t slot = (size_t)tile_base + tile;
        if (half == 0) {   // dz_3 = dy as a BF16 K-major tile of 16 columns
            float d[kOut];
#pragma unroll
            for (int c = 0; c < kOut; ++c) d[c] = (r < rows && c < out_dim) ? dy[(size_t)r * out_dim + c] : 0.f;
#pragma unroll
            for (int q = 0; q < 2; ++q) {
                uint4 pk;
                unsigned* pw = reinterpret_cast<unsigned*>(&pk);
#pragma unroll
                for (int e = 0; e < 4; ++e) pw[e] = pack_bf16(d[q * 8 + 2 * e], d[q * 8 + 2 * e + 1]);
                const unsigned off = tile_off(row, q * 8, kOut);
                *reinterpret_cast<uint4*>(sm.act + off) = pk;
                *reinterpret_cast<uint4*>(dzsave + ((size_t)3 * tile_cap + slot) * kActBytes + off) = pk;
            }
        }
        fence_async_shared();
        __syncthreads();
        for (int m = 3; m >= 0 && !failed; --m) {
            const int Kb = layer_n(m), Nb = layer_k(m);   // da_m = dz_m (., Kb) W_m (Kb, Nb)
            unsigned spins = 0;
            bool ok = true;
            while (!(ok = mbar_try_wait(&sm.tma_bar, tma_phase)) && ++spins < kWaitLimit) {
            }
            if (__syncthreads_or(!ok)) { failed = true; break; }
            tma_phase ^= 1u;
            tma_pending = false;
            if (tid == 0) {
                tc_fence_after();
                const uint32_t idesc = idesc_bf16(kRows, Nb);
                for (int kk = 0; kk < Kb / 16; ++kk)
                    mma_bf16(tmem, smem_desc(sm.act + kk * 256, 128, (Kb / 8) * 128),
                             smem_desc(sm.w + kk * 256, 128, (Kb / 8) * 128), idesc, kk > 0);
                mma_commit(&sm.mma_bar);
            }
            mma_pending = true;
            spins = 0;
            while (!(ok = mbar_try_wait(&sm.mma_bar, mma_phase)) && ++spins < kWaitLimit) {
            }
            if (__syncthreads_or(!ok)) { failed = true; break; }
            mma_phase ^= 1u;
            mma_pending = false;
            tc_fence_after();
            // the weight buffer is free: the next layer's (or next tile's first)
            // weights load beside this epilogue
            if (m > 0 || tile + (int)gridDim.x < n_tiles) {
                if (tid == 0) {
                    fence_async_shared();
                    issue_load(m > 0 ? m - 1 : 3);
                }
                tma_pending = true;
            }
            const unsigned lane_base = tmem + ((unsigned)(quarter * 32) << 16);
            if (m > 0) {
                const unsigned char* zt = zsave + ((size_t)(m - 1) * tile_cap + slot) * kActBytes;
                unsigned char* dzt = dzsave + ((size_t)(m - 1) * tile_cap + slot) * kActBytes;
                for (int c0 = half * (kHidden / kParts); c0 < (half + 1) * (kHidden / kParts); c0 += 32) {
                    float v[32];
                    tmem_ld32(lane_base + c0, v);
#pragma unroll
                    for (int q = 0; q < 4; ++q) {
                        const unsigned off = tile_off(row, c0 + q * 8, kHidden);
                        const uint4 zq = *reinterpret_cast<const uint4*>(zt + off);
                        const unsigned zw[4] = {zq.x, zq.y, zq.z, zq.w};
                        uint4 pk;
                        unsigned* pw = reinterpret_cast<unsigned*>(&pk);
#pragma unroll
                        for (int e = 0; e < 4; ++e)
                            pw[e] = pack_bf16(v[q * 8 + 2 * e] * silu_grad(bf_lo(zw[e])),
                                              v[q * 8 + 2 * e + 1] * silu_grad(bf_hi(zw[e])));
                        *reinterpret_cast<uint4*>(sm.act + off) = pk;
                        *reinterpret_cast<uint4*>(dzt + off) = pk;
                    }
                }
            } else if (dx && half == 0) {
                float v[32];
                tmem_ld32(lane_base, v);
                if (r < rows)
                    for (int c = 0; c < in_dim; ++c) dx[(size_t)r * in_dim + c] = v[c];
            }
            fence_async_shared();
            tc_fence_before();
            __syncthreads();
        }
    }
    if (failed && tid == 0) {
        atomicOr(err, 2);
        if (tma_pending)
            for (unsigned w = 0; w < kWaitLimit && !mbar_try_wait(&sm.tma_bar, tma_phase); ++w) {
            }
        if (mma_pending)
            for (unsigned w = 0; w < kWaitLimit && !mbar_try_wait(&sm.mma_bar, mma_phase); ++w) {
            }
    }
    __syncthreads();
    if (warp == 0) tmem_dealloc(tmem, kTmemCols);
}

// 8x8 transpose of 16-bit elements across a warp: thread t holds row t/4,
// columns 2(t%4) and 2(t%4)+1 before and after.
__device__ __forceinline__ unsigned transpose8x8(unsigned x) {
    unsigned y;
    asm volatile("movmatrix.sync.aligned.m8n8.trans.b16 %0, %1;" : "=r"(y) : "r"(x));
    return y;
}

// Weight gradient of one layer on the tensor cores: the sum over rows of
// outer products is an MMA whose reduction dimension K is the rows.  The
// saved activations and dz tiles are K-major with K = units (a 128-byte core
// matrix = 8 rows x 8 units); for this MMA the units become M and N and the
// rows become K, so each core matrix is transposed (movmatrix) into the
// K-major operand layout in shared memory:
//   D (M = 128 units of P per blockIdx.x) x (N = NQ units of Q)
//     += P^T (M x 128 rows) . Q (128 rows x N)      per 128-row tile,
// accumulated in TMEM over the tiles of this CTA's row split (blockIdx.y),
// then stored as the split's partial; a second kernel sums the splits in
// order (deterministic: no atomics).  The bias gradient of the dz operand's
// units is summed from the transposed operand, rows in order, per split.
constexpr int kDwMaxSplits = 128;
struct DwSmem {
    alignas(128) unsigned char A[kRows * kRows * 2];     // 32 KB: 128 units x 128 rows
    alignas(128) unsigned char B[kHidden * kRows * 2];   // 64 KB: up to 256 units x 128 rows
    uint64_t mma_bar;
    unsigned tmem_slot;
};

__global__ void __launch_bounds__(kThreads, 1)
mlp_dw_tc_kernel(const unsigned char* __restrict__ P, int KP, size_t p_stride,
                 const unsigned char* __restrict__ Q, int NQ, size_t q_stride, int n_tiles,
                 int tiles_per_split, float* __restrict__ part, float* __restrict__ dbp,
                 int dz_is_P, int* __restrict__ err) {
    extern __shared__ __align__(1024) unsigned char smem_raw[];
    DwSmem& sm = *reinterpret_cast<DwSmem*>(smem_raw);
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const unsigned cols = NQ <= 32 ? 32u : NQ <= 64 ? 64u : NQ <= 128 ? 128u : 256u;
    if (tid == 0) {
        mbar_init(&sm.mma_bar, 1);
        fence_async_shared();
    }
    if (warp == 0) tmem_alloc(&sm.tmem_slot, cols);
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const unsigned tmem = sm.tmem_slot;
    const int mb = blockIdx.x, split = blockIdx.y;
    const int t0 = split * tiles_per_split, t1 = min(n_tiles, t0 + tiles_per_split);
    // the dz operand's units whose bias gradient this CTA sums (thread u: unit u)
    const int n_bias = dz_is_P ? kRows : (mb == 0 ? NQ : 0);
    const unsigned char* bias_src = dz_is_P ? sm.A : sm.B;
    float bsum = 0.f;
    unsigned mma_phase = 0;
    bool failed = false, mma_pending = false;
    const int nA = 16 * 16, nB = 16 * (NQ / 8);
    for (int t = t0; t < t1 && !failed; ++t) {
        const unsigned char* Pt = P + (size_t)t * p_stride;
        const unsigned char* Qt = Q + (size_t)t * q_stride;
        // core matrix c: row group gs (8 rows) of unit group gu, transposed;
        // each warp first issues the loads of kBatch core matrices, so that
        // many are in flight, then transposes and stores them
        constexpr int kBatch = 8, kWarps = kThreads / 32;
        const int off = (lane >> 2) * 16 + (lane & 3) * 4;
        for (int c0 = warp; c0 < nA + nB; c0 += kBatch * kWarps) {
            unsigned w[kBatch];
            unsigned char* dst[kBatch];
#pragma unroll
            for (int u = 0; u < kBatch; ++u) {
                const int c = c0 + u * kWarps;
                dst[u] = nullptr;
                if (c < nA + nB) {
                    const bool isA = c < nA;
                    const int cc = isA ? c : c - nA, gs = cc & 15, gu = cc >> 4;
                    const unsigned char* src = isA ? Pt + gs * (KP / 8) * 128 + (mb * 16 + gu) * 128
                                                   : Qt + gs * (NQ / 8) * 128 + gu * 128;
                    dst[u] = (isA ? sm.A : sm.B) + gu * 2048 + gs * 128 + off;
                    w[u] = __ldg(reinterpret_cast<const unsigned*>(src + off));
                }
            }
#pragma unroll
            for (int u = 0; u < kBatch; ++u)
                if (c0 + u * kWarps < nA + nB)   // warp-uniform: movmatrix needs the whole warp
                    *reinterpret_cast<unsigned*>(dst[u]) = transpose8x8(w[u]);
        }
        fence_async_shared();
        tc_fence_before();
        __syncthreads();
        if (tid == 0) {
            tc_fence_after();
            const uint32_t idesc = idesc_bf16(kRows, NQ);
            for (int kk = 0; kk < kRows / 16; ++kk)
                mma_bf16(tmem, smem_desc(sm.A + kk * 256, 128, 2048),
                         smem_desc(sm.B + kk * 256, 128, 2048), idesc, (t > t0 || kk > 0) ? 1u : 0u);
            mma_commit(&sm.mma_bar);
        }
        mma_pending = true;
        if (tid < n_bias) {   // bias gradient: this unit's row of the operand, rows in order
            const unsigned char* rowp = bias_src + (tid >> 3) * 2048 + (tid & 7) * 16;
            for (int g = 0; g < kRows / 8; ++g) {
                const uint4 q = *reinterpret_cast<const uint4*>(rowp + g * 128);
                const unsigned w[4] = {q.x, q.y, q.z, q.w};
#pragma unroll
                for (int e = 0; e < 4; ++e) bsum += bf_lo(w[e]) + bf_hi(w[e]);
            }
        }
        unsigned spins = 0;
        bool ok = true;
        while (!(ok = mbar_try_wait(&sm.mma_bar, mma_phase)) && ++spins < kWaitLimit) {
        }
        if (__syncthreads_or(!ok)) { failed = true; break; }   // the MMA stays pending
        mma_phase ^= 1u;
        mma_pending = false;
        tc_fence_after();
    }
    if (!failed) {
        // epilogue: TMEM lane = unit of P (row of D), column = unit of Q
        const int quarter = warp & 3, cpart = warp >> 2, row = quarter * 32 + lane;
        const unsigned lane_base = tmem + ((unsigned)(quarter * 32) << 16);
        float* out = part + ((size_t)split * gridDim.x * kRows + mb * kRows + row) * NQ;
        if (NQ >= 128) {
            for (int c0 = cpart * (NQ / 4); c0 < (cpart + 1) * (NQ / 4); c0 += 32) {
                float v[32];
                tmem_ld32(lane_base + c0, v);
#pragma unroll
                for (int q = 0; q < 8; ++q)
                    reinterpret_cast<float4*>(out + c0)[q] =
                        make_float4(v[4 * q], v[4 * q + 1], v[4 * q + 2], v[4 * q + 3]);
            }
        } else if (cpart == 0 && NQ == 32) {
            float v[32];
            tmem_ld32(lane_base, v);
#pragma unroll
            for (int q = 0; q < 8; ++q)
                reinterpret_cast<float4*>(out)[q] = make_float4(v[4 * q], v[4 * q + 1], v[4 * q + 2], v[4 * q + 3]);
        } else if (cpart == 0) {   // NQ == 16
            float v[16];
            tmem_ld16(lane_base, v);
#pragma unroll
            for (int q = 0; q < 4; ++q)
                reinterpret_cast<float4*>(out)[q] = make_float4(v[4 * q], v[4 * q + 1], v[4 * q + 2], v[4 * q + 3]);
        }
        if (tid < n_bias) dbp[(size_t)split * kHidden + (dz_is_P ? mb * kRows : 0) + tid] = bsum;
    }
    if (failed && tid == 0) {
        atomicOr(err, 2);
        if (mma_pending)
            for (unsigned w = 0; w < kWaitLimit && !mbar_try_wait(&sm.mma_bar, mma_phase); ++w) {
            }
    }
    tc_fence_before();
    __syncthreads();
    if (warp == 0) tmem_dealloc(tmem, cols);
}

// dW (real sizes out_r x in_r, added to) and db (out_r, added to) from the
// splits' partials, summed in split order.  part: [split][M][NQ] with
// M = units of P; transpose: P holds the layer's inputs (D = dW^T).
__global__ void mlp_dw_reduce_kernel(const float* __restrict__ part, const float* __restrict__ dbp,
                                     int splits, int M, int NQ, int transpose, int out_r, int in_r,
                                     float* __restrict__ dW, float* __restrict__ db) {
    const int e = blockIdx.x * blockDim.x + threadIdx.x;
    if (e < M * NQ) {
        float s = 0.f;
        for (int q = 0; q < splits; ++q) s += part[(size_t)q * M * NQ + e];
        const int m = e / NQ, n = e % NQ;
        const int o = transpose ? n : m, i = transpose ? m : n;
        if (o < out_r && i < in_r) dW[(size_t)o * in_r + i] += s;
    }
    if (e < out_r) {
        float s = 0.f;
        for (int q = 0; q < splits; ++q) s += dbp[(size_t)q * kHidden + e];
        db[e] += s;
    }
}

// Mean squared error over rows x out_dim: dy = 2 (y - t) / n, loss += sum (y-t)^2 / n.
__global__ void mse_kernel(const float* __restrict__ y, const float* __restrict__ t, int n,
                           float* __restrict__ dy, float* __restrict__ loss) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    float e2 = 0.f;
    if (i < n) {
        const float e = y[i] - t[i];
        dy[i] = 2.f * e / (float)n;
        e2 = e * e / (float)n;
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) e2 += __shfl_xor_sync(0xffffffffu, e2, o);
    if ((threadIdx.x & 31) == 0 && e2 != 0.f) atomicAdd(loss, e2);
}

// Adam (Kingma & Ba 2015) minimising along g.
__global__ void param_adam_kernel(float* __restrict__ p, const float* __restrict__ g,
                                  float* __restrict__ m, float* __restrict__ v, int n, float lr,
                                  float bc1, float bc2) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const float mt = 0.9f * m[i] + 0.1f * g[i];
    const float vt = 0.999f * v[i] + 0.001f * g[i] * g[i];
    m[i] = mt;
    v[i] = vt;
    p[i] -= lr * (mt / bc1) / (sqrtf(vt / bc2) + 1e-8f);
}

}  // namespace

size_t fwd_smem_bytes() { return sizeof(FwdSmem) + 1024; }

cudaError_t pack_weights(const float* params, int in_dim, int out_dim, unsigned char* w_tiled,
                         unsigned char* wt_tiled, float* bias, cudaStream_t st) {
    pack_weights_kernel<<<dim3(64, 4), 256, 0, st>>>(params, in_dim, out_dim, w_tiled, wt_tiled,
                                                     bias);
    return cudaGetLastError();
}

cudaError_t forward(const float* x, int rows, int in_dim, int out_dim, const unsigned char* w_tiled,
                    const float* bias, unsigned char* x_tiled, float* ypad, float* y,
                    unsigned char* saved, unsigned char* zsave, int tile_base, int tile_cap,
                    int* err, int sm_count, cudaStream_t st) {
    const int n_tiles = (rows + kRows - 1) / kRows;
    unsigned char* xt = x_tiled + (size_t)tile_base * kInBytes;
    const int total = n_tiles * kRows * kIn;
    pack_input_kernel<<<(total + 255) / 256, 256, 0, st>>>(x, rows, in_dim, xt, n_tiles);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    const size_t smem = fwd_smem_bytes();
    e = cudaFuncSetAttribute(mlp_fwd_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    const int grid = n_tiles < sm_count ? n_tiles : sm_count;
    mlp_fwd_kernel<<<grid, kThreads, smem, st>>>(xt, n_tiles, w_tiled, bias, ypad, rows, saved,
                                                 zsave, tile_base, tile_cap, err);
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    unpack_output_kernel<<<(rows * out_dim + 255) / 256, 256, 0, st>>>(ypad, rows, out_dim, y);
    return cudaGetLastError();
}

cudaError_t backward(const float* dy, int rows, int in_dim, int out_dim,
                     const unsigned char* wt_tiled, const unsigned char* zsave,
                     unsigned char* dzsave, int tile_base, int tile_cap, float* dx, int* err,
                     int sm_count, cudaStream_t st) {
    const int n_tiles = (rows + kRows - 1) / kRows;
    const size_t smem = fwd_smem_bytes();
    cudaError_t e = cudaFuncSetAttribute(mlp_bwd_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)smem);
    if (e != cudaSuccess) return e;
    const int grid = n_tiles < sm_count ? n_tiles : sm_count;
    mlp_bwd_kernel<<<grid, kThreads, smem, st>>>(dy, rows, out_dim, n_tiles, wt_tiled, zsave,
                                                 dzsave, tile_base, tile_cap, dx, in_dim, err);
    return cudaGetLastError();
}

size_t dw_part_floats() { return (size_t)kDwMaxSplits * (kHidden * kHidden + kHidden); }

cudaError_t weight_grads(const unsigned char* x_tiled, const unsigned char* saved,
                         const unsigned char* dzsave, int tile_base, int tile_cap, int rows,
                         int in_dim, int out_dim, float* grad, float* part, int* err, int sm_count,
                         cudaStream_t st) {
    const int n_tiles = (rows + kRows - 1) / kRows;
    const size_t smem = sizeof(DwSmem) + 1024;
    cudaError_t e = cudaFuncSetAttribute(mlp_dw_tc_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)smem);
    if (e != cudaSuccess) return e;
    float* dbp = part + (size_t)kDwMaxSplits * kHidden * kHidden;
    for (int l = 0; l < kLayers; ++l) {
        const int in_r = l == 0 ? in_dim : kHidden, out_r = l == 3 ? out_dim : kHidden;
        const unsigned char* a = l == 0 ? x_tiled + (size_t)tile_base * kInBytes
                                        : saved + ((size_t)l * tile_cap + tile_base) * kActBytes;
        const size_t a_stride = l == 0 ? kInBytes : kActBytes;
        const unsigned char* dz = dzsave + ((size_t)l * tile_cap + tile_base) * kActBytes;
        // P: the operand of 256 units (M in 128-unit blocks); Q: the other one
        const bool dz_is_P = layer_n(l) == kHidden;
        const unsigned char* P = dz_is_P ? dz : a;
        const unsigned char* Q = dz_is_P ? a : dz;
        const int KP = dz_is_P ? layer_n(l) : layer_k(l), NQ = dz_is_P ? layer_k(l) : layer_n(l);
        const size_t p_stride = dz_is_P ? kActBytes : a_stride, q_stride = dz_is_P ? a_stride : kActBytes;
        const int mblocks = KP / kRows;
        int splits = sm_count / mblocks;
        splits = splits < 1 ? 1 : splits > kDwMaxSplits ? kDwMaxSplits : splits;
        splits = splits > n_tiles ? n_tiles : splits;
        const int per = (n_tiles + splits - 1) / splits;
        splits = (n_tiles + per - 1) / per;
        mlp_dw_tc_kernel<<<dim3(mblocks, splits), kThreads, smem, st>>>(
            P, KP, p_stride, Q, NQ, q_stride, n_tiles, per, part, dbp, dz_is_P ? 1 : 0, err);
        e = cudaGetLastError();
        if (e != cudaSuccess) return e;
        float* dW = grad + param_offset(l, in_dim, out_dim);
        mlp_dw_reduce_kernel<<<(KP * NQ + 255) / 256, 256, 0, st>>>(
            part, dbp, splits, KP, NQ, dz_is_P ? 0 : 1, out_r, in_r, dW, dW + (size_t)out_r * in_r);
        e = cudaGetLastError();
        if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
}

cudaError_t mse(const float* y, const float* t, int n, float* dy, float* loss, cudaStream_t st) {
    mse_kernel<<<(n + 255) / 256, 256, 0, st>>>(y, t, n, dy, loss);
    return cudaGetLastError();
}

cudaError_t adam(float* p, const float* g, float* m, float* v, int n, int step, float lr,
                 cudaStream_t st) {
    const float bc1 = 1.f - powf(0.9f, (float)step), bc2 = 1.f - powf(0.999f, (float)step);
    param_adam_kernel<<<(n + 255) / 256, 256, 0, st>>>(p, g, m, v, n, lr, bc1, bc2);
    return cudaGetLastError();
}

}  // namespace mlp
}  // namespace stamp

// ----------------------------- C ABI ----------------------------------------
struct stamp_mlp {
    int in_dim = 0, out_dim = 0, max_rows = 0, train_rows = 0, tile_cap = 0, sm_count = 0;
    size_t n_params = 0;
    cudaStream_t stream = nullptr;
    char* arena = nullptr;
    unsigned char *w_tiled = nullptr, *wt_tiled = nullptr, *x_tiled = nullptr;
    unsigned char *saved = nullptr, *zsave = nullptr, *dzsave = nullptr;
    float *bias = nullptr, *ypad = nullptr, *ytrain = nullptr, *dy = nullptr;
    float *grad = nullptr, *adam_m = nullptr, *adam_v = nullptr, *loss = nullptr;
    float* dw_part = nullptr;   // per-split partial weight gradients (deterministic reduction)
    int* err = nullptr;
    int step = 0;
};

namespace {
stamp_status mlp_fail(stamp_status s, const char* msg, cudaError_t e = cudaSuccess) {
    char buf[256];
    std::strncpy(buf, msg, sizeof buf - 1);
    buf[sizeof buf - 1] = 0;
    if (e != cudaSuccess) {
        cudaGetLastError();
        std::strncat(buf, ": ", sizeof buf - std::strlen(buf) - 1);
        std::strncat(buf, cudaGetErrorString(e), sizeof buf - std::strlen(buf) - 1);
    }
    stamp::set_last_error(buf);
    return s;
}
bool on_device(const void* p) {
    cudaPointerAttributes at;
    if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return at.type == cudaMemoryTypeDevice || at.type == cudaMemoryTypeManaged;
}
#define MLP_TRY(call, what)                                          \
    do {                                                             \
        cudaError_t e_ = (call);                                     \
        if (e_ != cudaSuccess) return mlp_fail(STAMP_ECUDA, what, e_); \
    } while (0)
}  // namespace

extern "C" stamp_status stamp_mlp_create(int in_dim, int out_dim, int max_rows, int train_rows,
                                         void* cuda_stream, stamp_mlp** out) {
    using namespace stamp::mlp;
    if (!out) return mlp_fail(STAMP_EINVAL, "out is NULL");
    *out = nullptr;
    if (in_dim < 1 || in_dim > kIn || out_dim < 1 || out_dim > kOut || max_rows < 1 || train_rows < 0)
        return mlp_fail(STAMP_EINVAL,
                        "need 1 <= in_dim <= 32, 1 <= out_dim <= 16, max_rows >= 1, train_rows >= 0");
    stamp_mlp* m = new stamp_mlp();
    m->in_dim = in_dim; m->out_dim = out_dim; m->max_rows = max_rows; m->train_rows = train_rows;
    m->tile_cap = (train_rows + 127) / 128;
    m->n_params = param_count(in_dim, out_dim);
    m->stream = static_cast<cudaStream_t>(cuda_stream);
    int dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&m->sm_count, cudaDevAttrMultiProcessorCount, dev);
    const size_t xt = (size_t)((max_rows > train_rows ? max_rows : train_rows) + 127) / 128;
    const size_t cap = (size_t)m->tile_cap, np = m->n_params;
    void** dst[] = {(void**)&m->w_tiled, (void**)&m->wt_tiled, (void**)&m->x_tiled, (void**)&m->bias,
                    (void**)&m->ypad,    (void**)&m->saved,    (void**)&m->zsave,   (void**)&m->dzsave,
                    (void**)&m->ytrain,  (void**)&m->dy,       (void**)&m->grad,    (void**)&m->adam_m,
                    (void**)&m->adam_v,  (void**)&m->loss,     (void**)&m->err,     (void**)&m->dw_part};
    const size_t bytes[] = {kWeightBytes, kWeightBytes, xt * 128 * kIn * 2, (size_t)kLayers * kHidden * 4,
                            (size_t)max_rows * kOut * 4, 4 * cap * kRows * kHidden * 2,
                            3 * cap * kRows * kHidden * 2, 4 * cap * kRows * kHidden * 2,
                            (size_t)train_rows * out_dim * 4, (size_t)train_rows * out_dim * 4,
                            np * 4, np * 4, np * 4, 4, 4,
                            train_rows > 0 ? dw_part_floats() * 4 : 0};
    size_t total = 0;
    for (size_t b : bytes) total += (b + 255) / 256 * 256;
    cudaError_t e = cudaMalloc(&m->arena, total);
    if (e != cudaSuccess) { delete m; return mlp_fail(STAMP_ENOMEM, "cudaMalloc failed", e); }
    char* p = m->arena;
    for (size_t q = 0; q < sizeof bytes / sizeof bytes[0]; ++q) {
        *dst[q] = p;
        p += (bytes[q] + 255) / 256 * 256;
    }
    e = cudaMemset(m->arena, 0, total);
    if (e != cudaSuccess) { cudaFree(m->arena); delete m; return mlp_fail(STAMP_ECUDA, "memset failed", e); }
    *out = m;
    return STAMP_OK;
}

extern "C" void stamp_mlp_destroy(stamp_mlp* m) {
    if (!m) return;
    cudaStreamSynchronize(m->stream);
    cudaFree(m->arena);
    delete m;
}

extern "C" size_t stamp_mlp_param_count(int in_dim, int out_dim) {
    return stamp::mlp::param_count(in_dim, out_dim);
}

extern "C" stamp_status stamp_mlp_set_params(stamp_mlp* m, const float* params) {
    if (!m || !params || !on_device(params)) return mlp_fail(STAMP_EINVAL, "NULL mlp or non-device params");
    MLP_TRY(stamp::mlp::pack_weights(params, m->in_dim, m->out_dim, m->w_tiled, m->wt_tiled, m->bias,
                                     m->stream), "weight packing failed");
    return STAMP_OK;
}

extern "C" stamp_status stamp_mlp_forward(stamp_mlp* m, const float* x, int rows, float* y) {
    if (!m || !x || !y || !on_device(x) || !on_device(y)) return mlp_fail(STAMP_EINVAL, "NULL or non-device argument");
    if (rows < 1 || rows > m->max_rows) return mlp_fail(STAMP_EINVAL, "rows outside [1, max_rows]");
    MLP_TRY(stamp::mlp::forward(x, rows, m->in_dim, m->out_dim, m->w_tiled, m->bias, m->x_tiled,
                                m->ypad, y, nullptr, nullptr, 0, 0, m->err, m->sm_count, m->stream),
            "MLP forward launch failed");
    return STAMP_OK;
}

extern "C" stamp_status stamp_mlp_forward_saved(stamp_mlp* m, const float* x, int rows, float* y,
                                                int tile_base) {
    if (!m || !x || !y || !on_device(x) || !on_device(y)) return mlp_fail(STAMP_EINVAL, "NULL or non-device argument");
    const int tiles = (rows + 127) / 128;
    if (rows < 1 || rows > m->max_rows || tile_base < 0 || tile_base + tiles > m->tile_cap)
        return mlp_fail(STAMP_EINVAL, "rows / tile_base outside the saved-activation capacity");
    MLP_TRY(stamp::mlp::forward(x, rows, m->in_dim, m->out_dim, m->w_tiled, m->bias, m->x_tiled,
                                m->ypad, y, m->saved, m->zsave, tile_base, m->tile_cap, m->err,
                                m->sm_count, m->stream),
            "MLP forward launch failed");
    return STAMP_OK;
}

extern "C" stamp_status stamp_mlp_backward(stamp_mlp* m, const float* dy, int rows, int tile_base,
                                           float* dx, float* dparams) {
    if (!m || !dy || !on_device(dy) || (dx && !on_device(dx)) || (dparams && !on_device(dparams)))
        return mlp_fail(STAMP_EINVAL, "NULL or non-device argument");
    const int tiles = (rows + 127) / 128;
    if (rows < 1 || tile_base < 0 || tile_base + tiles > m->tile_cap)
        return mlp_fail(STAMP_EINVAL, "rows / tile_base outside the saved-activation capacity");
    MLP_TRY(stamp::mlp::backward(dy, rows, m->in_dim, m->out_dim, m->wt_tiled, m->zsave, m->dzsave,
                                 tile_base, m->tile_cap, dx, m->err, m->sm_count, m->stream),
            "MLP backward launch failed");
    if (dparams) {
        MLP_TRY(cudaMemsetAsync(dparams, 0, m->n_params * 4, m->stream), "memset failed");
        MLP_TRY(stamp::mlp::weight_grads(m->x_tiled, m->saved, m->dzsave, tile_base, m->tile_cap,
                                         rows, m->in_dim, m->out_dim, dparams, m->dw_part, m->err,
                                         m->sm_count, m->stream),
                "weight-gradient launch failed");
    }
    return STAMP_OK;
}

extern "C" stamp_status stamp_mlp_train(stamp_mlp* m, float* params, const float* x,
                                        const float* target, int rows, int epochs, int batch,
                                        float lr, float* loss_out) {
    if (!m || !params || !x || !target || !on_device(params) || !on_device(x) || !on_device(target))
        return mlp_fail(STAMP_EINVAL, "NULL or non-device argument");
    if (batch < 1 || batch > m->train_rows || batch > m->max_rows || rows < batch || epochs < 1)
        return mlp_fail(STAMP_EINVAL, "need 1 <= batch <= train_rows, rows >= batch, epochs >= 1");
    const int nb = rows / batch, n = batch * m->out_dim;
    std::vector<float> losses(epochs);
    for (int ep = 0; ep < epochs; ++ep) {
        MLP_TRY(cudaMemsetAsync(m->loss, 0, 4, m->stream), "memset failed");
        for (int b = 0; b < nb; ++b) {
            MLP_TRY(stamp::mlp::pack_weights(params, m->in_dim, m->out_dim, m->w_tiled, m->wt_tiled,
                                             m->bias, m->stream), "weight packing failed");
            MLP_TRY(stamp::mlp::forward(x + (size_t)b * batch * m->in_dim, batch, m->in_dim, m->out_dim,
                                        m->w_tiled, m->bias, m->x_tiled, m->ypad, m->ytrain, m->saved,
                                        m->zsave, 0, m->tile_cap, m->err, m->sm_count, m->stream),
                    "MLP forward launch failed");
            MLP_TRY(stamp::mlp::mse(m->ytrain, target + (size_t)b * n, n, m->dy, m->loss, m->stream),
                    "loss launch failed");
            MLP_TRY(stamp::mlp::backward(m->dy, batch, m->in_dim, m->out_dim, m->wt_tiled, m->zsave,
                                         m->dzsave, 0, m->tile_cap, nullptr, m->err, m->sm_count,
                                         m->stream), "MLP backward launch failed");
            MLP_TRY(cudaMemsetAsync(m->grad, 0, m->n_params * 4, m->stream), "memset failed");
            MLP_TRY(stamp::mlp::weight_grads(m->x_tiled, m->saved, m->dzsave, 0, m->tile_cap, batch,
                                             m->in_dim, m->out_dim, m->grad, m->dw_part, m->err,
                                             m->sm_count, m->stream),
                    "weight-gradient launch failed");
            MLP_TRY(stamp::mlp::adam(params, m->grad, m->adam_m, m->adam_v, (int)m->n_params,
                                     ++m->step, lr, m->stream), "Adam launch failed");
        }
        float l = 0.f;
        MLP_TRY(cudaMemcpyAsync(&l, m->loss, 4, cudaMemcpyDeviceToHost, m->stream), "copy failed");
        MLP_TRY(cudaStreamSynchronize(m->stream), "synchronisation failed");
        losses[ep] = l / nb;
    }
    if (loss_out) std::memcpy(loss_out, losses.data(), epochs * sizeof(float));
    int f = 0;
    MLP_TRY(cudaMemcpy(&f, m->err, sizeof f, cudaMemcpyDeviceToHost), "flag read failed");
    if (f) {
        cudaMemset(m->err, 0, sizeof(int));
        return mlp_fail(STAMP_ETIMEOUT, "a bounded device wait of the MLP kernels gave up");
    }
    return STAMP_OK;
}

extern "C" stamp_status stamp_mlp_sync(stamp_mlp* m) {
    if (!m) return mlp_fail(STAMP_EINVAL, "NULL mlp");
    MLP_TRY(cudaStreamSynchronize(m->stream), "stream synchronisation failed");
    int f = 0;
    MLP_TRY(cudaMemcpy(&f, m->err, sizeof f, cudaMemcpyDeviceToHost), "flag read failed");
    if (f) {
        cudaMemset(m->err, 0, sizeof(int));
        return mlp_fail(STAMP_ETIMEOUT, "a bounded device wait of the MLP kernels gave up");
    }
    return STAMP_OK;
}
