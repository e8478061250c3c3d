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

#include "mlp.cuh"
#include "stamp.h"
#include "stamp_internal.cuh"

namespace stamp {
namespace mlp {
namespace {

__device__ __forceinline__ unsigned smem_u32(const void* p) {
    return (unsigned)__cvta_generic_to_shared(p);
}

// ---------------- mbarrier + TMA bulk copy ----------------------------------
__device__ __forceinline__ void mbar_init(uint64_t* bar, unsigned count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count)
                 : "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, unsigned bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)),
                 "r"(bytes)
                 : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, unsigned parity) {
    unsigned ok;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
        " selp.u32 %0, 1, 0, p;\n}"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}
__device__ __forceinline__ void tma_load_1d(void* dst, const void* src, unsigned bytes,
                                           uint64_t* bar) {
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];"
        ::"r"(smem_u32(dst)), "l"(src), "r"(bytes), "r"(smem_u32(bar))
        : "memory");
}
__device__ __forceinline__ void fence_async_shared() {
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}
constexpr unsigned kWaitLimit = 1u << 22;

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
__device__ __forceinline__ float silu(float z) { return z / (1.f + __expf(-z)); }

// Byte offset of element (row, col) in a K-major core-matrix tile of K columns.
__host__ __device__ __forceinline__ unsigned tile_off(int row, int col, int K) {
    return (unsigned)((row >> 3) * (K / 8) * 128 + (col >> 3) * 128 + (row & 7) * 16 + (col & 7) * 2);
}

constexpr int kRows = 128;                        // rows per tile (MMA M)
constexpr int kThreads = 128;                     // 4 warps: one TMEM lane quarter each
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
// Optionally stores every layer's input activation (BF16, tiled) for the
// backward pass: saved + l * rows_pad * kHidden * 2 bytes (layer 0 input is x).
__global__ void __launch_bounds__(kThreads, 1)
mlp_fwd_kernel(const unsigned char* __restrict__ x_tiled, int n_tiles,
               const unsigned char* __restrict__ w_tiled, const float* __restrict__ bias,
               float* __restrict__ y, int rows, unsigned char* __restrict__ saved,
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
    bool failed = false;
    for (int tile = blockIdx.x; tile < n_tiles && !failed; tile += gridDim.x) {
        for (int l = 0; l < 4 && !failed; ++l) {
            const int K = layer_k(l), N = layer_n(l);
            if (tid == 0) {
                // act and w are free: the previous MMA has completed
                const unsigned wbytes = (unsigned)(N * K * 2);
                mbar_expect_tx(&sm.tma_bar, wbytes + (l == 0 ? kInBytes : 0u));
                tma_load_1d(sm.w, w_tiled + layer_w_offset(l), wbytes, &sm.tma_bar);
                if (l == 0) tma_load_1d(sm.act, x_tiled + (size_t)tile * kInBytes, kInBytes, &sm.tma_bar);
            }
            unsigned spins = 0;
            while (!mbar_try_wait(&sm.tma_bar, tma_phase) && ++spins < kWaitLimit) {
            }
            tma_phase ^= 1u;
            if (__syncthreads_or(spins >= kWaitLimit)) { failed = true; break; }
            if (saved && l > 0) {   // this layer's input activation, for the backward pass
                unsigned char* dst = saved + ((size_t)l * n_tiles + tile) * kActBytes;
                for (int b = tid * 16; b < (int)kActBytes; b += kThreads * 16)
                    *reinterpret_cast<uint4*>(dst + b) = *reinterpret_cast<const uint4*>(sm.act + b);
            }
            if (tid == 0) {
                tc_fence_after();
                const uint32_t idesc = idesc_bf16(kRows, N);
                for (int kk = 0; kk < K / 16; ++kk)
                    mma_bf16(tmem, smem_desc(sm.act + kk * 256, 128, (K / 8) * 128),
                             smem_desc(sm.w + kk * 256, 128, (K / 8) * 128), idesc, kk > 0);
                mma_commit(&sm.mma_bar);
            }
            spins = 0;
            while (!mbar_try_wait(&sm.mma_bar, mma_phase) && ++spins < kWaitLimit) {
            }
            mma_phase ^= 1u;
            if (__syncthreads_or(spins >= kWaitLimit)) { failed = true; break; }
            tc_fence_after();
            // epilogue: this warp's 32 rows, all N columns
            const int row = warp * 32 + lane;
            const unsigned lane_base = tmem + ((unsigned)(warp * 32) << 16);
            const float* bl = bias + l * kHidden;
            if (l < 3) {
                for (int c0 = 0; c0 < N; c0 += 32) {
                    float v[32];
                    tmem_ld32(lane_base + c0, v);
#pragma unroll
                    for (int q = 0; q < 4; ++q) {
                        uint4 pk;
                        unsigned* pw = reinterpret_cast<unsigned*>(&pk);
#pragma unroll
                        for (int e = 0; e < 4; ++e) {
                            const int c = c0 + q * 8 + 2 * e;
                            pw[e] = pack_bf16(silu(v[q * 8 + 2 * e] + __ldg(bl + c)),
                                              silu(v[q * 8 + 2 * e + 1] + __ldg(bl + c + 1)));
                        }
                        *reinterpret_cast<uint4*>(sm.act + tile_off(row, c0 + q * 8, kHidden)) = pk;
                    }
                }
            } else {
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
        for (unsigned w = 0; w < kWaitLimit && !mbar_try_wait(&sm.tma_bar, tma_phase ^ 1u); ++w) {
        }
        for (unsigned w = 0; w < kWaitLimit && !mbar_try_wait(&sm.mma_bar, mma_phase ^ 1u); ++w) {
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
                                    unsigned char* __restrict__ w_tiled, float* __restrict__ bias) {
    const int l = blockIdx.y;
    const int K = layer_k(l), N = layer_n(l);
    const int kr = l == 0 ? in_dim : kHidden, nr = l == 3 ? out_dim : kHidden;
    const float* W = params + param_offset(l, in_dim, out_dim);
    for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < N * K; t += gridDim.x * blockDim.x) {
        const int n = t / K, k = t % K;
        const float v = (n < nr && k < kr) ? W[n * kr + k] : 0.f;
        *reinterpret_cast<__nv_bfloat16*>(w_tiled + layer_w_offset(l) + tile_off(n, k, K)) =
            __float2bfloat16_rn(v);
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

}  // namespace

size_t fwd_smem_bytes() { return sizeof(FwdSmem) + 1024; }

cudaError_t pack_weights(const float* params, int in_dim, int out_dim, unsigned char* w_tiled,
                         float* bias, cudaStream_t st) {
    pack_weights_kernel<<<dim3(64, 4), 256, 0, st>>>(params, in_dim, out_dim, w_tiled, bias);
    return cudaGetLastError();
}

cudaError_t forward(const float* x, int rows, int in_dim, int out_dim, const unsigned char* w_tiled,
                    const float* bias, unsigned char* x_tiled, float* ypad, float* y,
                    unsigned char* saved, int* err, int sm_count, cudaStream_t st) {
    const int n_tiles = (rows + kRows - 1) / kRows;
    const int total = n_tiles * kRows * kIn;
    pack_input_kernel<<<(total + 255) / 256, 256, 0, st>>>(x, rows, in_dim, x_tiled, n_tiles);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    const size_t smem = fwd_smem_bytes();
    e = cudaFuncSetAttribute(mlp_fwd_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    const int grid = n_tiles < sm_count ? n_tiles : sm_count;
    mlp_fwd_kernel<<<grid, kThreads, smem, st>>>(x_tiled, n_tiles, w_tiled, bias, ypad, rows, saved,
                                                 err);
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    unpack_output_kernel<<<(rows * out_dim + 255) / 256, 256, 0, st>>>(ypad, rows, out_dim, y);
    return cudaGetLastError();
}

}  // namespace mlp
}  // namespace stamp

// ----------------------------- C ABI ----------------------------------------
struct stamp_mlp {
    int in_dim = 0, out_dim = 0, max_rows = 0, sm_count = 0;
    cudaStream_t stream = nullptr;
    char* arena = nullptr;
    unsigned char *w_tiled = nullptr, *x_tiled = nullptr;
    float *bias = nullptr, *ypad = nullptr;
    int* err = nullptr;
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
}  // namespace

extern "C" stamp_status stamp_mlp_create(int in_dim, int out_dim, int max_rows, void* cuda_stream,
                                         stamp_mlp** out) {
    using namespace stamp::mlp;
    if (!out) return mlp_fail(STAMP_EINVAL, "out is NULL");
    *out = nullptr;
    if (in_dim < 1 || in_dim > kIn || out_dim < 1 || out_dim > kOut || max_rows < 1)
        return mlp_fail(STAMP_EINVAL, "need 1 <= in_dim <= 32, 1 <= out_dim <= 16, max_rows >= 1");
    stamp_mlp* m = new stamp_mlp();
    m->in_dim = in_dim; m->out_dim = out_dim; m->max_rows = max_rows;
    m->stream = static_cast<cudaStream_t>(cuda_stream);
    int dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&m->sm_count, cudaDevAttrMultiProcessorCount, dev);
    const size_t tiles = ((size_t)max_rows + 127) / 128;
    const size_t parts[] = {kWeightBytes, tiles * 128 * kIn * 2, (size_t)kLayers * kHidden * 4,
                            (size_t)max_rows * kOut * 4, 256};
    size_t total = 0;
    for (size_t b : parts) total += (b + 255) / 256 * 256;
    cudaError_t e = cudaMalloc(&m->arena, total);
    if (e != cudaSuccess) { delete m; return mlp_fail(STAMP_ENOMEM, "cudaMalloc failed", e); }
    char* p = m->arena;
    m->w_tiled = reinterpret_cast<unsigned char*>(p); p += (parts[0] + 255) / 256 * 256;
    m->x_tiled = reinterpret_cast<unsigned char*>(p); p += (parts[1] + 255) / 256 * 256;
    m->bias = reinterpret_cast<float*>(p); p += (parts[2] + 255) / 256 * 256;
    m->ypad = reinterpret_cast<float*>(p); p += (parts[3] + 255) / 256 * 256;
    m->err = reinterpret_cast<int*>(p);
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
    if (!m || !params) return mlp_fail(STAMP_EINVAL, "NULL mlp or params");
    cudaError_t e = stamp::mlp::pack_weights(params, m->in_dim, m->out_dim, m->w_tiled, m->bias,
                                             m->stream);
    return e == cudaSuccess ? STAMP_OK : mlp_fail(STAMP_ECUDA, "weight packing failed", e);
}

extern "C" stamp_status stamp_mlp_forward(stamp_mlp* m, const float* x, int rows, float* y) {
    if (!m || !x || !y) return mlp_fail(STAMP_EINVAL, "NULL argument");
    if (rows < 1 || rows > m->max_rows) return mlp_fail(STAMP_EINVAL, "rows outside [1, max_rows]");
    cudaError_t e = stamp::mlp::forward(x, rows, m->in_dim, m->out_dim, m->w_tiled, m->bias,
                                        m->x_tiled, m->ypad, y, nullptr, m->err, m->sm_count,
                                        m->stream);
    return e == cudaSuccess ? STAMP_OK : mlp_fail(STAMP_ECUDA, "MLP forward launch failed", e);
}

extern "C" stamp_status stamp_mlp_sync(stamp_mlp* m) {
    if (!m) return mlp_fail(STAMP_EINVAL, "NULL mlp");
    cudaError_t e = cudaStreamSynchronize(m->stream);
    if (e != cudaSuccess) return mlp_fail(STAMP_ECUDA, "stream synchronisation failed", e);
    int f = 0;
    e = cudaMemcpy(&f, m->err, sizeof f, cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) return mlp_fail(STAMP_ECUDA, "flag read failed", e);
    if (f) {
        cudaMemset(m->err, 0, sizeof(int));
        return mlp_fail(STAMP_ETIMEOUT, "a bounded device wait of the MLP kernel gave up");
    }
    return STAMP_OK;
}
