// Persistent batched Stein iteration: one launch per iteration of Algorithm 1
// over every active instance of a batch (instances of 1-4 blocks, any
// horizon and particle count).
//
// The grid is the GPU's resident capacity (one CTA of 256 threads per SM at
// the adjoint's register count; two CTAs of 128 threads, which let a Stein
// item share an SM with a rollout item, measured slower: the two items'
// loop bodies contend for the instruction cache).  Each CTA takes the next
// work item from a device-wide counter until the queue is empty:
//   rollout items     8 warp tasks; a task is one warp's teams of one
//                     instance: the forward rollout (tape + cost), then the
//                     checkpointed reverse sweep over that tape (gradient of
//                     log rho) -- the same team bodies as the per-class
//                     launches, lanes fixed per block count; the CTA's warps
//                     all finish their forwards before the adjoints start
//                     (one loop body in the SM's instruction cache at a time);
//   pairwise strips   d2 for up to eight tile pairs of one tile row, and the
//                     median's first radix digit;
//   median CTAs       the second digit, then the third (h);
//   Stein blocks      phi for 32 rows and one j-share (Eq. svgd);
//   Adam chunks       4096 elements of theta, m, v (the shares summed in
//                     order, as the per-piece Adam does).
// An item waits only on items of its own instance that come earlier in the
// queue (per-instance completion counters); every item it waits on has been
// taken by a running CTA and waits only on earlier items in turn, so the
// waits end without any assumption on how many CTAs are resident.  Each wait
// is bounded in time: on expiry the CTA sets the error flag and an abort word,
// and every CTA skips the rest of the queue.  The last CTA out resets the
// queue and the counters and advances the iteration and Adam step, so the
// launch can be replayed from a CUDA graph.
//
// Rollout items are dealt longest first (the host orders them by horizon and
// block count); the Stein blocks follow in the order the host expects the
// instances' rollouts to finish.  Every per-instance buffer starts on a
// 128-byte boundary, so no cache line is shared by two instances' data.
#include "rollout.cuh"
#include "svgd_bodies.cuh"

namespace stamp {
namespace {

constexpr unsigned kMaxPolls = 1u << 26;   // backstop of the timed waits

// trace: when the CTA's current item had its dependencies met
__shared__ unsigned long long start_sh;

__device__ __forceinline__ unsigned ld_acquire(const unsigned* p) {
    unsigned v;
    asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}
__device__ __forceinline__ unsigned long long now_ns() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

// Whole CTA: thread 0 polls until c0 >= t0 and (c1 == NULL or c1 >= t1).
// False if the wait ran out (flag and abort word set) or another CTA aborted.
__device__ bool wait_counts(const PersistArgs& p, const unsigned* c0, unsigned t0,
                            const unsigned* c1, unsigned t1) {
    __shared__ int ok_sh;
    if (threadIdx.x == 0) {
        int ok = 1;
        const unsigned long long start = now_ns();
        unsigned polls = 0;
        while (ld_acquire(c0) < t0 || (c1 && ld_acquire(c1) < t1)) {
            if (ld_acquire(p.ctr + 2)) {
                ok = 0;
                break;
            }
            if (++polls >= kMaxPolls || now_ns() - start > p.wait_ns) {
                atomicOr(p.flag, 2);
                atomicExch(p.ctr + 2, 1u);
                ok = 0;
                break;
            }
            __nanosleep(256);
        }
        __threadfence();
        ok_sh = ok;
        if (p.trace) start_sh = now_ns();
    }
    __syncthreads();
    const bool ok = ok_sh != 0;
    __syncthreads();
    return ok;
}

// Whole CTA: every thread's writes, then one count.
__device__ __forceinline__ void cta_signal(unsigned* c) {
    __threadfence();
    __syncthreads();
    if (threadIdx.x == 0) atomicAdd(c, 1u);
}

// One warp task: the warp's teams of instance g starting at particle `first`;
// phase 0 the forward rollout, phase 1 the adjoint over the tape it wrote.
template <int NB>
__device__ __forceinline__ void roll_warp(const SimConst& sc0, const PersistArgs& p, int g,
                                          int first, float2* wseg, int phase) {
    constexpr int L = persist_lanes(NB);
    const BatchInst& in = p.inst[g];
    SimConst sc = sc0;
    sc.H = in.H;
    sc.D = in.D;
    sc.n_ckpt = in.n_ckpt;
#pragma unroll
    for (int q = 0; q < NB; ++q)
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            sc.init[q][c] = in.init[q][c];
            sc.goal[q][c] = in.goal[q][c];
        }
    RolloutArgs a{};
    a.theta = in.theta;
    a.N = in.N;
    a.seed = in.seed;
    a.iter = *p.iter;
    a.hard = 0;
    a.tape = in.tape;
    a.cost = in.cost;
    a.grad = in.grad;
    a.dropped = p.dropped;
    const int lane32 = threadIdx.x & 31;
    int i = first + lane32 / L;
    const bool on = i < in.N;
    if (!on) i = in.N - 1;   // surplus teams shadow the last particle, store nothing
    if (phase == 0)
        rollout::fwd_team<NB, L>(sc, a, i, on, lane32 & (L - 1));
    else
        rollout::adj_team<NB, L, true>(sc, a, i, on, lane32 & (L - 1),
                                       wseg + (size_t)(lane32 / L) * rollout::seg_stride<NB>(sc.C));
}

// Adam (Kingma & Ba 2015) on elements [chunk*kPersistAdamChunk, ...) of instance s.
__device__ __forceinline__ void adam_chunk(const PersistArgs& p, const SvgdInst& s, int chunk) {
    const long long ne = (long long)s.N * s.D;
    const long long b0 = (long long)chunk * kPersistAdamChunk;
    const long long e0 = b0 + kPersistAdamChunk < ne ? b0 + kPersistAdamChunk : ne;
    const float2 b12 = p.bc[*p.step + 1];
    const float bc1 = b12.x, bc2 = b12.y;
    // four elements per thread at a time: every load before any store, so
    // the loads are in flight together (the stores may alias them)
    constexpr int U = 4;
    for (long long l0 = b0 + threadIdx.x; l0 < e0; l0 += U * kPersistThreads) {
        float phi[U], m0[U], v0[U], t0[U];
#pragma unroll
        for (int u = 0; u < U; ++u) {
            const long long loc = l0 + u * kPersistThreads, t = s.elem0 + loc;
            const bool ok = loc < e0;
            phi[u] = ok ? s.part[loc] : 0.f;
            m0[u] = ok ? p.m[t] : 0.f;
            v0[u] = ok ? p.v[t] : 0.f;
            t0[u] = ok ? p.theta[t] : 0.f;
        }
#pragma unroll
        for (int u = 0; u < U; ++u) {
            const long long loc = l0 + u * kPersistThreads;
            if (loc < e0)
                for (int q = 1; q < s.shares; ++q) phi[u] += s.part[(size_t)q * ne + loc];
        }
#pragma unroll
        for (int u = 0; u < U; ++u) {
            const long long loc = l0 + u * kPersistThreads, t = s.elem0 + loc;
            if (loc >= e0) continue;
            const float gr = -phi[u];
            const float mt = 0.9f * m0[u] + 0.1f * gr;
            const float vt = 0.999f * v0[u] + 0.001f * gr * gr;
            const float th = t0[u] - p.lr * (mt / bc1) / (sqrtf(vt / bc2) + 1e-8f);
            p.m[t] = mt;
            p.v[t] = vt;
            p.theta[t] = th;
            if (!isfinite(th) || !isfinite(gr)) atomicOr(p.flag, 1);
        }
    }
}

__device__ __forceinline__ bool run_phi(const PersistArgs& p, const SvgdInst& s, int rblock,
                                        int share) {
    switch (p.dp) {
        case 3:
            return phi_body<3, kPersistWarps, 1>(s.theta, s.grad, s.N, s.D, s.d2, s.h, s.part,
                                              s.j_chunk, p.flag, rblock, share, nullptr,
                                              kWaitLimit, false, 0, s.N);
        case 6:
            return phi_body<6, kPersistWarps, 1>(s.theta, s.grad, s.N, s.D, s.d2, s.h, s.part,
                                              s.j_chunk, p.flag, rblock, share, nullptr,
                                              kWaitLimit, false, 0, s.N);
        default:
            return phi_body<9, kPersistWarps, 1>(s.theta, s.grad, s.N, s.D, s.d2, s.h, s.part,
                                              s.j_chunk, p.flag, rblock, share, nullptr,
                                              kWaitLimit, false, 0, s.N);
    }
}

__global__ void __launch_bounds__(kPersistThreads, 1)
    persist_kernel(const PersistArgs p, const SimConst c1, const SimConst c2, const SimConst c3,
                   const SimConst c4) {
    extern __shared__ __align__(128) float2 pdyn[];
    __shared__ int item_sh, stop_sh, last_sh;
    const int tid = threadIdx.x, warp = tid >> 5;
    const int e_roll = p.n_roll, e_pw = e_roll + p.n_pw, e_m1 = e_pw + p.n_med;
    const int e_m2 = e_m1 + p.n_med, e_phi = e_m2 + p.n_phi, e_all = e_phi + p.n_adam;
    for (;;) {
        if (tid == 0) {
            item_sh = (int)atomicAdd(p.ctr, 1u);
            stop_sh = (int)ld_acquire(p.ctr + 2);
        }
        __syncthreads();
        const int k = item_sh;
        const bool stop = stop_sh != 0;
        __syncthreads();
        if (k >= e_all) break;
        if (stop) continue;   // drain the queue after an abort
        unsigned long long t_claim = 0;
        if (p.trace && tid == 0) start_sh = t_claim = now_ns();
        if (k < e_roll) {
            // every warp's forward, then (the tapes visible CTA-wide) every
            // warp's adjoint: the SM's warps run one loop body at a time
            const int4 w = p.warps[(size_t)k * kPersistWarps + warp];
            const bool run = w.x >= 0 && p.active[w.x];
            float2* wseg = pdyn + (size_t)warp * p.seg_warp;
            for (int phase = 0; phase < 2; ++phase) {
                if (run) {
                    switch (w.z) {
                        case 1: roll_warp<1>(c1, p, w.x, w.y, wseg, phase); break;
                        case 2: roll_warp<2>(c2, p, w.x, w.y, wseg, phase); break;
                        case 3: roll_warp<3>(c3, p, w.x, w.y, wseg, phase); break;
                        default: roll_warp<4>(c4, p, w.x, w.y, wseg, phase); break;
                    }
                }
                __syncthreads();
            }
            if (run) {
                __threadfence();
                __syncwarp();
                if ((tid & 31) == 0) atomicAdd(p.dep + (size_t)kPersistDeps * w.x, 1u);
            }
        } else if (k < e_pw) {
            const int4 it = p.pw[k - e_roll];
            if (p.active[it.x]) {
                const SvgdInst& s = p.sinst[it.x];
                pairwise_strip_body<kPersistThreads>(s.theta, s.N, s.D, s.d2, s.hist, s.sel,
                                                     s.counter, s.h, it.y, it.z, it.w,
                                                     (unsigned)p.need[it.x].y);
                cta_signal(p.dep + (size_t)kPersistDeps * it.x + 1);
            }
        } else if (k < e_m2) {
            const int dg = k < e_m1 ? 1 : 2;
            const int2 it = p.med[k - (dg == 1 ? e_pw : e_m1)];
            const int g = it.x;
            if (p.active[g]) {
                const SvgdInst& s = p.sinst[g];
                unsigned* dep = p.dep + (size_t)kPersistDeps * g;
                const unsigned target = dg == 1 ? (unsigned)p.need[g].y : (unsigned)s.med_ctas;
                if (wait_counts(p, dep + dg, target, nullptr, 0u)) {
                    if (s.N >= 2)
                        median_digit_body<kPersistThreads>(s.N, dg, s.d2, s.hist, s.sel,
                                                           s.counter + dg, s.h, nullptr, it.y,
                                                           s.med_ctas);
                    cta_signal(dep + dg + 1);
                }
            }
        } else if (k < e_phi) {
            const int4 it = p.phi[k - e_m2];
            const int g = it.x;
            if (p.active[g]) {
                const SvgdInst& s = p.sinst[g];
                const int4 nd = p.need[g];
                unsigned* dep = p.dep + (size_t)kPersistDeps * g;
                if (wait_counts(p, dep + 3, (unsigned)nd.z, dep, (unsigned)(nd.x + p.extra_wait))) {
                    if (!run_phi(p, s, it.y, it.z) && tid == 0) atomicExch(p.ctr + 2, 1u);
                    cta_signal(dep + 4);
                }
            }
        } else {
            const int2 it = p.adam[k - e_phi];
            const int g = it.x;
            if (p.active[g]) {
                const SvgdInst& s = p.sinst[g];
                unsigned* dep = p.dep + (size_t)kPersistDeps * g;
                if (wait_counts(p, dep + 4, (unsigned)p.need[g].w, nullptr, 0u)) {
                    adam_chunk(p, s, it.y);
                    if (it.y == 0)   // the median passes are done: clear the histograms
                        for (int q = tid; q < kBins0 + kBins1 + kBins2; q += kPersistThreads)
                            s.hist[q] = 0u;
                }
            }
        }
        __syncthreads();   // shared memory is free for the next item
        if (p.trace && tid == 0 && k < p.trace_cap) {
            stamp_trace_entry& e = p.trace[k];
            e.claim_ns = t_claim;
            e.start_ns = start_sh;
            e.end_ns = now_ns();
            e.item = (unsigned)k;
            unsigned sm;
            asm volatile("mov.u32 %0, %%smid;" : "=r"(sm));
            e.sm = sm;
        }
    }
    // the last CTA out re-arms the queue and advances the iteration
    if (tid == 0) {
        __threadfence();
        last_sh = atomicAdd(p.ctr + 1, 1u) == gridDim.x - 1;
    }
    __syncthreads();
    if (last_sh) {
        __threadfence();
        for (int q = tid; q < kPersistDeps * p.n_inst; q += kPersistThreads) p.dep[q] = 0u;
        if (tid == 0) {
            p.ctr[0] = 0u;
            p.ctr[1] = 0u;
            p.ctr[2] = 0u;
            ++*p.iter;
            ++*p.step;
        }
    }
}

}  // namespace

size_t persist_smem(int max_D, int seg_warp) {
    const int dp = persist_dp(max_D);
    const size_t phi = (size_t)4 * phi_stage_floats(max_D, dp) * sizeof(float) +
                       (size_t)kPersistWarps * kTJ * sizeof(float4) + 2 * sizeof(uint64_t);
    const size_t pw = 2 * kTile * (size_t)(max_D + 1) * sizeof(float);
    const size_t seg = (size_t)kPersistWarps * seg_warp * sizeof(float2);
    size_t m = phi > pw ? phi : pw;
    return m > seg ? m : seg;
}

cudaError_t persist_grid(size_t smem, int* grid) {
    cudaError_t e = cudaFuncSetAttribute(persist_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)smem);
    if (e != cudaSuccess) return e;
    int per_sm = 0;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, persist_kernel, kPersistThreads, smem);
    if (e != cudaSuccess) return e;
    if (per_sm < 1) return cudaErrorInvalidConfiguration;
    *grid = per_sm * sm_count();
    return cudaSuccess;
}

cudaError_t launch_persist(const PersistArgs& p, const SimConst* cls, int grid, size_t smem,
                           cudaStream_t st) {
    persist_kernel<<<grid, kPersistThreads, smem, st>>>(p, cls[0], cls[1], cls[2], cls[3]);
    return cudaGetLastError();
}

}  // namespace stamp
