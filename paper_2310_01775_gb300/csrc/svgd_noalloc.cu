// Stein step for callers that cannot allocate device memory.
//
// stamp_svgd_step needs a stamp_problem, and creating one calls cudaMalloc.
// Some callers cannot: code running where the allocator is owned by someone
// else (a framework's caching allocator or a memory pool that must not be
// bypassed), inside a region where allocation is forbidden (between
// allocation-free checkpoints of a long job), or on a device whose memory is
// already fully reserved.  stamp_svgd_step_noalloc runs the same kernels with
// their scratch memory (pairwise distances, Stein direction, radix-select
// histograms and selections, last-CTA counters, bandwidth, error flags) in
// one file-scope device array below, reserved when the library is loaded on
// a device and held there until the process exits.
#include <cmath>
#include <cstdint>
#include <cstring>
#include <mutex>

#include "stamp.h"
#include "stamp_internal.cuh"

namespace {

constexpr int kMaxN = STAMP_NOALLOC_MAX_N;
constexpr int kMaxD = STAMP_NOALLOC_MAX_D;

constexpr size_t align256(size_t b) { return (b + 255) / 256 * 256; }
// Layout of the scratch array (each part 256-byte aligned).
constexpr size_t kOffD2 = 0;
constexpr size_t kOffPhi = kOffD2 + align256((size_t)kMaxN * kMaxN * sizeof(float));
constexpr size_t kOffHist = kOffPhi + align256((size_t)kMaxN * kMaxD * sizeof(float));
constexpr size_t kOffSel = kOffHist + align256((2048 + 2048 + 1024) * sizeof(unsigned));
constexpr size_t kOffCounter = kOffSel + 256;
constexpr size_t kOffH = kOffCounter + 256;
constexpr size_t kOffFlag = kOffH + 256;
constexpr size_t kScratchBytes = kOffFlag + 256;

// The scratch: one array per device that loads this library (about 5.4 MB).
// In host code `g_noalloc_scratch` is a host-side stand-in, not a device
// address: kernels get the address that cudaGetSymbolAddress returns.
static __device__ __align__(256) unsigned char g_noalloc_scratch[kScratchBytes];
// h of the SGD phase; initialised with the module, never written.
static __device__ __align__(16) float g_noalloc_one = 1.f;

constexpr int kMaxDevices = 64;
std::mutex g_mu;
struct Bases {
    unsigned char* scratch;
    const float* one;
};
Bases g_base[kMaxDevices] = {};

// Report through stamp_last_error(), like every other call of the library.
stamp_status noalloc_fail(stamp_status s, const char* msg, cudaError_t e = cudaSuccess) {
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

// Device addresses of the scratch and of the constant 1 on the current
// device: looked up (cudaGetSymbolAddress, with that device current) on the
// first call per device and kept for the life of the process.
stamp_status scratch_base(Bases* out) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return noalloc_fail(STAMP_ECUDA, "cudaGetDevice failed", e);
    if (dev < 0 || dev >= kMaxDevices) return noalloc_fail(STAMP_EINVAL, "device index too large");
    std::lock_guard<std::mutex> lock(g_mu);
    if (!g_base[dev].scratch) {
        void* p = nullptr;
        void* one = nullptr;
        e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e == cudaSuccess) e = cudaGetSymbolAddress(&one, g_noalloc_one);
        if (e != cudaSuccess) return noalloc_fail(STAMP_ECUDA, "cudaGetSymbolAddress failed", e);
        g_base[dev] = Bases{static_cast<unsigned char*>(p), static_cast<const float*>(one)};
    }
    *out = g_base[dev];
    return STAMP_OK;
}

}  // namespace

extern "C" stamp_status stamp_svgd_step_noalloc(float* theta, const float* grad_logp, int N, int D,
                                                float* adam_m, float* adam_v, int step, float lr,
                                                int sgd_phase, float* h_out, float* phi_out,
                                                void* cuda_stream) {
    if (N < 1 || N > kMaxN)
        return noalloc_fail(STAMP_EINVAL, "N outside [1, STAMP_NOALLOC_MAX_N]");
    if (D < 1 || D > kMaxD)
        return noalloc_fail(STAMP_EINVAL, "D outside [1, STAMP_NOALLOC_MAX_D]");
    if (step < 1 || !std::isfinite(lr)) return noalloc_fail(STAMP_EINVAL, "need step >= 1, finite lr");
    if (!theta || !grad_logp || !adam_m || !adam_v)
        return noalloc_fail(STAMP_EINVAL, "NULL theta, grad_logp or Adam moments");
    if (!on_device(theta) || !on_device(grad_logp) || !on_device(adam_m) || !on_device(adam_v) ||
        (h_out && !on_device(h_out)) || (phi_out && !on_device(phi_out)))
        return noalloc_fail(STAMP_EINVAL, "a pointer is not device memory");
    if ((reinterpret_cast<uintptr_t>(theta) | reinterpret_cast<uintptr_t>(grad_logp)) & 15u)
        return noalloc_fail(STAMP_EINVAL, "theta and grad_logp must be 16-byte aligned");
    Bases bases{};
    stamp_status st = scratch_base(&bases);
    if (st != STAMP_OK) return st;
    unsigned char* base = bases.scratch;
    cudaStream_t s = static_cast<cudaStream_t>(cuda_stream);
    stamp::SvgdScratch sc{reinterpret_cast<float*>(base + kOffD2),
                          reinterpret_cast<unsigned*>(base + kOffHist),
                          reinterpret_cast<unsigned*>(base + kOffSel),
                          reinterpret_cast<unsigned*>(base + kOffCounter),
                          reinterpret_cast<float*>(base + kOffH),
                          reinterpret_cast<int*>(base + kOffFlag)};
    // the array keeps the last call's contents: clear what must start at zero
    cudaError_t e = cudaMemsetAsync(base + kOffHist, 0, kOffSel - kOffHist, s);
    if (e == cudaSuccess) e = cudaMemsetAsync(base + kOffCounter, 0, 256, s);
    if (e == cudaSuccess) e = cudaMemsetAsync(base + kOffFlag, 0, sizeof(int), s);
    if (e != cudaSuccess) return noalloc_fail(STAMP_ECUDA, "clearing the scratch failed", e);
    const float* part = grad_logp;   // SGD phase: phi = grad log rho
    int shares = 1;
    const float* h_src = bases.one;
    if (!sgd_phase) {
        float* phi = reinterpret_cast<float*>(base + kOffPhi);   // room for one share
        e = stamp::launch_pairwise(theta, N, D, sc, s);
        for (int dg = 1; dg <= 2 && e == cudaSuccess && N >= 2; ++dg)
            e = stamp::launch_median_digit(N, dg, sc, nullptr, s);
        if (e == cudaSuccess) e = stamp::launch_phi(theta, grad_logp, N, D, sc, phi, 1, &shares, s);
        if (e != cudaSuccess) return noalloc_fail(STAMP_ECUDA, "Stein direction launch failed", e);
        part = phi;
        h_src = sc.h;
    }
    if (h_out) {
        e = cudaMemcpyAsync(h_out, h_src, sizeof(float), cudaMemcpyDeviceToDevice, s);
        if (e != cudaSuccess) return noalloc_fail(STAMP_ECUDA, "copy of h failed", e);
    }
    e = stamp::launch_adam(theta, part, shares, phi_out, adam_m, adam_v, N * D, step, lr, sc.err, s);
    if (e != cudaSuccess) return noalloc_fail(STAMP_ECUDA, "Adam launch failed", e);
    int flag = 0;
    e = cudaMemcpyAsync(&flag, sc.err, sizeof flag, cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return noalloc_fail(STAMP_ECUDA, "stream synchronisation failed", e);
    if (flag & 2) return noalloc_fail(STAMP_ETIMEOUT, "a bounded device wait gave up");
    if (flag & 1) return noalloc_fail(STAMP_ENONFINITE, "a non-finite particle or Stein direction");
    return STAMP_OK;
}
