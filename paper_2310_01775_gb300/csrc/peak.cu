// FP32 fused-multiply-add throughput of the device: the roof of the
// ALU-bound rollout and reverse-sweep kernels.  Every thread runs kChains
// independent FMA chains (no chain waits on another, so issue latency never
// starves the FMA pipes), the grid fills every SM to full occupancy, and the
// chains' results feed a store that never happens but that the compiler
// cannot remove.
#include <algorithm>
#include <vector>

#include "stamp.h"
#include "stamp_internal.cuh"

namespace {

constexpr int kChains = 8;     // independent chains per thread
constexpr int kUnroll = 16;    // FMAs per chain per loop trip
constexpr int kThreads = 256;
constexpr int kCtasPerSm = 8;  // 2048 threads per SM

__global__ void __launch_bounds__(kThreads) fma_peak_kernel(float a, float b, int trips,
                                                            float* sink) {
    float x[kChains];
#pragma unroll
    for (int c = 0; c < kChains; ++c) x[c] = (float)(threadIdx.x + c) * 1e-3f;
    for (int t = 0; t < trips; ++t) {
#pragma unroll
        for (int u = 0; u < kUnroll; ++u)
#pragma unroll
            for (int c = 0; c < kChains; ++c) x[c] = fmaf(x[c], a, b);
    }
    float s = 0.f;
#pragma unroll
    for (int c = 0; c < kChains; ++c) s += x[c];
    if (s == -1.f) sink[blockIdx.x * blockDim.x + threadIdx.x] = s;   // never true for a, b > 0
}

}  // namespace

extern "C" stamp_status stamp_fp32_fma_peak(int launches, double* tflops_out,
                                            double* ms_per_launch_out) {
    if (launches < 1 || !tflops_out) {
        stamp::set_last_error("need launches >= 1 and tflops_out");
        return STAMP_EINVAL;
    }
    const int grid = stamp::sm_count() * kCtasPerSm;
    const int trips = 1024;
    float* sink = nullptr;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    cudaStream_t st = nullptr;
    std::vector<float> ms;
    cudaError_t e = cudaMalloc(&sink, sizeof(float) * grid * kThreads);
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaEventCreate(&e0);
    if (e == cudaSuccess) e = cudaEventCreate(&e1);
    for (int l = -2; l < launches && e == cudaSuccess; ++l) {   // two launches warm up
        e = cudaEventRecord(e0, st);
        if (e == cudaSuccess) {
            fma_peak_kernel<<<grid, kThreads, 0, st>>>(0.999999f, 1e-7f, trips, sink);
            e = cudaGetLastError();
        }
        if (e == cudaSuccess) e = cudaEventRecord(e1, st);
        if (e == cudaSuccess) e = cudaEventSynchronize(e1);
        float t = 0.f;
        if (e == cudaSuccess) e = cudaEventElapsedTime(&t, e0, e1);
        if (e == cudaSuccess && l >= 0) ms.push_back(t);
    }
    if (e1) cudaEventDestroy(e1);
    if (e0) cudaEventDestroy(e0);
    if (st) cudaStreamDestroy(st);
    if (sink) cudaFree(sink);
    if (e != cudaSuccess) {
        cudaGetLastError();
        stamp::set_last_error(cudaGetErrorString(e));
        return STAMP_ECUDA;
    }
    std::sort(ms.begin(), ms.end());
    const double med = ms[ms.size() / 2];
    const double flop = 2.0 * grid * kThreads * (double)trips * kUnroll * kChains;
    *tflops_out = flop / (med * 1e-3) / 1e12;
    if (ms_per_launch_out) *ms_per_launch_out = med;
    return STAMP_OK;
}
