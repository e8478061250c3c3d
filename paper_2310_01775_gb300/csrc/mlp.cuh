// Sizes and packed layouts of the BF16 tensor-core MLP (mlp.cu).
#pragma once

#include <cstddef>
#include <cuda_bf16.h>
#include <cuda_runtime.h>

namespace stamp {
namespace mlp {

constexpr int kIn = 32;        // padded input width (K of layer 0)
constexpr int kHidden = 256;   // hidden width
constexpr int kOut = 16;       // padded output width (N of layer 3)
constexpr int kLayers = 4;

// Byte offset of layer l's packed BF16 weights (N_l x K_l) in the weight tiles.
__host__ __device__ constexpr size_t layer_w_offset(int l) {
    return l == 0 ? 0
         : l == 1 ? (size_t)kHidden * kIn * 2
         : l == 2 ? (size_t)kHidden * kIn * 2 + (size_t)kHidden * kHidden * 2
                  : (size_t)kHidden * kIn * 2 + 2 * (size_t)kHidden * kHidden * 2;
}
constexpr size_t kWeightBytes = layer_w_offset(3) + (size_t)kOut * kHidden * 2;

// Float offset of layer l's (W_l, b_l) in the packed FP32 parameter vector:
// W_l is (out_l, in_l) row-major with the real sizes, then b_l (out_l).
__host__ __device__ constexpr size_t param_offset(int l, int in_dim, int out_dim) {
    return l == 0 ? 0
         : l == 1 ? (size_t)kHidden * in_dim + kHidden
         : l == 2 ? (size_t)kHidden * in_dim + kHidden + (size_t)kHidden * kHidden + kHidden
                  : (size_t)kHidden * in_dim + kHidden + 2 * ((size_t)kHidden * kHidden + kHidden);
}
__host__ __device__ constexpr size_t param_count(int in_dim, int out_dim) {
    return param_offset(3, in_dim, out_dim) + (size_t)out_dim * kHidden + out_dim;
}

size_t fwd_smem_bytes();
// W_l -> BF16 K-major tiles for the forward (N = out, K = in) and for the
// input-gradient backward (W_l^T: N = in, K = out), plus FP32 biases.
cudaError_t pack_weights(const float* params, int in_dim, int out_dim, unsigned char* w_tiled,
                         unsigned char* wt_tiled, float* bias, cudaStream_t st);
// y (rows x out_dim FP32) = MLP(x (rows x in_dim FP32)).  x_tiled: input
// tiles (8 KB each, written at tile_base); ypad: rows x 16 FP32 scratch.
// saved / zsave (NULL or buffers of tile_cap 64 KB tiles per layer) receive
// the activations for the backward pass at tiles tile_base...
cudaError_t forward(const float* x, int rows, int in_dim, int out_dim, const unsigned char* w_tiled,
                    const float* bias, unsigned char* x_tiled, float* ypad, float* y,
                    unsigned char* saved, unsigned char* zsave, int tile_base, int tile_cap,
                    int* err, int sm_count, cudaStream_t st);
// dx (rows x in_dim, or NULL) from dy (rows x out_dim) for the forward saved at tile_base;
// dz of every layer goes to dzsave.
cudaError_t backward(const float* dy, int rows, int in_dim, int out_dim,
                     const unsigned char* wt_tiled, const unsigned char* zsave,
                     unsigned char* dzsave, int tile_base, int tile_cap, float* dx, int* err,
                     int sm_count, cudaStream_t st);
// grad (packed like the parameters) += dL/dW_l, dL/db_l, on the tensor
// cores (BF16 operands, FP32 accumulation in TMEM), reduced over row splits
// in a fixed order; part: dw_part_floats() floats of scratch; err: bit 2 if
// a bounded wait gave up.
size_t dw_part_floats();
cudaError_t weight_grads(const unsigned char* x_tiled, const unsigned char* saved,
                         const unsigned char* dzsave, int tile_base, int tile_cap, int rows,
                         int in_dim, int out_dim, float* grad, float* part, int* err, int sm_count,
                         cudaStream_t st);
cudaError_t mse(const float* y, const float* t, int n, float* dy, float* loss, cudaStream_t st);
cudaError_t adam(float* p, const float* g, float* m, float* v, int n, int step, float lr,
                 cudaStream_t st);

}  // namespace mlp
}  // namespace stamp
