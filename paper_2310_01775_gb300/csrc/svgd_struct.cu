// Stein direction with the structured kernel of App. D.3, restated for plans
// of [logits a_k, offset parameter u_k, distance parameter v_k] per action:
//   K(a, b) = (1/2H) sum_k [ exp(-|c_k(a) - c_k(b)|^2 / h_c)
//                            + exp(-|softmax(a_k) - softmax(b_k)|^2 / h_z) ],
// c_k = (u_k, v_k), K(a, a) = 1.  (The paper's kernel is defined on DMP goal
// poses: RBF on goal positions, RBF on softmax(a_k), von Mises on goal yaws;
// these plans have push parameters where it has goal positions and no angle.)
// phi_i = sum_j wn_j [K_ji grad log rho_j + grad_{theta_j} K_ji], wn_j = 1/N or
// the normalised weights of Eq. dsvgd, with
//   grad_{u,v of action k} K_ji = (1/2H)(2/h_c) e^c_ijk (c_ik - c_jk),
//   grad_{a_jk} K_ji          = (1/2H)(2/h_z) e^z_ijk J(a_jk)^T (s_ik - s_jk),
//   J^T x = s (x - s.x)  (softmax Jacobian, symmetric).
// h_c, h_z: the median heuristic on the concatenated component (pairwise
// distances and radix-select median of svgd.cu) divided by H.
#include <cstdint>

#include "stamp_internal.cuh"

namespace stamp {
namespace {

constexpr int kRows = 8;        // rows i per CTA (one warp each)
constexpr int kTJ = 16;         // j per tile
constexpr int kMaxHs = 16;      // actions per plan

// C (N x 2H): (u_k, v_k); S (N x M H): softmax(a_k).
__global__ void struct_prep_kernel(const float* __restrict__ theta, int N, int H, int M,
                                   float* __restrict__ C, float* __restrict__ S) {
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= N * H) return;
    const int i = t / H, k = t % H, P = M + 2;
    const float* a = theta + (size_t)i * H * P + k * P;
    float mx = a[0];
    for (int c = 1; c < M; ++c) mx = fmaxf(mx, a[c]);
    float sum = 0.f;
    float* s = S + (size_t)i * M * H + k * M;
    for (int c = 0; c < M; ++c) {
        const float e = expf(a[c] - mx);
        s[c] = e;
        sum += e;
    }
    const float inv = 1.f / sum;
    for (int c = 0; c < M; ++c) s[c] *= inv;
    C[(size_t)i * 2 * H + 2 * k] = a[M];
    C[(size_t)i * 2 * H + 2 * k + 1] = a[M + 1];
}

template <int DP>
__global__ void __launch_bounds__(kRows * 32)
struct_phi_kernel(const float* __restrict__ theta, const float* __restrict__ grad,
                  const float* __restrict__ C, const float* __restrict__ S, int N, int H, int M,
                  const float* __restrict__ hc_dev, const float* __restrict__ hz_dev,
                  const float* __restrict__ wn, float* __restrict__ phi, int j_chunk) {
    __shared__ float Ec[kRows][kTJ][kMaxHs + 1], Ez[kRows][kTJ][kMaxHs + 1], Q[kRows][kTJ][kMaxHs + 1];
    __shared__ float Ks[kRows][kTJ];
    const int P = M + 2, D = H * P;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int i0 = blockIdx.x * kRows, i = i0 + warp;
    const float Hf = (float)H;
    const float inv_hc = Hf / __ldg(hc_dev), inv_hz = Hf / __ldg(hz_dev);   // h = h_plain / H
    const float alpha = 0.5f / Hf;
    float ti[DP], si[DP], acc[DP];   // theta_i and, on logit slots, softmax(a_ik)
#pragma unroll
    for (int q = 0; q < DP; ++q) {
        const int d = lane + 32 * q;
        const bool ok = i < N && d < D;
        ti[q] = ok ? theta[(size_t)i * D + d] : 0.f;
        si[q] = (ok && d % P < M) ? S[(size_t)i * M * H + (d / P) * M + d % P] : 0.f;
        acc[q] = 0.f;
    }
    // this CTA's share of the sum over j; partial directions go to share blockIdx.y
    const int jb = blockIdx.y * j_chunk, je = min(N, jb + j_chunk);
    phi += (size_t)blockIdx.y * N * D;
    for (int j0 = jb; j0 < je; j0 += kTJ) {
        const int nj = min(kTJ, je - j0);
        // per (row, j, action): e^c, e^z and s_j.(s_i - s_j)
        for (int e = tid; e < kRows * kTJ * H; e += kRows * 32) {
            const int r = e / (kTJ * H), jj = (e / H) % kTJ, k = e % H;
            const int ii = i0 + r, j = j0 + jj;
            float ec = 0.f, ez = 0.f, q = 0.f;
            if (ii < N && jj < nj) {
                const float* ci = C + (size_t)ii * 2 * H + 2 * k;
                const float* cj = C + (size_t)j * 2 * H + 2 * k;
                const float du = __ldg(ci) - __ldg(cj), dv = __ldg(ci + 1) - __ldg(cj + 1);
                ec = expf(-(du * du + dv * dv) * inv_hc);
                const float* s_i = S + (size_t)ii * M * H + k * M;
                const float* s_j = S + (size_t)j * M * H + k * M;
                float dz = 0.f;
                for (int c = 0; c < M; ++c) {
                    const float a = __ldg(s_i + c), b = __ldg(s_j + c), x = a - b;
                    dz = fmaf(x, x, dz);
                    q = fmaf(b, x, q);
                }
                ez = expf(-dz * inv_hz);
            }
            Ec[r][jj][k] = ec;
            Ez[r][jj][k] = ez;
            Q[r][jj][k] = q;
        }
        __syncthreads();
        if (tid < kRows * kTJ) {   // K_ij = alpha sum_k (e^c + e^z), times wn_j (or 1; 1/N at the end)
            const int r = tid / kTJ, jj = tid % kTJ;
            float ksum = 0.f;
            for (int k = 0; k < H; ++k) ksum += Ec[r][jj][k] + Ez[r][jj][k];
            const float w = (jj < nj && wn) ? wn[j0 + jj] : 1.f;
            Ks[r][jj] = jj < nj ? alpha * ksum * w : 0.f;
        }
        __syncthreads();
        if (i < N) {
            for (int jj = 0; jj < nj; ++jj) {
                const int j = j0 + jj;
                const float kij = Ks[warp][jj];
                const float w = wn ? wn[j] : 1.f;
#pragma unroll
                for (int q = 0; q < DP; ++q) {
                    const int d = lane + 32 * q;
                    if (d >= D) continue;
                    const int k = d / P, comp = d % P;
                    const float gj = __ldg(grad + (size_t)j * D + d);
                    float rep;
                    if (comp < M) {
                        const float sj = __ldg(S + (size_t)j * M * H + k * M + comp);
                        rep = 2.f * inv_hz * Ez[warp][jj][k] * sj * ((si[q] - sj) - Q[warp][jj][k]);
                    } else {
                        rep = 2.f * inv_hc * Ec[warp][jj][k] * (ti[q] - __ldg(theta + (size_t)j * D + d));
                    }
                    acc[q] = fmaf(kij, gj, fmaf(alpha * w, rep, acc[q]));
                }
            }
        }
        __syncthreads();
    }
    const float scale = wn ? 1.f : 1.f / (float)N;
    if (i < N)
#pragma unroll
        for (int q = 0; q < DP; ++q) {
            const int d = lane + 32 * q;
            if (d < D) phi[(size_t)i * D + d] = acc[q] * scale;
        }
}

__global__ void scale_scalar_kernel(const float* src, float s, float* dst) { *dst = *src * s; }

}  // namespace

cudaError_t launch_scale_scalar(const float* src, float s, float* dst, cudaStream_t st) {
    scale_scalar_kernel<<<1, 1, 0, st>>>(src, s, dst);
    return cudaGetLastError();
}

cudaError_t launch_struct_prep(const float* theta, int N, int H, int M, float* C, float* S,
                               cudaStream_t st) {
    struct_prep_kernel<<<(N * H + 127) / 128, 128, 0, st>>>(theta, N, H, M, C, S);
    return cudaGetLastError();
}

cudaError_t launch_struct_phi(const float* theta, const float* grad, const float* C, const float* S,
                              int N, int H, int M, const float* hc_dev, const float* hz_dev,
                              const float* wn, float* phi, int max_shares, int* shares,
                              cudaStream_t st) {
    if (H > kMaxHs) return cudaErrorInvalidValue;
    const int D = H * (M + 2), rows = (N + kRows - 1) / kRows;
    // split the sum over j so that about four CTAs per SM are in flight
    int want = (4 * sm_count() + rows - 1) / rows;
    want = want < 1 ? 1 : (want > max_shares ? max_shares : want);
    const int j_chunk = ((N + want - 1) / want + kTJ - 1) / kTJ * kTJ;
    *shares = (N + j_chunk - 1) / j_chunk;
    const dim3 grid(rows, *shares);
    switch ((D + 31) / 32) {
        case 1: struct_phi_kernel<1><<<grid, kRows * 32, 0, st>>>(theta, grad, C, S, N, H, M, hc_dev, hz_dev, wn, phi, j_chunk); break;
        case 2: struct_phi_kernel<2><<<grid, kRows * 32, 0, st>>>(theta, grad, C, S, N, H, M, hc_dev, hz_dev, wn, phi, j_chunk); break;
        case 3: struct_phi_kernel<3><<<grid, kRows * 32, 0, st>>>(theta, grad, C, S, N, H, M, hc_dev, hz_dev, wn, phi, j_chunk); break;
        case 4: struct_phi_kernel<4><<<grid, kRows * 32, 0, st>>>(theta, grad, C, S, N, H, M, hc_dev, hz_dev, wn, phi, j_chunk); break;
        case 5: case 6: struct_phi_kernel<6><<<grid, kRows * 32, 0, st>>>(theta, grad, C, S, N, H, M, hc_dev, hz_dev, wn, phi, j_chunk); break;
        case 7: case 8: case 9: struct_phi_kernel<9><<<grid, kRows * 32, 0, st>>>(theta, grad, C, S, N, H, M, hc_dev, hz_dev, wn, phi, j_chunk); break;
        default: return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

}  // namespace stamp
