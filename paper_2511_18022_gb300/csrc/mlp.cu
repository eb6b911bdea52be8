// Surrogate network for screening local-search neighbours: training and
// inference kernels. BF16 weights, per-position features as BF16 hi + lo
// pairs (about 16 significant bits), FP32 activations and accumulation.
// The products of layers 1 and 2, forward and backward, run on the tensor
// cores (mlp_tc.cu); this file holds the rest: the output layer, the loss,
// the layer-2 bias gradient and Adam.
//
// Architecture (width H = 256):
//   per position k of a tour:  phi_k = (x, y, mu / Q, sd / Q, frac(cum_k / Q))
//                              (coordinates / 1000; cum_k = expected load of
//                               positions 1..k along the tour)
//   layer 1 (per position):    h_k = relu(W1 phi_k + b1)            H x 5
//   pooling:                   z = mean_k h_k
//   tour-length feature:       t = (c(0,s_1) + D[n] + c(s_n,0) - m) / sd, with (m, sd)
//                              set by the caller (default m = 0, sd = 500 n)
//   layer 2:                   u = relu(W2 [z; t] + b2)              H x (H+1)
//   layer 3:                   y = w3 . u + b3
// Parameters are one fp32 vector (layout in mlp.h); the kernels read bf16
// copies of the weight matrices. The backward pass recomputes layer 1 from the
// tour instead of storing an activation per position.
#include <cuda_bf16.h>
#include <stdint.h>

#include "mlp.h"

namespace cvrpsd {

// ---------------------------------------------------------------- layer 3, loss

// y[b] = w3 . u_b + b3; with targets: dy = 2 (y - target) / B, loss partials.
__global__ void mlp_out_kernel(const float *U, int B, const __nv_bfloat16 *w3, const __nv_bfloat16 *b3, float *y,
                               const float *target, float *dy, float *loss)
{
    const int lane = threadIdx.x & 31;
    const int b = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    if (b >= B) return;
    float s = 0.0f;
    for (int j = lane; j < kMlpH; j += 32) s += U[(long long)b * kMlpH + j] * __bfloat162float(w3[j]);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if (lane == 0) {
        const float v = s + __bfloat162float(b3[0]);
        y[b] = v;
        if (target) {
            const float e = v - target[b];
            dy[b] = 2.0f * e / (float)B;
            atomicAdd(loss, e * e / (float)B);
        }
    }
}

// dU[b][j] = dy_b w3_j [u_bj > 0]; g_w3[j] += sum_b dy_b u_bj; g_b3 += sum_b dy_b
__global__ void mlp_out_backward_kernel(const float *U, int B, const float *dy, const __nv_bfloat16 *w3, float *dU,
                                        float *gw3, float *gb3)
{
    const int j = threadIdx.x;                // kMlpH threads
    float acc = 0.0f, accb = 0.0f;
    const float wj = __bfloat162float(w3[j]);
    for (int b = blockIdx.x; b < B; b += gridDim.x) {
        const float u = U[(long long)b * kMlpH + j];
        const float d = dy[b];
        acc += d * u;
        accb += d;
        dU[(long long)b * kMlpH + j] = u > 0.0f ? d * wj : 0.0f;
    }
    atomicAdd(gw3 + j, acc);
    if (j == 0) atomicAdd(gb3, accb);
}

// g_b2[j] += sum_b dU[b][j]: blocks take 64-row slabs, one atomic per column
// and slab.
__global__ void colsum_kernel(const float *G, int B, int N, int ldg, float *out)
{
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= N) return;
    const int b0 = blockIdx.y * 64, b1 = min(B, b0 + 64);
    float s = 0.0f;
    for (int b = b0; b < b1; ++b) s += G[(long long)b * ldg + j];
    atomicAdd(out + j, s);
}

// ---------------------------------------------------------------- Adam

__global__ void adam_kernel(float *p, const float *g, float *m, float *v, long long P, float lr, float b1, float b2,
                            float eps, float c1, float c2)
{
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < P; i += (long long)gridDim.x * blockDim.x) {
        const float gi = g[i];
        const float mi = b1 * m[i] + (1.0f - b1) * gi;
        const float vi = b2 * v[i] + (1.0f - b2) * gi * gi;
        m[i] = mi;
        v[i] = vi;
        p[i] -= lr * (mi / c1) / (sqrtf(vi / c2) + eps);
    }
}

__global__ void to_bf16_kernel(const float *p, __nv_bfloat16 *q, long long P)
{
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < P; i += (long long)gridDim.x * blockDim.x)
        q[i] = __float2bfloat16_rn(p[i]);
}

// ---------------------------------------------------------------- host launchers


cudaError_t mlp_forward(const MlpLayer1Args &l1, const MlpWeights &wt, float *U, float *y, const float *target,
                        float *dy, float *loss, cudaStream_t st)
{
    const int T = l1.T;
    cudaError_t e = mlp_layer1_tc(l1, l1.sm_count > 0 ? l1.sm_count : 1, st);
    if (e != cudaSuccess) return e;
    e = mlp_layer2_tc(l1.zt, T, wt.w2, wt.b2, U, l1.err, st);
    if (e != cudaSuccess) return e;
    mlp_out_kernel<<<(T + 7) / 8, 256, 0, st>>>(U, T, wt.w3, wt.b3, y, target, dy, loss);
    return cudaGetLastError();
}

cudaError_t mlp_backward(const MlpLayer1Args &l1, const MlpWeights &wt, const float *U, const float *dy, float *dU,
                         float *dzt, float *grad, cudaStream_t st)
{
    const int T = l1.T;
    float *gw1 = grad + kOffW1, *gb1 = grad + kOffB1, *gw2 = grad + kOffW2, *gb2 = grad + kOffB2;
    float *gw3 = grad + kOffW3, *gb3 = grad + kOffB3;
    mlp_out_backward_kernel<<<T < 512 ? T : 512, kMlpH, 0, st>>>(U, T, dy, wt.w3, dU, gw3, gb3);
    cudaError_t e = mlp_grad_w2_tc(dU, l1.zt, T, gw2, l1.err, st);
    if (e != cudaSuccess) return e;
    colsum_kernel<<<dim3(1, (unsigned)((T + 63) / 64)), kMlpH, 0, st>>>(dU, T, kMlpH, kMlpH, gb2);
    e = mlp_grad_zt_tc(dU, T, wt.w2, dzt, l1.err, st);
    if (e != cudaSuccess) return e;
    MlpLayer1Args b = l1;
    b.dzt = dzt;
    b.gw1 = gw1;
    b.gb1 = gb1;
    e = mlp_layer1_bwd_tc(b, l1.sm_count > 0 ? l1.sm_count : 1, st);
    if (e != cudaSuccess) return e;
    return cudaGetLastError();
}

cudaError_t mlp_adam(float *p, const float *g, float *m, float *v, __nv_bfloat16 *pb, float lr, int step,
                     cudaStream_t st)
{
    const float b1 = 0.9f, b2 = 0.999f, eps = 1e-8f;
    const float c1 = 1.0f - powf(b1, (float)step), c2 = 1.0f - powf(b2, (float)step);
    adam_kernel<<<128, 256, 0, st>>>(p, g, m, v, kMlpParams, lr, b1, b2, eps, c1, c2);
    to_bf16_kernel<<<128, 256, 0, st>>>(p, pb, kMlpParams);
    return cudaGetLastError();
}

cudaError_t mlp_to_bf16(const float *p, __nv_bfloat16 *pb, cudaStream_t st)
{
    to_bf16_kernel<<<128, 256, 0, st>>>(p, pb, kMlpParams);
    return cudaGetLastError();
}

}  // namespace cvrpsd
