// Internal interface of the surrogate network kernels (mlp.cu).
#pragma once

#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <stdint.h>

namespace cvrpsd {

constexpr int kMlpH = 256;                 // hidden width
constexpr int kMlpIn1 = 5;                 // per-position features
constexpr int kMlpIn2 = kMlpH + 1;         // pooled features + tour length

// Offsets into the flat parameter vector: W1 [H][5], b1 [H], W2 [H][H+1],
// b2 [H], w3 [H], b3 [1].
constexpr long long kOffW1 = 0;
constexpr long long kOffB1 = kOffW1 + (long long)kMlpH * kMlpIn1;
constexpr long long kOffW2 = kOffB1 + kMlpH;
constexpr long long kOffB2 = kOffW2 + (long long)kMlpH * kMlpIn2;
constexpr long long kOffW3 = kOffB2 + kMlpH;
constexpr long long kOffB3 = kOffW3 + kMlpH;
constexpr long long kMlpParams = kOffB3 + 1;

struct MlpWeights {                        // bf16 views into one vector
    const __nv_bfloat16 *w1, *b1, *w2, *b2, *w3, *b3;
};

struct MlpLayer1Args {
    const int32_t *tours;                  // device [T][n]
    int T, n;
    const float *cust;                     // device [n][4]: x/1000, y/1000, mu/Q, sd/Q of customer k at k-1
    const int32_t *dist;                   // device (n+1)^2
    const __nv_bfloat16 *w1, *b1;
    float len_mean, len_inv_sd;            // tour-length feature t = (length - len_mean) * len_inv_sd
    float *zt;                             // device [T][H+1]: pooled features and tour length
    const float *dzt;                      // backward: gradient of zt
    float *gw1, *gb1;                      // backward: accumulated gradients
    unsigned int *err;                     // device word: set if a tensor-core wait gave up
    int sm_count;                          // SMs of the device (grid of the tensor-core kernel)
};

// Layer 1 forward (features, W1, ReLU, mean pool; writes zt) on the tensor
// cores: tcgen05 MMAs with the accumulators in tensor memory (mlp_tc.cu).
cudaError_t mlp_layer1_tc(const MlpLayer1Args &l1, int sm_count, cudaStream_t st);
// Layer 1 backward (dW1, db1 from dzt) on the tensor cores (mlp_tc.cu).
cudaError_t mlp_layer1_bwd_tc(const MlpLayer1Args &l1, int sm_count, cudaStream_t st);
// Layer 2 forward, U = relu(zt W2^T + b2), on the tensor cores (mlp_tc.cu).
cudaError_t mlp_layer2_tc(const float *zt, int T, const __nv_bfloat16 *w2, const __nv_bfloat16 *b2, float *U,
                          unsigned int *err, cudaStream_t st);

// Backward products on the tensor cores (mlp_tc.cu): dZT = dU W2 and
// gW2 += dU^T ZT (FP32 operands as BF16 hi/lo pairs, FP32 accumulation).
cudaError_t mlp_grad_zt_tc(const float *dU, int T, const __nv_bfloat16 *w2, float *dzt, unsigned int *err,
                           cudaStream_t st);
cudaError_t mlp_grad_w2_tc(const float *dU, const float *zt, int T, float *gw2, unsigned int *err, cudaStream_t st);

cudaError_t mlp_forward(const MlpLayer1Args &l1, const MlpWeights &wt, float *U, float *y, const float *target,
                        float *dy, float *loss, cudaStream_t st);
cudaError_t mlp_backward(const MlpLayer1Args &l1, const MlpWeights &wt, const float *U, const float *dy, float *dU,
                         float *dzt, float *grad, cudaStream_t st);
cudaError_t mlp_adam(float *p, const float *g, float *m, float *v, __nv_bfloat16 *pb, float lr, int step,
                     cudaStream_t st);
cudaError_t mlp_to_bf16(const float *p, __nv_bfloat16 *pb, cudaStream_t st);

}  // namespace cvrpsd
