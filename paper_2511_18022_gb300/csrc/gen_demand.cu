// Seeded scenario generator: fills a [n][ld] demand matrix on the device.
//
// Random words come from Philox4x32-10 (Salmon, Moraes, Dror, Shaw, "Parallel
// random numbers: as easy as 1, 2, 3", SC 2011), keyed by the 64-bit seed and
// counted by (scenario, index, domain, 0), so every entry is a pure function
// of its coordinates. Standard normals are Box-Muller draws in float64 from
// the first two words. Each float64 operation is written with an explicit
// round-to-nearest intrinsic so that no multiply-add is fused and the result
// is the one a plain IEEE evaluation in the written order gives.
#include <stdint.h>

#include "kernels.h"

namespace cvrpsd {

// Round multipliers and Weyl key increments of Philox4x32.
constexpr uint32_t kPhiloxM0 = 0xD2511F53u, kPhiloxM1 = 0xCD9E8D57u;
constexpr uint32_t kPhiloxW0 = 0x9E3779B9u, kPhiloxW1 = 0xBB67AE85u;

__device__ __forceinline__ uint4 philox4x32_10(uint4 c, uint32_t k0, uint32_t k1)
{
#pragma unroll
    for (int r = 0; r < 10; ++r) {
        if (r > 0) { k0 += kPhiloxW0; k1 += kPhiloxW1; }
        const uint32_t lo0 = kPhiloxM0 * c.x, hi0 = __umulhi(kPhiloxM0, c.x);
        const uint32_t lo1 = kPhiloxM1 * c.z, hi1 = __umulhi(kPhiloxM1, c.z);
        c = make_uint4(hi1 ^ c.y ^ k0, lo1, hi0 ^ c.w ^ k1, lo0);
    }
    return c;
}

__device__ __forceinline__ double std_normal(uint32_t s, uint32_t index, uint32_t domain,
                                             uint32_t k0, uint32_t k1)
{
    const uint4 w = philox4x32_10(make_uint4(s, index, domain, 0u), k0, k1);
    const double inv32 = 2.3283064365386963e-10;   // 2^-32
    const double two_pi = 6.283185307179586;
    const double u1 = __dmul_rn(__dadd_rn((double)w.x, 0.5), inv32);
    const double u2 = __dmul_rn((double)w.y, inv32);
    const double r = sqrt(__dmul_rn(-2.0, log(u1)));
    return __dmul_rn(r, cos(__dmul_rn(two_pi, u2)));
}

template <typename DT>
__global__ void __launch_bounds__(256) gen_demand_kernel(GenParams g, int rows_per_block)
{
    const long long s = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= g.S) return;
    const uint32_t k0 = (uint32_t)g.seed, k1 = (uint32_t)(g.seed >> 32);
    const int r0 = blockIdx.y * rows_per_block;
    const int r1 = min(g.n, r0 + rows_per_block);
    const double dmax = sizeof(DT) == 2 ? 32767.0 : 2147483647.0;
    double f[4];
    if (g.kind == 1) {
#pragma unroll
        for (int r = 0; r < 4; ++r) f[r] = std_normal((uint32_t)s, (uint32_t)r, 1u, k0, k1);
    }
    DT *out = reinterpret_cast<DT *>(g.out);
    for (int row = r0; row < r1; ++row) {
        const double mu = (double)g.mu[row];
        double x;
        if (g.kind == 1) {
            const double e = std_normal((uint32_t)s, (uint32_t)row, 0u, k0, k1);
            const int reg = g.region[row] & 3;
            const double fr = reg == 0 ? f[0] : reg == 1 ? f[1] : reg == 2 ? f[2] : f[3];
            const double y = __dadd_rn(__dmul_rn(0.6, fr), __dmul_rn(0.8, e));
            x = __dmul_rn(mu, exp(__dsub_rn(__dmul_rn(0.3, y), 0.045)));
        } else {
            const double z = std_normal((uint32_t)s, (uint32_t)row, 2u, k0, k1);
            x = __dadd_rn(mu, __dmul_rn(__dmul_rn(0.3, mu), z));
        }
        double rnd = floor(x);
        if (__dsub_rn(x, rnd) >= 0.5) rnd = __dadd_rn(rnd, 1.0);   // half away from zero
        rnd = fmin(fmax(rnd, 0.0), dmax);
        out[(long long)row * g.ld + s] = (DT)(long long)rnd;
    }
}

template <typename TI, typename TO>
__global__ void convert_demand_kernel(const TI *in, long long ld_in, TO *out, long long ld_out, int n, long long S,
                                      unsigned int *saturated)
{
    const long long s = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= S) return;
    for (int r = blockIdx.y; r < n; r += gridDim.y) {
        const long long v = (long long)in[(long long)r * ld_in + s];
        if (sizeof(TO) == 2 && (v > 32767 || v < -32768)) atomicOr(saturated, 1u);
        out[(long long)r * ld_out + s] = (TO)(v > 32767 && sizeof(TO) == 2 ? 32767 : v);
    }
}

cudaError_t launch_convert_demand(const void *in, int esize_in, long long ld_in, void *out, int esize_out,
                                  long long ld_out, int n, long long S, unsigned int *saturated,
                                  cudaStream_t stream)
{
    if (S == 0 || n == 0) return cudaSuccess;
    dim3 grid((unsigned)((S + 255) / 256), (unsigned)(n < 64 ? n : 64));
    if (esize_in == 2 && esize_out == 2)
        convert_demand_kernel<int16_t, int16_t><<<grid, 256, 0, stream>>>((const int16_t *)in, ld_in, (int16_t *)out,
                                                                          ld_out, n, S, saturated);
    else if (esize_in == 2)
        convert_demand_kernel<int16_t, int32_t><<<grid, 256, 0, stream>>>((const int16_t *)in, ld_in, (int32_t *)out,
                                                                          ld_out, n, S, saturated);
    else if (esize_out == 2)
        convert_demand_kernel<int32_t, int16_t><<<grid, 256, 0, stream>>>((const int32_t *)in, ld_in, (int16_t *)out,
                                                                          ld_out, n, S, saturated);
    else
        convert_demand_kernel<int32_t, int32_t><<<grid, 256, 0, stream>>>((const int32_t *)in, ld_in, (int32_t *)out,
                                                                          ld_out, n, S, saturated);
    return cudaGetLastError();
}

cudaError_t launch_gen_demand(const GenParams &g, int esize, cudaStream_t stream)
{
    if (g.S == 0 || g.n == 0) return cudaSuccess;
    const int threads = 256;
    const long long bx = (g.S + threads - 1) / threads;
    const int rows_per_block = 64;
    const int by = (g.n + rows_per_block - 1) / rows_per_block;
    dim3 grid((unsigned)bx, (unsigned)by);
    if (esize == 2) gen_demand_kernel<int16_t><<<grid, threads, 0, stream>>>(g, rows_per_block);
    else gen_demand_kernel<int32_t><<<grid, threads, 0, stream>>>(g, rows_per_block);
    return cudaGetLastError();
}

}  // namespace cvrpsd
