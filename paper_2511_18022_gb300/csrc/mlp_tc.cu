// Layer 1 of the surrogate network on the tensor cores (tcgen05, TMEM).
//
// Per tour the layer is a small matrix product: the pre-activations of the
// H = 256 hidden units at the n positions are W1' (H x 16) times F' (16 x n),
// where F' holds the five per-position features, a constant 1 (so that the
// bias b1 rides in W1' as a sixth column) and zero padding to K = 16, one MMA
// step of kind::f16 with BF16 operands. The accumulators land in tensor
// memory as FP32, hidden units on the 128 TMEM lanes and positions on the
// columns, so the mean-pooling over positions is a sum along each thread's
// own row: ReLU and sum in registers, no cross-thread reduction.
//
// One persistent CTA per SM (eight warps), looping over tours:
//   - W1' is staged in shared memory once, in the canonical K-major layout
//     without swizzle (8-row x 16-byte core matrices; 128 bytes between the
//     two core matrices along K, 256 bytes between 8-row groups);
//   - per chunk of up to 256 positions the threads compute the features
//     (the cumulative expected load is a block scan) and write F' in the same
//     layout; one thread issues two MMAs (hidden units 0-127 and 128-255 into
//     TMEM columns [0, 256) and [256, 512)) and commits them to an mbarrier;
//   - every warp waits on the mbarrier (bounded: after a fixed number of
//     polls it records an error and stops), loads its 32 lanes x 32 columns
//     at a time (tcgen05.ld 32x32b) and accumulates ReLU over the positions.
// The CTA allocates all 512 TMEM columns once and releases them at exit; its
// shared-memory request keeps one CTA per SM, so allocations never contend.
#include <cuda_bf16.h>
#include <stdint.h>

#include "mlp.h"

namespace cvrpsd {

namespace {

constexpr int kTcThreads = 256;          // eight warps
constexpr int kTcChunk = 256;            // positions per MMA (N <= 256)
constexpr int kTcK = 16;                 // one kind::f16 MMA step
constexpr uint32_t kTmemCols = 512;      // two 128 x 256 FP32 accumulators
constexpr uint32_t kPollLimit = 1u << 26;
// Shared memory the kernel asks for beyond its static arrays: enough that a
// second CTA cannot share the SM (and its tensor memory).
constexpr size_t kTcSmemPad = 120 * 1024;

// Byte offset of element (row, k) of a K-major, unswizzled BF16 operand of
// 16 columns: 8-row x 16-byte core matrices, two per 8-row group along K.
__device__ __forceinline__ uint32_t kmajor_offset(int row, int k)
{
    return (uint32_t)(((row >> 3) * 2 + (k >> 3)) * 128 + (row & 7) * 16 + (k & 7) * 2);
}

// Shared-memory matrix descriptor (sm_100 format): start address, leading
// byte offset (between core matrices along K), stride byte offset (between
// 8-row groups), descriptor version 1, no swizzle.
__device__ __forceinline__ uint64_t smem_desc(uint32_t saddr, uint32_t lbo, uint32_t sbo)
{
    uint64_t d = 0;
    d |= (uint64_t)((saddr & 0x3FFFFu) >> 4);
    d |= (uint64_t)((lbo >> 4) & 0x3FFFu) << 16;
    d |= (uint64_t)((sbo >> 4) & 0x3FFFu) << 32;
    d |= (uint64_t)1 << 46;
    return d;
}

// Instruction descriptor of kind::f16: FP32 accumulator, BF16 A and B, both
// K-major, M = 128, N = n_cols.
__device__ __forceinline__ uint32_t instr_desc(uint32_t n_cols)
{
    return (1u << 4) | (1u << 7) | (1u << 10) | ((n_cols >> 3) << 17) | ((128u >> 4) << 24);
}

__device__ __forceinline__ void mma_bf16(uint32_t d_tmem, uint64_t a, uint64_t b, uint32_t idesc, bool acc)
{
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "setp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}"
        ::"r"(d_tmem), "l"(a), "l"(b), "r"(idesc), "r"((uint32_t)acc) : "memory");
}

__device__ __forceinline__ void mma_commit(uint32_t mbar)
{
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(mbar)
                 : "memory");
}

// Poll the mbarrier's phase `parity` at most kPollLimit times.
__device__ __forceinline__ bool mbar_wait(uint32_t mbar, uint32_t parity)
{
    for (uint32_t it = 0; it < kPollLimit; ++it) {
        uint32_t done = 0;
        asm volatile(
            "{\n\t.reg .pred p;\n\t"
            "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
            "selp.u32 %0, 1, 0, p;\n\t}"
            : "=r"(done) : "r"(mbar), "r"(parity) : "memory");
        if (done) return true;
    }
    return false;
}

__device__ __forceinline__ void tmem_ld32(uint32_t taddr, float (&v)[32])
{
    uint32_t r[32];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x32.b32 "
        "{%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, %15, "
        "%16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, %28, %29, %30, %31}, [%32];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]),
          "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]),
          "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
        : "r"(taddr));
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
    for (int i = 0; i < 32; ++i) v[i] = __uint_as_float(r[i]);
}

__global__ void __launch_bounds__(kTcThreads, 1) mlp_layer1_tc_kernel(MlpLayer1Args a)
{
    __shared__ __align__(128) unsigned char s_w1[kMlpH * kTcK * 2];      // W1' (H x 16), 8 KB
    __shared__ __align__(128) unsigned char s_f[kTcChunk * kTcK * 2];    // F' (256 x 16), 8 KB
    __shared__ __align__(8) unsigned long long s_mbar;
    __shared__ uint32_t s_tmem;
    __shared__ float s_part[kTcThreads / 32];
    __shared__ float s_carry;
    __shared__ int s_abort;
    extern __shared__ unsigned char s_pad[];   // occupancy guard only (kTcSmemPad bytes)
    (void)s_pad;

    const int j = threadIdx.x, lane = j & 31, w = j >> 5;
    const int n = a.n;
    const long long N1 = (long long)n + 1;
    const uint32_t w1_s = (uint32_t)__cvta_generic_to_shared(s_w1);
    const uint32_t f_s = (uint32_t)__cvta_generic_to_shared(s_f);
    const uint32_t mbar = (uint32_t)__cvta_generic_to_shared(&s_mbar);

    // W1' = [W1 | b1 | 0]: row h, columns 0..4 weights, 5 bias, 6..15 zero.
    for (int e = j; e < kMlpH * kTcK; e += kTcThreads) {
        const int h = e / kTcK, k = e % kTcK;
        __nv_bfloat16 v = __float2bfloat16_rn(0.0f);
        if (k < kMlpIn1) v = a.w1[h * kMlpIn1 + k];
        else if (k == kMlpIn1) v = a.b1[h];
        *reinterpret_cast<__nv_bfloat16 *>(s_w1 + kmajor_offset(h, k)) = v;
    }
    if (j == 0) {
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(mbar) : "memory");
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        s_abort = 0;
    }
    if (w == 0) {
        const uint32_t dst = (uint32_t)__cvta_generic_to_shared(&s_tmem);
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(dst),
                     "r"(kTmemCols) : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const uint32_t tmem = s_tmem;
    const uint64_t a_desc0 = smem_desc(w1_s, 128, 256);
    const uint64_t a_desc1 = smem_desc(w1_s + 16 * 256, 128, 256);   // hidden units 128..255
    const uint64_t b_desc = smem_desc(f_s, 128, 256);
    // This warp's TMEM rows: lanes 32 (w % 4) .. +31 of accumulator w / 4.
    const int half = w >> 2;
    const uint32_t t_row = tmem + ((uint32_t)(32 * (w & 3)) << 16) + (uint32_t)(half * kTcChunk);
    const int h = half * 128 + 32 * (w & 3) + lane;
    const __nv_bfloat16 one = __float2bfloat16_rn(1.0f), zero = __float2bfloat16_rn(0.0f);
    uint32_t parity = 0;

    for (int t = blockIdx.x; t < a.T; t += gridDim.x) {
        const int32_t *tour = a.tours + (long long)t * n;
        float len = 0.0f, acc = 0.0f;
        if (j == 0) s_carry = 0.0f;
        __syncthreads();
        for (int k0 = 0; k0 < n; k0 += kTcChunk) {
            // features of positions k0 .. k0 + 255 (thread j: position k0 + j)
            const int k = k0 + j;
            float m = 0.0f;
            int c = 1;
            if (k < n) {
                c = min(max(tour[k], 1), n);
                m = a.cust[(c - 1) * 4 + 2];
                const int nx = k + 1 < n ? min(max(tour[k + 1], 1), n) : 0;
                len += (float)a.dist[(long long)c * N1 + nx];
                if (k == 0) len += (float)a.dist[c];
            }
            float v = m;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const float u = __shfl_up_sync(0xffffffffu, v, o);
                if (lane >= o) v += u;
            }
            if (lane == 31) s_part[w] = v;
            __syncthreads();
            float off = s_carry;
            for (int q = 0; q < w; ++q) off += s_part[q];
            const float cum = off + v;
            __nv_bfloat16 f[kTcK];
#pragma unroll
            for (int q = 0; q < kTcK; ++q) f[q] = zero;
            if (k < n) {
                f[0] = __float2bfloat16_rn(a.cust[(c - 1) * 4 + 0]);
                f[1] = __float2bfloat16_rn(a.cust[(c - 1) * 4 + 1]);
                f[2] = __float2bfloat16_rn(m);
                f[3] = __float2bfloat16_rn(a.cust[(c - 1) * 4 + 3]);
                f[4] = __float2bfloat16_rn(cum - floorf(cum));
                f[5] = one;
            }
            // row j of F': two 16-byte halves (k 0..7 and 8..15)
#pragma unroll
            for (int half_k = 0; half_k < 2; ++half_k) {
                uint4 pack;
                uint32_t *pw = reinterpret_cast<uint32_t *>(&pack);
#pragma unroll
                for (int q = 0; q < 4; ++q) {
                    const uint32_t lo = __bfloat16_as_ushort(f[half_k * 8 + 2 * q]);
                    const uint32_t hi = __bfloat16_as_ushort(f[half_k * 8 + 2 * q + 1]);
                    pw[q] = lo | (hi << 16);
                }
                *reinterpret_cast<uint4 *>(s_f + kmajor_offset(j, half_k * 8)) = pack;
            }
            __syncthreads();
            if (j == kTcThreads - 1) s_carry = cum;
            // operands visible to the tensor cores, previous TMEM reads retired
            asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
            asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
            __syncthreads();
            asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
            const int cnt = min(kTcChunk, n - k0);
            const uint32_t ncols = (uint32_t)((cnt + 31) / 32 * 32);
            if (j == 0) {
                const uint32_t idesc = instr_desc(ncols);
                mma_bf16(tmem, a_desc0, b_desc, idesc, false);
                mma_bf16(tmem + kTcChunk, a_desc1, b_desc, idesc, false);
                mma_commit(mbar);
            }
            if (!mbar_wait(mbar, parity)) {
                atomicOr(a.err, 1u);
                s_abort = 1;
            }
            parity ^= 1u;
            asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
            __syncthreads();
            if (s_abort) break;
            // ReLU and sum along this thread's row (positions past n hold 0)
            for (uint32_t col = 0; col < ncols; col += 32) {
                float r[32];
                tmem_ld32(t_row + col, r);
#pragma unroll
                for (int q = 0; q < 32; ++q) acc += fmaxf(r[q], 0.0f);
            }
        }
        if (s_abort) break;
        // tour length: block sum of the per-thread partial lengths
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) len += __shfl_xor_sync(0xffffffffu, len, o);
        __syncthreads();
        if (lane == 0) s_part[w] = len;
        __syncthreads();
        if (j == 0) {
            float tl = 0.0f;
            for (int q = 0; q < kTcThreads / 32; ++q) tl += s_part[q];
            a.zt[(long long)t * kMlpIn2 + kMlpH] = (tl - a.len_mean) * a.len_inv_sd;
        }
        a.zt[(long long)t * kMlpIn2 + h] = acc / (float)n;
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    if (w == 0)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(kTmemCols) : "memory");
}

}  // namespace

cudaError_t mlp_layer1_tc(const MlpLayer1Args &l1, int sm_count, cudaStream_t st)
{
    cudaError_t e = cudaFuncSetAttribute(mlp_layer1_tc_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)kTcSmemPad);
    if (e != cudaSuccess) return e;
    const int grid = l1.T < sm_count ? l1.T : sm_count;
    mlp_layer1_tc_kernel<<<grid, kTcThreads, kTcSmemPad, st>>>(l1);
    return cudaGetLastError();
}

}  // namespace cvrpsd
