// Layers 1 and 2 of the surrogate network's forward pass on the tensor cores
// (tcgen05, TMEM). Layer 1:
//
// Per tour the layer is a small matrix product: the pre-activations of the
// H = 256 hidden units at the n positions are W1' (H x 16) times F' (16 x n),
// one MMA step of kind::f16 with BF16 operands. F' holds each of the five
// per-position features as two BF16 numbers, hi = bf16(v) in columns 0-4 and
// lo = bf16(v - hi) in columns 6-10, with a constant 1 in column 5; W1' holds
// W1 in columns 0-4 and again in 6-10, and the bias b1 in column 5. So the
// product keeps about 16 significant bits of the features against the exact
// BF16 weights, at no extra MMA: K = 16 has room. The accumulators land in tensor
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
#include "tcgen05.h"

namespace cvrpsd {

namespace {

constexpr int kTcThreads = 256;          // eight warps
constexpr int kTcChunk = 256;            // positions per MMA (N <= 256)
constexpr int kTcK = 16;                 // one kind::f16 MMA step
constexpr uint32_t kTmemCols = 512;      // two 128 x 256 FP32 accumulators
// Shared memory the kernel asks for beyond its static arrays: enough that a
// second CTA cannot share the SM (and its tensor memory).
constexpr size_t kTcSmemPad = 120 * 1024;

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

    // W1' = [W1 | b1 | W1 | 0]: row h, columns 0..4 and 6..10 weights, 5 bias,
    // 11..15 zero.
    for (int e = j; e < kMlpH * kTcK; e += kTcThreads) {
        const int h = e / kTcK, k = e % kTcK;
        __nv_bfloat16 v = __float2bfloat16_rn(0.0f);
        if (k < kMlpIn1) v = a.w1[h * kMlpIn1 + k];
        else if (k == kMlpIn1) v = a.b1[h];
        else if (k < 2 * kMlpIn1 + 1) v = a.w1[h * kMlpIn1 + k - kMlpIn1 - 1];
        *reinterpret_cast<__nv_bfloat16 *>(s_w1 + tc::kmajor_offset(h, k, 2)) = v;
    }
    if (j == 0) {
        tc::mbar_init(mbar);
        s_abort = 0;
    }
    if (w == 0) tc::tmem_alloc((uint32_t)__cvta_generic_to_shared(&s_tmem), kTmemCols);
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
    const uint32_t tmem = s_tmem;
    const uint64_t a_desc0 = tc::smem_desc(w1_s, 128, 256);
    const uint64_t a_desc1 = tc::smem_desc(w1_s + 16 * 256, 128, 256);   // hidden units 128..255
    const uint64_t b_desc = tc::smem_desc(f_s, 128, 256);
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
                const float v[kMlpIn1] = {a.cust[(c - 1) * 4 + 0], a.cust[(c - 1) * 4 + 1], m,
                                          a.cust[(c - 1) * 4 + 3], cum - floorf(cum)};
#pragma unroll
                for (int q = 0; q < kMlpIn1; ++q) {
                    f[q] = __float2bfloat16_rn(v[q]);
                    f[q + kMlpIn1 + 1] = __float2bfloat16_rn(v[q] - __bfloat162float(f[q]));
                }
                f[kMlpIn1] = one;
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
                *reinterpret_cast<uint4 *>(s_f + tc::kmajor_offset(j, half_k * 8, 2)) = pack;
            }
            __syncthreads();
            if (j == kTcThreads - 1) s_carry = cum;
            // operands visible to the tensor cores, previous TMEM reads retired
            tc::fence_operands();
            tc::fence_before_sync();
            __syncthreads();
            tc::fence_after_sync();
            const int cnt = min(kTcChunk, n - k0);
            const uint32_t ncols = (uint32_t)((cnt + 31) / 32 * 32);
            if (j == 0) {
                const uint32_t idesc = tc::instr_desc(ncols);
                tc::mma_bf16(tmem, a_desc0, b_desc, idesc, false);
                tc::mma_bf16(tmem + kTcChunk, a_desc1, b_desc, idesc, false);
                tc::mma_commit(mbar);
            }
            if (!tc::mbar_wait(mbar, parity)) {
                atomicOr(a.err, 1u);
                s_abort = 1;
            }
            parity ^= 1u;
            tc::fence_after_sync();
            __syncthreads();
            if (s_abort) break;
            // ReLU and sum along this thread's row (positions past n hold 0)
            for (uint32_t col = 0; col < ncols; col += 32) {
                float r[32];
                tc::tmem_ld32(t_row + col, r);
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
    tc::fence_before_sync();
    __syncthreads();
    if (w == 0) tc::tmem_dealloc(tmem, kTmemCols);
}

// ---------------------------------------------------------------- layer 2
//
// U = relu([z; t] W2^T + b2) for a tile of 128 tours and 64 of the 256 hidden
// units: M = 128 tours, N = 64, K = 257 inputs + 1 (the bias rides in W2' as
// column 257 against a constant 1) padded to 272 = 17 MMA steps. The pooled
// inputs are FP32; each is split into BF16 hi + lo parts (hi = bf16(v),
// lo = bf16(v - hi)) and both products are accumulated, so the result keeps
// about 16 significant bits of the inputs against the exact BF16 weights:
// the FP32 layer's accuracy on the tensor cores. Operands are staged 16 bytes
// (one core-matrix row) per store.
constexpr int kL2K = 272;                 // padded K
constexpr int kL2Kc = kL2K / 8;           // 16-byte core-matrix columns per row group
constexpr int kL2M = 128;                 // tours per CTA
constexpr int kL2N = 64;                  // hidden units per CTA
constexpr size_t kL2A = (size_t)kL2M * kL2K * 2;   // one 128 x 272 BF16 operand
constexpr size_t kL2B = (size_t)kL2N * kL2K * 2;
constexpr size_t kL2Smem = 2 * kL2A + kL2B;        // A hi, A lo, B
constexpr uint32_t kL2TmemCols = 64;

__device__ __forceinline__ uint32_t pack_bf16x2(__nv_bfloat16 a, __nv_bfloat16 b)
{
    return (uint32_t)__bfloat16_as_ushort(a) | ((uint32_t)__bfloat16_as_ushort(b) << 16);
}

__global__ void __launch_bounds__(kTcThreads, 1) mlp_layer2_tc_kernel(const float *zt, int T,
                                                                      const __nv_bfloat16 *w2,
                                                                      const __nv_bfloat16 *b2, float *U,
                                                                      unsigned int *err)
{
    extern __shared__ __align__(128) unsigned char smem[];   // A hi | A lo | B
    __shared__ __align__(8) unsigned long long s_mbar;
    __shared__ uint32_t s_tmem;
    unsigned char *a_hi = smem, *a_lo = smem + kL2A, *bw = smem + 2 * kL2A;
    const int j = threadIdx.x, lane = j & 31, w = j >> 5;
    const int t0 = blockIdx.x * kL2M, o0 = blockIdx.y * kL2N;
    const uint32_t mbar = (uint32_t)__cvta_generic_to_shared(&s_mbar);
    // B = W2' rows o0 .. o0 + 63: weights, bias at column 257, zeros after;
    // item = (row, group of 8 columns)
    for (int e = j; e < kL2N * kL2Kc; e += kTcThreads) {
        const int r = e / kL2Kc, g = e % kL2Kc;
        uint32_t pw[4];
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            __nv_bfloat16 v[2];
#pragma unroll
            for (int h = 0; h < 2; ++h) {
                const int k = 8 * g + 2 * q + h;
                v[h] = k < kMlpIn2 ? w2[(long long)(o0 + r) * kMlpIn2 + k]
                                   : (k == kMlpIn2 ? b2[o0 + r] : __float2bfloat16_rn(0.0f));
            }
            pw[q] = pack_bf16x2(v[0], v[1]);
        }
        *reinterpret_cast<uint4 *>(bw + tc::kmajor_offset(r, 8 * g, kL2Kc)) = make_uint4(pw[0], pw[1], pw[2], pw[3]);
    }
    // A = [z; t; 1] of tours t0 .. t0 + 127, split into BF16 hi and lo parts
    for (int e = j; e < kL2M * kL2Kc; e += kTcThreads) {
        const int r = e / kL2Kc, g = e % kL2Kc;
        const int t = t0 + r;
        uint32_t ph[4], pl[4];
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            __nv_bfloat16 hi[2], lo[2];
#pragma unroll
            for (int h = 0; h < 2; ++h) {
                const int k = 8 * g + 2 * q + h;
                float v = 0.0f;
                if (t < T) v = k < kMlpIn2 ? zt[(long long)t * kMlpIn2 + k] : (k == kMlpIn2 ? 1.0f : 0.0f);
                hi[h] = __float2bfloat16_rn(v);
                lo[h] = __float2bfloat16_rn(v - __bfloat162float(hi[h]));
            }
            ph[q] = pack_bf16x2(hi[0], hi[1]);
            pl[q] = pack_bf16x2(lo[0], lo[1]);
        }
        const uint32_t off = tc::kmajor_offset(r, 8 * g, kL2Kc);
        *reinterpret_cast<uint4 *>(a_hi + off) = make_uint4(ph[0], ph[1], ph[2], ph[3]);
        *reinterpret_cast<uint4 *>(a_lo + off) = make_uint4(pl[0], pl[1], pl[2], pl[3]);
    }
    if (j == 0) tc::mbar_init(mbar);
    if (w == 0) tc::tmem_alloc((uint32_t)__cvta_generic_to_shared(&s_tmem), kL2TmemCols);
    tc::fence_operands();
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
    const uint32_t tmem = s_tmem;
    if (j == 0) {
        const uint32_t idesc = tc::instr_desc(kL2N);
        const uint32_t sa_hi = (uint32_t)__cvta_generic_to_shared(a_hi);
        const uint32_t sa_lo = (uint32_t)__cvta_generic_to_shared(a_lo);
        const uint32_t sb = (uint32_t)__cvta_generic_to_shared(bw);
        const uint32_t sbo = kL2Kc * 128;
        for (int step = 0; step < kL2K / 16; ++step) {
            const uint32_t koff = (uint32_t)step * 256;     // two 16-byte core-matrix columns per step
            const uint64_t bd = tc::smem_desc(sb + koff, 128, sbo);
            tc::mma_bf16(tmem, tc::smem_desc(sa_hi + koff, 128, sbo), bd, idesc, step > 0);
            tc::mma_bf16(tmem, tc::smem_desc(sa_lo + koff, 128, sbo), bd, idesc, true);
        }
        tc::mma_commit(mbar);
    }
    const bool ok = tc::mbar_wait(mbar, 0);
    if (!ok && lane == 0) atomicOr(err, 1u);
    tc::fence_after_sync();
    __syncthreads();
    if (ok && w < 4) {
        // warp w: tours (lanes) 32 w .. 32 w + 31, all 64 hidden columns
        const int t = t0 + 32 * w + lane;
        const uint32_t row = tmem + ((uint32_t)(32 * w) << 16);
#pragma unroll
        for (int c = 0; c < kL2N; c += 32) {
            float r[32];
            tc::tmem_ld32(row + c, r);
            if (t < T) {
                float *out = U + (long long)t * kMlpH + o0 + c;
#pragma unroll
                for (int q = 0; q < 32; q += 4)
                    *reinterpret_cast<float4 *>(out + q) = make_float4(fmaxf(r[q], 0.0f), fmaxf(r[q + 1], 0.0f),
                                                                       fmaxf(r[q + 2], 0.0f), fmaxf(r[q + 3], 0.0f));
            }
        }
    }
    tc::fence_before_sync();
    __syncthreads();
    if (w == 0) tc::tmem_dealloc(tmem, kL2TmemCols);
}

// ---------------------------------------------------------------- backward GEMMs
//
// C (M x N) = A (M x K) B (N x K)^T on the tensor cores, stored or added
// atomically (split-K over blockIdx.z). One CTA computes a 128 x 160 tile of C
// in tensor memory, K in chunks of 64 staged in shared memory in the K-major
// layout of the forward kernels. FP32 operands are split into BF16 hi and
// lo parts (hi = bf16(v), lo = bf16(v - hi)); a product of two split
// operands takes hi*hi + hi*lo + lo*hi (the lo*lo term, at most 2^-18 of
// the product, is the order of the pair's own rounding and is left out),
// one with an exact BF16 operand hi*B + lo*B. Operands
// are read through an element rule: A(m, k) at a[m * lda + k], or at
// a[k * lda + m] when transposed (AT); B likewise (BT), FP32 or BF16.
constexpr int kGM = 128;                       // rows of C per CTA
constexpr int kGN = 160;                       // columns of C per CTA (5 x 32)
constexpr int kGK = 64;                        // K per staged chunk
constexpr int kGKc = kGK / 8;                  // 16-byte core-matrix columns per row group
constexpr size_t kGA = (size_t)kGM * kGK * 2;  // one BF16 A part
constexpr size_t kGB = (size_t)kGN * kGK * 2;  // one BF16 B part
constexpr size_t kGSmem = 2 * kGA + 2 * kGB;   // A hi, A lo, B hi, B lo
// Requested dynamic shared memory: the operands plus padding so that at
// most two CTAs share an SM (each holds 256 TMEM columns).
constexpr size_t kGSmemReq = 100 * 1024;
static_assert(kGSmem <= kGSmemReq, "GEMM operands exceed the requested shared memory");
constexpr uint32_t kGTmemCols = 256;

struct TcGemm {
    const float *a;          // FP32 A
    int lda;
    const float *bf;         // FP32 B (or nullptr)
    const __nv_bfloat16 *bh; // BF16 B (or nullptr)
    int ldb;
    int M, N, K;
    int k_slab;              // K per blockIdx.z
    float *out;
    int ldo;
    unsigned int *err;
};

template <bool AT, bool BT, bool BBF16, bool ATOMIC>
__global__ void __launch_bounds__(kTcThreads, 1) tc_gemm_kernel(TcGemm g)
{
    extern __shared__ __align__(128) unsigned char smem[];   // A hi | A lo | B hi | B lo
    __shared__ __align__(8) unsigned long long s_mbar;
    __shared__ uint32_t s_tmem;
    unsigned char *a_hi = smem, *a_lo = smem + kGA, *b_hi = smem + 2 * kGA, *b_lo = smem + 2 * kGA + kGB;
    const int j = threadIdx.x, lane = j & 31, w = j >> 5;
    const int m0 = blockIdx.x * kGM, n0 = blockIdx.y * kGN;
    const int k_begin = blockIdx.z * g.k_slab, k_end = min(g.K, k_begin + g.k_slab);
    const uint32_t mbar = (uint32_t)__cvta_generic_to_shared(&s_mbar);
    if (j == 0) tc::mbar_init(mbar);
    if (w == 0) tc::tmem_alloc((uint32_t)__cvta_generic_to_shared(&s_tmem), kGTmemCols);
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
    const uint32_t tmem = s_tmem;
    uint32_t parity = 0;
    bool ok = true, any = false;
    for (int kc0 = k_begin; kc0 < k_end; kc0 += kGK) {
        // A: item = (row, group of 8 K columns); transposed operands read the
        // row index fastest, so neighbouring threads read neighbouring words
        for (int e = j; e < kGM * kGKc; e += kTcThreads) {
            const int r = AT ? e % kGM : e / kGKc, gk = AT ? e / kGM : e % kGKc;
            const int m = m0 + r;
            uint32_t ph[4], pl[4];
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                __nv_bfloat16 hi[2], lo[2];
#pragma unroll
                for (int h = 0; h < 2; ++h) {
                    const int k = kc0 + 8 * gk + 2 * q + h;
                    float v = 0.0f;
                    if (m < g.M && k < k_end) v = AT ? g.a[(long long)k * g.lda + m] : g.a[(long long)m * g.lda + k];
                    hi[h] = __float2bfloat16_rn(v);
                    lo[h] = __float2bfloat16_rn(v - __bfloat162float(hi[h]));
                }
                ph[q] = pack_bf16x2(hi[0], hi[1]);
                pl[q] = pack_bf16x2(lo[0], lo[1]);
            }
            const uint32_t off = tc::kmajor_offset(r, 8 * gk, kGKc);
            *reinterpret_cast<uint4 *>(a_hi + off) = make_uint4(ph[0], ph[1], ph[2], ph[3]);
            *reinterpret_cast<uint4 *>(a_lo + off) = make_uint4(pl[0], pl[1], pl[2], pl[3]);
        }
        for (int e = j; e < kGN * kGKc; e += kTcThreads) {
            const int r = BT ? e % kGN : e / kGKc, gk = BT ? e / kGN : e % kGKc;
            const int nn = n0 + r;
            uint32_t ph[4], pl[4];
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                __nv_bfloat16 hi[2], lo[2];
#pragma unroll
                for (int h = 0; h < 2; ++h) {
                    const int k = kc0 + 8 * gk + 2 * q + h;
                    const bool in = nn < g.N && k < k_end;
                    if (BBF16) {
                        hi[h] = in ? (BT ? g.bh[(long long)k * g.ldb + nn] : g.bh[(long long)nn * g.ldb + k])
                                   : __float2bfloat16_rn(0.0f);
                        lo[h] = __float2bfloat16_rn(0.0f);
                    } else {
                        const float v = in ? (BT ? g.bf[(long long)k * g.ldb + nn] : g.bf[(long long)nn * g.ldb + k])
                                           : 0.0f;
                        hi[h] = __float2bfloat16_rn(v);
                        lo[h] = __float2bfloat16_rn(v - __bfloat162float(hi[h]));
                    }
                }
                ph[q] = pack_bf16x2(hi[0], hi[1]);
                pl[q] = pack_bf16x2(lo[0], lo[1]);
            }
            const uint32_t off = tc::kmajor_offset(r, 8 * gk, kGKc);
            *reinterpret_cast<uint4 *>(b_hi + off) = make_uint4(ph[0], ph[1], ph[2], ph[3]);
            if (!BBF16) *reinterpret_cast<uint4 *>(b_lo + off) = make_uint4(pl[0], pl[1], pl[2], pl[3]);
        }
        tc::fence_operands();
        tc::fence_before_sync();
        __syncthreads();
        tc::fence_after_sync();
        if (j == 0) {
            const uint32_t idesc = tc::instr_desc(kGN);
            const uint32_t sah = (uint32_t)__cvta_generic_to_shared(a_hi), sal = (uint32_t)__cvta_generic_to_shared(a_lo);
            const uint32_t sbh = (uint32_t)__cvta_generic_to_shared(b_hi), sbl = (uint32_t)__cvta_generic_to_shared(b_lo);
            const uint32_t sbo = kGKc * 128;
            for (int step = 0; step < kGK / 16; ++step) {
                const uint32_t koff = (uint32_t)step * 256;
                const uint64_t ah = tc::smem_desc(sah + koff, 128, sbo), al = tc::smem_desc(sal + koff, 128, sbo);
                const uint64_t bh = tc::smem_desc(sbh + koff, 128, sbo);
                tc::mma_bf16(tmem, ah, bh, idesc, any || step > 0);
                tc::mma_bf16(tmem, al, bh, idesc, true);
                if (!BBF16) tc::mma_bf16(tmem, ah, tc::smem_desc(sbl + koff, 128, sbo), idesc, true);
            }
            tc::mma_commit(mbar);
        }
        any = true;
        // the operands are overwritten next chunk: wait for the MMAs
        ok = tc::mbar_wait(mbar, parity);
        parity ^= 1u;
        if (!ok && lane == 0) atomicOr(g.err, 1u);
        tc::fence_after_sync();
        __syncthreads();
        if (!ok) break;
    }
    if (ok && any && w < 4) {
        const int m = m0 + 32 * w + lane;
        const uint32_t row = tmem + ((uint32_t)(32 * w) << 16);
#pragma unroll 1
        for (int c = 0; c < kGN; c += 32) {
            float r[32];
            tc::tmem_ld32(row + c, r);
            if (m < g.M) {
                float *out = g.out + (long long)m * g.ldo + n0 + c;
#pragma unroll
                for (int q = 0; q < 32; ++q) {
                    if (n0 + c + q < g.N) {
                        if (ATOMIC) atomicAdd(out + q, r[q]);
                        else out[q] = r[q];
                    }
                }
            }
        }
    }
    tc::fence_before_sync();
    __syncthreads();
    if (w == 0) tc::tmem_dealloc(tmem, kGTmemCols);
}

template <bool AT, bool BT, bool BBF16, bool ATOMIC>
cudaError_t tc_gemm(const TcGemm &g, cudaStream_t st)
{
    auto kern = tc_gemm_kernel<AT, BT, BBF16, ATOMIC>;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kGSmemReq);
    if (e != cudaSuccess) return e;
    const int slabs = (g.K + g.k_slab - 1) / g.k_slab;
    const dim3 grid((unsigned)((g.M + kGM - 1) / kGM), (unsigned)((g.N + kGN - 1) / kGN), (unsigned)slabs);
    kern<<<grid, kTcThreads, kGSmemReq, st>>>(g);
    return cudaGetLastError();
}

// ---------------------------------------------------------------- layer 1 backward
//
// dW1 and db1 on the tensor cores. With m_hk = [pre_hk > 0] the ReLU mask of
// hidden unit h at position k, the gradient of tour t is
//     dW1'[h][:] += (dz_th / n) * sum_k m_hk F'[k][:]
// (F' the 16-column feature rows of the forward pass: hi parts, the 1 of
// the bias, lo parts), so per tour the contraction is Mask (H x n) times F'
// (n x 16): the mask is exact in BF16 and F' is the forward operand, and
// the per-unit factor is applied to the FP32 result. Per chunk of 224
// positions one CTA recomputes the pre-activations as the forward pass does
// (two 128 x 224 MMAs into TMEM columns [0, 224) and [256, 480)), turns them
// into the mask in shared memory (K-major, row h, K = positions), and adds
// Mask x F'^T into two 128 x 16 accumulators at columns 224 and 480
// (14 MMA steps each) against F' stored transposed (row = feature, K =
// position). After the tour's last chunk each thread scales its unit's row
// by dz_th / n and keeps the sums; they reach the gradient once per CTA.
constexpr int kBwChunk = 224;                  // positions per chunk (7 x 32)
constexpr int kBwKc = kBwChunk / 8;            // 28 core-matrix columns along positions
constexpr size_t kBwMaskHalf = (size_t)128 * kBwChunk * 2;   // one half's mask, BF16
constexpr size_t kBwF2 = (size_t)16 * kBwChunk * 2;          // F' transposed
constexpr size_t kBwSmem = 2 * kBwMaskHalf + kBwF2;          // dynamic part
constexpr uint32_t kBwAcc0 = kBwChunk, kBwAcc1 = 256 + kBwChunk;   // TMEM columns of the two sums

__global__ void __launch_bounds__(kTcThreads, 1) mlp_layer1_bwd_tc_kernel(MlpLayer1Args a)
{
    __shared__ __align__(128) unsigned char s_w1[kMlpH * kTcK * 2];      // W1' (H x 16), as forward
    __shared__ __align__(128) unsigned char s_f[kBwChunk * kTcK * 2];    // F' (224 x 16), as forward
    __shared__ __align__(8) unsigned long long s_mbar;
    __shared__ uint32_t s_tmem;
    __shared__ float s_part[kTcThreads / 32];
    __shared__ float s_carry;
    __shared__ int s_abort;
    extern __shared__ __align__(128) unsigned char s_dyn[];   // mask half 0 | mask half 1 | F' transposed
    unsigned char *s_mask = s_dyn, *s_f2 = s_dyn + 2 * kBwMaskHalf;

    const int j = threadIdx.x, lane = j & 31, w = j >> 5;
    const int n = a.n;
    const uint32_t w1_s = (uint32_t)__cvta_generic_to_shared(s_w1);
    const uint32_t f_s = (uint32_t)__cvta_generic_to_shared(s_f);
    const uint32_t m_s = (uint32_t)__cvta_generic_to_shared(s_mask);
    const uint32_t f2_s = (uint32_t)__cvta_generic_to_shared(s_f2);
    const uint32_t mbar = (uint32_t)__cvta_generic_to_shared(&s_mbar);

    for (int e = j; e < kMlpH * kTcK; e += kTcThreads) {
        const int h = e / kTcK, k = e % kTcK;
        __nv_bfloat16 v = __float2bfloat16_rn(0.0f);
        if (k < kMlpIn1) v = a.w1[h * kMlpIn1 + k];
        else if (k == kMlpIn1) v = a.b1[h];
        else if (k < 2 * kMlpIn1 + 1) v = a.w1[h * kMlpIn1 + k - kMlpIn1 - 1];
        *reinterpret_cast<__nv_bfloat16 *>(s_w1 + tc::kmajor_offset(h, k, 2)) = v;
    }
    if (j == 0) {
        tc::mbar_init(mbar);
        s_abort = 0;
    }
    if (w == 0) tc::tmem_alloc((uint32_t)__cvta_generic_to_shared(&s_tmem), kTmemCols);
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
    const uint32_t tmem = s_tmem;
    const uint64_t a_desc0 = tc::smem_desc(w1_s, 128, 256);
    const uint64_t a_desc1 = tc::smem_desc(w1_s + 16 * 256, 128, 256);
    const uint64_t b_desc = tc::smem_desc(f_s, 128, 256);
    const int half = w >> 2;
    const int hl = 32 * (w & 3) + lane;                  // row within the half
    const int h = half * 128 + hl;
    const uint32_t t_row = tmem + ((uint32_t)(32 * (w & 3)) << 16);
    const uint32_t pre_col = (uint32_t)(half * 256), acc_col = half ? kBwAcc1 : kBwAcc0;
    unsigned char *my_mask = s_mask + (size_t)half * kBwMaskHalf;
    const __nv_bfloat16 one = __float2bfloat16_rn(1.0f), zero = __float2bfloat16_rn(0.0f);
    const uint32_t one2 = (uint32_t)__bfloat16_as_ushort(one);
    uint32_t parity = 0;
    float gw[kMlpIn1 + 1] = {0, 0, 0, 0, 0, 0};

    for (int t = blockIdx.x; t < a.T; t += gridDim.x) {
        const int32_t *tour = a.tours + (long long)t * n;
        if (j == 0) s_carry = 0.0f;
        __syncthreads();
        int chunk = 0;
        for (int k0 = 0; k0 < n; k0 += kBwChunk, ++chunk) {
            // features of positions k0 .. k0 + 223 (thread j < 224: position k0 + j)
            const int k = k0 + j;
            const bool valid = j < kBwChunk && k < n;
            float m = 0.0f;
            int c = 1;
            if (valid) {
                c = min(max(tour[k], 1), n);
                m = a.cust[(c - 1) * 4 + 2];
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
            if (valid) {
                const float v5[kMlpIn1] = {a.cust[(c - 1) * 4 + 0], a.cust[(c - 1) * 4 + 1], m,
                                           a.cust[(c - 1) * 4 + 3], cum - floorf(cum)};
#pragma unroll
                for (int q = 0; q < kMlpIn1; ++q) {
                    f[q] = __float2bfloat16_rn(v5[q]);
                    f[q + kMlpIn1 + 1] = __float2bfloat16_rn(v5[q] - __bfloat162float(f[q]));
                }
                f[kMlpIn1] = one;
            }
            if (j < kBwChunk) {
#pragma unroll
                for (int half_k = 0; half_k < 2; ++half_k) {
                    uint32_t pw[4];
#pragma unroll
                    for (int q = 0; q < 4; ++q)
                        pw[q] = (uint32_t)__bfloat16_as_ushort(f[half_k * 8 + 2 * q]) |
                                ((uint32_t)__bfloat16_as_ushort(f[half_k * 8 + 2 * q + 1]) << 16);
                    *reinterpret_cast<uint4 *>(s_f + tc::kmajor_offset(j, half_k * 8, 2)) =
                        make_uint4(pw[0], pw[1], pw[2], pw[3]);
                }
                // the same values transposed: row = feature, K = position
#pragma unroll
                for (int q = 0; q < kTcK; ++q)
                    *reinterpret_cast<__nv_bfloat16 *>(s_f2 + tc::kmajor_offset(q, j, kBwKc)) = f[q];
            }
            // the scan carry: the last position of this chunk (thread 223)
            __syncthreads();
            if (j == kBwChunk - 1) s_carry = cum;
            tc::fence_operands();
            tc::fence_before_sync();
            __syncthreads();
            tc::fence_after_sync();
            const int cnt = min(kBwChunk, n - k0);
            const uint32_t ncols = (uint32_t)((cnt + 31) / 32 * 32);
            if (j == 0) {
                const uint32_t idesc = tc::instr_desc(ncols);
                tc::mma_bf16(tmem, a_desc0, b_desc, idesc, false);
                tc::mma_bf16(tmem + 256, a_desc1, b_desc, idesc, false);
                tc::mma_commit(mbar);
            }
            if (!tc::mbar_wait(mbar, parity)) {
                atomicOr(a.err, 1u);
                s_abort = 1;
            }
            parity ^= 1u;
            tc::fence_after_sync();
            __syncthreads();
            if (s_abort) break;
            // the mask of this thread's unit: 8 positions per 16-byte store
            for (uint32_t col = 0; col < (uint32_t)kBwChunk; col += 32) {
                float r[32];
                if (col < ncols) tc::tmem_ld32(t_row + pre_col + col, r);
#pragma unroll
                for (int g8 = 0; g8 < 4; ++g8) {
                    uint32_t pw[4];
#pragma unroll
                    for (int q = 0; q < 4; ++q) {
                        const bool m0 = col < ncols && r[g8 * 8 + 2 * q] > 0.0f;
                        const bool m1 = col < ncols && r[g8 * 8 + 2 * q + 1] > 0.0f;
                        pw[q] = (m0 ? one2 : 0u) | ((m1 ? one2 : 0u) << 16);
                    }
                    *reinterpret_cast<uint4 *>(my_mask + tc::kmajor_offset(hl, (int)col + 8 * g8, kBwKc)) =
                        make_uint4(pw[0], pw[1], pw[2], pw[3]);
                }
            }
            tc::fence_operands();
            tc::fence_before_sync();
            __syncthreads();
            tc::fence_after_sync();
            if (j == 0) {
                const uint32_t idesc = tc::instr_desc(16);
                const uint32_t sbo = kBwKc * 128;
                for (int step = 0; step < kBwChunk / 16; ++step) {
                    const uint32_t koff = (uint32_t)step * 256;
                    const uint64_t bd = tc::smem_desc(f2_s + koff, 128, sbo);
                    tc::mma_bf16(tmem + kBwAcc0, tc::smem_desc(m_s + koff, 128, sbo), bd, idesc,
                                 chunk > 0 || step > 0);
                    tc::mma_bf16(tmem + kBwAcc1, tc::smem_desc(m_s + (uint32_t)kBwMaskHalf + koff, 128, sbo), bd,
                                 idesc, chunk > 0 || step > 0);
                }
                tc::mma_commit(mbar);
            }
            if (!tc::mbar_wait(mbar, parity)) {
                atomicOr(a.err, 1u);
                s_abort = 1;
            }
            parity ^= 1u;
            tc::fence_after_sync();
            __syncthreads();
            if (s_abort) break;
        }
        if (s_abort) break;
        // this unit's row of Mask x F'^T: hi columns 0-4, bias 5, lo columns 6-10
        float r[32];
        tc::tmem_ld32(t_row + acc_col, r);
        const float g = a.dzt[(long long)t * kMlpIn2 + h] / (float)n;
#pragma unroll
        for (int q = 0; q < kMlpIn1; ++q) gw[q] += g * (r[q] + r[q + kMlpIn1 + 1]);
        gw[kMlpIn1] += g * r[kMlpIn1];
        tc::fence_before_sync();
        __syncthreads();                          // TMEM and shared operands are reused by the next tour
        tc::fence_after_sync();
    }
#pragma unroll
    for (int q = 0; q < kMlpIn1; ++q) atomicAdd(a.gw1 + h * kMlpIn1 + q, gw[q]);
    atomicAdd(a.gb1 + h, gw[kMlpIn1]);
    tc::fence_before_sync();
    __syncthreads();
    if (w == 0) tc::tmem_dealloc(tmem, kTmemCols);
}

}  // namespace

cudaError_t mlp_layer2_tc(const float *zt, int T, const __nv_bfloat16 *w2, const __nv_bfloat16 *b2, float *U,
                          unsigned int *err, cudaStream_t st)
{
    cudaError_t e = cudaFuncSetAttribute(mlp_layer2_tc_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)kL2Smem);
    if (e != cudaSuccess) return e;
    const dim3 grid((unsigned)((T + kL2M - 1) / kL2M), kMlpH / kL2N);
    mlp_layer2_tc_kernel<<<grid, kTcThreads, kL2Smem, st>>>(zt, T, w2, b2, U, err);
    return cudaGetLastError();
}

cudaError_t mlp_layer1_tc(const MlpLayer1Args &l1, int sm_count, cudaStream_t st)
{
    cudaError_t e = cudaFuncSetAttribute(mlp_layer1_tc_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)kTcSmemPad);
    if (e != cudaSuccess) return e;
    const int grid = l1.T < sm_count ? l1.T : sm_count;
    mlp_layer1_tc_kernel<<<grid, kTcThreads, kTcSmemPad, st>>>(l1);
    return cudaGetLastError();
}

// dZT (T x 257) = dU (T x 256) W2 (256 x 257): A = dU, B(n, k) = W2[k][n].
cudaError_t mlp_grad_zt_tc(const float *dU, int T, const __nv_bfloat16 *w2, float *dzt, unsigned int *err,
                           cudaStream_t st)
{
    TcGemm g{};
    g.a = dU;
    g.lda = kMlpH;
    g.bh = w2;
    g.ldb = kMlpIn2;
    g.M = T;
    g.N = kMlpIn2;
    g.K = kMlpH;
    g.k_slab = kMlpH;
    g.out = dzt;
    g.ldo = kMlpIn2;
    g.err = err;
    return tc_gemm<false, true, true, false>(g, st);
}

// gW2 (256 x 257) += dU^T (256 x T) ZT (T x 257): A(m, k) = dU[k][m],
// B(n, k) = ZT[k][n]; split-K over slabs of 128 tours (a CTA per slab and
// tile fills the GPU), added atomically.
cudaError_t mlp_grad_w2_tc(const float *dU, const float *zt, int T, float *gw2, unsigned int *err, cudaStream_t st)
{
    TcGemm g{};
    g.a = dU;
    g.lda = kMlpH;
    g.bf = zt;
    g.ldb = kMlpIn2;
    g.M = kMlpH;
    g.N = kMlpIn2;
    g.K = T;
    g.k_slab = 128;
    g.out = gw2;
    g.ldo = kMlpIn2;
    g.err = err;
    return tc_gemm<true, true, false, true>(g, st);
}

cudaError_t mlp_layer1_bwd_tc(const MlpLayer1Args &l1, int sm_count, cudaStream_t st)
{
    cudaError_t e = cudaFuncSetAttribute(mlp_layer1_bwd_tc_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)kBwSmem);
    if (e != cudaSuccess) return e;
    const int grid = l1.T < sm_count ? l1.T : sm_count;
    mlp_layer1_bwd_tc_kernel<<<grid, kTcThreads, kBwSmem, st>>>(l1);
    return cudaGetLastError();
}

}  // namespace cvrpsd
