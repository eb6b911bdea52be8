// Sequence-parallel Split for few scenarios: the recursion over tour
// positions written as a chain of min-plus matrix products over the graph of
// positions (the abstract frames the Split that way), evaluated in parallel
// along the positions rather than across scenarios.
//
// With g(p) = f(p) + c(0, sigma_{p+1}) - D[p+1] the recursion is
// g(i) = C_i + min_{p in W(i)} g(p). The state after position i is the vector
// x_i = (g(i), g(i-1), ..., g(i-W+1)) of the last W values, and
// x_i = A_i (x) x_{i-1} in the (min, +) semiring: row 0 of A_i holds C_i at the
// columns of the window W(i) = [lo(i), i-1] and +inf elsewhere, the other rows
// shift the state down. The positions are cut into blocks of kSeqBlock; the
// transfer matrix of each block (a kSeqW x kSeqW min-plus matrix) is built
// independently, in parallel over blocks and over its columns; a last pass
// folds the block matrices over the initial state x_0 = (g(0), +inf, ...).
// f(n) comes out as row 0 of the final state, position n using C_n = D[n] +
// c(sigma_n, 0). A scenario whose window is longer than kSeqW, or with a
// demand above Q or below 0, is handed to the warp kernel.
#include <stdint.h>

#include "kernels.h"
#include "tour_table.h"

namespace cvrpsd {

constexpr int kSeqW = 64;        // state width (longest window handled)
constexpr int kSeqBlock = 64;    // positions per block
constexpr int kInf = 0x3FFFFFFF;

__device__ __forceinline__ int sat_add(int a, int b) { return (a >= kInf || b >= kInf) ? kInf : a + b; }

// Window starts: lo[s][i-1] = smallest p >= i - L with P(i) - P(p) <= Q.
// One block per scenario; flags[s] = 1 if the scenario must go elsewhere.
template <typename DT>
__global__ void seqpar_windows_kernel(SeqParParams a)
{
    extern __shared__ int P[];                    // [n + 1] prefix loads
    const int n = a.n, s = blockIdx.x;
    if (s >= a.S) return;
    const DT *dem = reinterpret_cast<const DT *>(a.demand);
    __shared__ int s_bad;
    if (threadIdx.x == 0) s_bad = 0;
    __syncthreads();
    for (int i = 1 + threadIdx.x; i <= n; i += blockDim.x) {
        int q = (int)dem[(long long)(a.tab[i - 1].row & kRowMask) * a.ld + s];
        if (q < 0 || q > a.Q) { atomicOr(&s_bad, 1); q = 0; }
        P[i] = q;
    }
    if (threadIdx.x == 0) P[0] = 0;
    __syncthreads();
    // inclusive scan (one warp walks the chunks; n is at most a few thousand)
    if (threadIdx.x < 32) {
        const int lane = threadIdx.x;
        int carry = 0;
        for (int b = 1; b <= n; b += 32) {
            const int i = b + lane;
            int v = i <= n ? P[i] : 0;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const int t = __shfl_up_sync(0xffffffffu, v, o);
                if (lane >= o) v += t;
            }
            if (i <= n) P[i] = v + carry;
            carry += __shfl_sync(0xffffffffu, v, 31);
        }
    }
    __syncthreads();
    int too_long = 0;
    for (int i = 1 + threadIdx.x; i <= n; i += blockDim.x) {
        int lo = i - a.L > 0 ? i - a.L : 0, hi = i - 1;   // P(i) - P(i-1) <= Q always (bad demands zeroed)
        while (lo < hi) {                                 // first p in [lo, hi] with P(i) - P(p) <= Q
            const int mid = (lo + hi) >> 1;
            if (P[i] - P[mid] <= a.Q) hi = mid; else lo = mid + 1;
        }
        a.lo[(long long)s * n + (i - 1)] = lo;
        too_long |= (i - lo) > kSeqW;
    }
    if (too_long) atomicOr(&s_bad, 2);
    __syncthreads();
    if (threadIdx.x == 0) a.flags[s] = s_bad;
}

// Transfer matrix of block b of scenario s: kSeqW threads, thread j owns
// column j (the image of unit state j). The state is kept per position p in
// a ring (slot p mod kSeqW; windows are at most kSeqW long), and the window
// minimum by the two-stack method: the older part of the window [lo, m) has
// suffix minima SF, the newer part [m, i-1] a running minimum bm. When the
// window start passes m, the suffix minima are rebuilt over the whole window
// and m moves to i. Every column walks the same window starts (they depend
// on the scenario only), so the rebuilds happen at the same positions in all
// threads: O(1) amortised work per position, with no divergence.
__global__ void __launch_bounds__(kSeqW) seqpar_block_kernel(SeqParParams a)
{
    __shared__ int G[kSeqW][kSeqW + 1];           // [slot of position][column]
    __shared__ int SF[kSeqW][kSeqW + 1];          // suffix minima of the older part
    __shared__ int s_lo[kSeqBlock], s_c[kSeqBlock];
    const int s = blockIdx.y, b = blockIdx.x, j = threadIdx.x, n = a.n;
    if (s >= a.S || a.flags[s]) return;
    const int i0 = b * kSeqBlock + 1, i1 = min(n, i0 + kSeqBlock - 1);
    for (int u = j; u < kSeqBlock; u += kSeqW) {
        const int i = i0 + u;
        s_lo[u] = i <= i1 ? a.lo[(long long)s * n + (i - 1)] : 0;
        s_c[u] = i <= i1 ? a.tab[i - 1].c : 0;
    }
    // the unit state: position i0 - 1 - j holds 0, the other kSeqW - 1 earlier
    // positions +inf; all of them form the older part (m = i0)
    for (int r = 0; r < kSeqW; ++r) {
        const int p = i0 - 1 - r;
        G[p & (kSeqW - 1)][j] = r == j ? 0 : kInf;
        SF[p & (kSeqW - 1)][j] = r >= j ? 0 : kInf;      // min over [p, i0 - 1]
    }
    __syncthreads();
    int m = i0, bm = kInf;
    for (int i = i0; i <= i1; ++i) {
        const int lo = s_lo[i - i0];
        if (lo >= m) {                                   // uniform across the block
            int run = kInf;
            for (int p = i - 1; p >= lo; --p) {
                run = min(run, G[p & (kSeqW - 1)][j]);
                SF[p & (kSeqW - 1)][j] = run;
            }
            m = i;
            bm = kInf;
        }
        const int g = sat_add(min(SF[lo & (kSeqW - 1)][j], bm), s_c[i - i0]);
        G[i & (kSeqW - 1)][j] = g;
        bm = min(bm, g);
    }
    // Row r of the block's matrix is position i1 - r. Stored transposed,
    // out[c * kSeqW + r] = M[r][c], so that the fold reads it with unit
    // stride; thread j writes element j of every stored row (coalesced).
    __syncthreads();
    int *out = a.mats + ((long long)s * a.blocks + b) * kSeqW * kSeqW;
    const int slot = (i1 - j) & (kSeqW - 1);
    for (int c = 0; c < kSeqW; ++c) out[c * kSeqW + j] = G[slot][c];
}

__device__ __forceinline__ void cp_async16(uint32_t dst, const void *src)
{
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(dst), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async_commit()
{
    asm volatile("cp.async.commit_group;" ::: "memory");
}
template <int N>
__device__ __forceinline__ void cp_async_wait()
{
    asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory");
}

// Fold the block matrices over x_0 and write f(n). Each (transposed) matrix
// is copied into shared memory with async copies one block ahead of its use.
// 256 threads per scenario: thread (r, q) takes row r of the mat-vec over the
// columns c = q mod 4, and two shuffles combine the four partial minima.
// Shared rows are kFoldPitch ints apart (16-byte aligned for the copies), so
// the 32 lanes of a warp, rows r..r+7 times q = 0..3, hit 32 distinct banks.
constexpr int kFoldThreads = 4 * kSeqW;
constexpr int kFoldPitch = kSeqW + 8;

__global__ void __launch_bounds__(kFoldThreads) seqpar_fold_kernel(SeqParParams a)
{
    __shared__ int x[kSeqW];
    __shared__ __align__(16) int Mt[2][kSeqW * kFoldPitch];
    const int s = blockIdx.x, t = threadIdx.x;
    const int lane = t & 31, q = lane >> 3, r = (t >> 5) * 8 + (lane & 7);
    if (s >= a.S) return;
    if (a.flags[s]) {                              // handed to the warp kernel
        if (t == 0) {
            const unsigned long long idx = atomicAdd(a.acc + ACC_OVERFLOW, 1ull);
            a.list[idx] = s;
        }
        return;
    }
    if (t < kSeqW) x[t] = t == 0 ? a.g0 : kInf;
    auto load = [&](int b) {   // 16-byte chunks of matrix b: coalesced reads, padded rows
        const int *M = a.mats + ((long long)s * a.blocks + b) * kSeqW * kSeqW;
        const uint32_t dst = (uint32_t)__cvta_generic_to_shared(&Mt[b & 1][0]);
        for (int k = t; k < kSeqW * kSeqW / 4; k += kFoldThreads) {
            const int c = k / (kSeqW / 4), part = k % (kSeqW / 4);
            cp_async16(dst + 4u * (c * kFoldPitch + 4 * part), M + 4 * k);
        }
        cp_async_commit();
    };
    load(0);
    for (int b = 0; b < a.blocks; ++b) {
        if (b + 1 < a.blocks) {
            load(b + 1);
            cp_async_wait<1>();    // matrix b has landed (this thread's part)
        } else {
            cp_async_wait<0>();
        }
        __syncthreads();           // every thread's part of matrix b, and x
        const int *M = Mt[b & 1];
        int v = kInf;
#pragma unroll
        for (int k = 0; k < kSeqW / 4; ++k) {
            const int c = 4 * k + q;
            v = min(v, sat_add(M[c * kFoldPitch + r], x[c]));
        }
        v = min(v, __shfl_xor_sync(0xffffffffu, v, 8));
        v = min(v, __shfl_xor_sync(0xffffffffu, v, 16));
        __syncthreads();           // all reads of x and of this buffer are done
        if (q == 0) x[r] = v;
    }
    __syncthreads();
    if (t == 0) {
        const int cost = x[0];
        if (a.out_cost) a.out_cost[s] = cost;
        atomicAdd(a.acc + ACC_SUM, (unsigned long long)cost);
    }
}

cudaError_t launch_seqpar(const SeqParParams &a, int esize, cudaStream_t st)
{
    const size_t smem = (size_t)(a.n + 1) * sizeof(int);
    if (esize == 2) {
        cudaError_t e = cudaFuncSetAttribute(seqpar_windows_kernel<int16_t>,
                                             cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
        seqpar_windows_kernel<int16_t><<<(unsigned)a.S, 1024, smem, st>>>(a);
    } else {
        cudaError_t e = cudaFuncSetAttribute(seqpar_windows_kernel<int32_t>,
                                             cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
        seqpar_windows_kernel<int32_t><<<(unsigned)a.S, 1024, smem, st>>>(a);
    }
    seqpar_block_kernel<<<dim3((unsigned)a.blocks, (unsigned)a.S), kSeqW, 0, st>>>(a);
    seqpar_fold_kernel<<<(unsigned)a.S, kFoldThreads, 0, st>>>(a);
    return cudaGetLastError();
}

int seqpar_blocks(int n) { return (n + kSeqBlock - 1) / kSeqBlock; }
int seqpar_width() { return kSeqW; }

}  // namespace cvrpsd
