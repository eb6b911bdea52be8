// C ABI of the device-side local search around the Split: many candidate
// tours of one instance split at once, neighbour generation, top-k, and the
// surrogate network that screens neighbours (include/cvrpsd.h).
#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <string.h>

#include <cmath>
#include <vector>

#include "ctx.h"
#include "kernels.h"
#include "trace.h"
#include "mlp.h"
#include "tour_table.h"

using namespace cvrpsd;

#define CK(call, what)                                          \
    do {                                                        \
        cudaError_t e_ = (call);                                \
        if (e_ != cudaSuccess) {                                \
            cudaGetLastError();                                 \
            return cuda_fail(ctx, e_, what);                    \
        }                                                       \
    } while (0)

namespace {

template <typename T>
int grow(cvrpsd_ctx *ctx, T **buf, long long *cap, long long need, const char *what)
{
    if (need <= *cap) return CVRPSD_OK;
    if (*buf) cudaFree(*buf);
    *buf = nullptr;
    *cap = 0;
    cudaError_t e = dev_alloc(ctx, buf, sizeof(T) * (size_t)need);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return fail(ctx, CVRPSD_ERR_NOMEM, "%s (%lld entries): %s", what, need, cudaGetErrorString(e));
    }
    *cap = need;
    return CVRPSD_OK;
}

bool is_device_ptr(const void *p, int device)
{
    if (!p) return false;
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return (a.type == cudaMemoryTypeDevice && a.device == device) || a.type == cudaMemoryTypeManaged;
}

}  // namespace

extern "C" {

int cvrpsd_split_eval_tours(cvrpsd_ctx *ctx, const int32_t *d_tours, int32_t T, int32_t n, const int32_t *dist,
                            const void *demand, int32_t demand_dtype, int64_t S, int64_t ld, int32_t Q, int32_t L,
                            double *d_mean, int64_t *d_sum, int64_t *d_infeasible, void *stream_ptr)
{
    CVRPSD_TRACE("cvrpsd_split_eval_tours");
    if (!ctx) return CVRPSD_ERR_ARG;
    ctx->err[0] = 0;
    cudaStream_t stream = reinterpret_cast<cudaStream_t>(stream_ptr);
    if (T < 1 || n < 1 || n > CVRPSD_MAX_N) return fail(ctx, CVRPSD_ERR_ARG, "T = %d, n = %d", T, n);
    if (demand_dtype != CVRPSD_I16 && demand_dtype != CVRPSD_I32) return fail(ctx, CVRPSD_ERR_DTYPE, "dtype");
    if (S < 1 || S > INT32_MAX || ld < S) return fail(ctx, CVRPSD_ERR_ARG, "S = %lld, ld = %lld", (long long)S,
                                                    (long long)ld);
    if (Q < 0 || L < 1) return fail(ctx, CVRPSD_ERR_ARG, "Q = %d, L = %d", Q, L);
    if (!dist) return fail(ctx, CVRPSD_ERR_ARG, "dist is required");
    CK(cudaSetDevice(ctx->device), "cudaSetDevice");
    if (!is_device_ptr(d_tours, ctx->device) || !is_device_ptr(demand, ctx->device))
        return fail(ctx, CVRPSD_ERR_ARG, "tours and demand must be device memory");
    if ((d_mean && !is_device_ptr(d_mean, ctx->device)) || (d_sum && !is_device_ptr(d_sum, ctx->device)) ||
        (d_infeasible && !is_device_ptr(d_infeasible, ctx->device)))
        return fail(ctx, CVRPSD_ERR_ARG, "outputs must be device memory");
    if (L > n) L = n;
    // Bounds that hold for every tour of this instance, and a hash of the
    // matrix (FNV-1a over its words) in the same pass: a search calls this
    // every iteration with the same distances, which are then not uploaded
    // again.
    const long long N1 = (long long)n + 1;
    long long singles = 0, maxd = 0;
    unsigned long long key = 0xcbf29ce484222325ull ^ (unsigned long long)n;
    for (long long k = 0; k < N1 * N1; ++k) {
        if (dist[k] < 0) return fail(ctx, CVRPSD_ERR_ARG, "negative distance");
        maxd = dist[k] > maxd ? dist[k] : maxd;
        key = (key ^ (uint32_t)dist[k]) * 0x100000001b3ull;
    }
    if (key == 0) key = 1;
    for (int c = 1; c <= n; ++c) singles += (long long)dist[c] + dist[(long long)c * N1];
    if (singles + (long long)n * maxd + 3 * maxd >= (1LL << 30))
        return fail(ctx, CVRPSD_ERR_OVERFLOW, "route costs of this instance could overflow int32");
    const uint32_t K = key_scale(n);
    if ((long long)(Q + 1LL) * K + n >= (1LL << 31)) return fail(ctx, CVRPSD_ERR_UNSUPPORTED, "Q too large for n");

    DequeShape shape{256, 1, 16};
    if (ctx->cfg.threads && (ctx->cfg.threads == 128 || ctx->cfg.threads == 256) && ctx->cfg.spt == 1 &&
        (ctx->cfg.ring == 16 || ctx->cfg.ring == 32))
        shape = DequeShape{ctx->cfg.threads, 1, ctx->cfg.ring};
    const long long tiles = (S + shape.threads - 1) / shape.threads;
    if (tiles * T > INT32_MAX) return fail(ctx, CVRPSD_ERR_UNSUPPORTED, "too many work items");
    long long dcap = ctx->mt_descs_cap, acap = ctx->mt_acc_cap;
    int rc = grow(ctx, &ctx->mt_tabs, &ctx->mt_tabs_cap, (long long)T * n, "tour tables");
    if (!rc) rc = grow(ctx, &ctx->mt_descs, &dcap, T, "tour descriptors");
    if (!rc) rc = grow(ctx, &ctx->mt_acc, &acap, BACC_WORDS + 3LL * T, "accumulators");
    if (!rc) rc = grow(ctx, &ctx->mt_list, &ctx->mt_list_cap, std::min<long long>((long long)T * S, 1LL << 24),
                       "set-aside list");
    const bool same_dist = ctx->mt_dist && ctx->mt_dist_key == key && ctx->mt_dist_n == n;
    if (!rc && !same_dist) {
        ctx->mt_dist_key = 0;   // invalid until the new matrix is staged
        rc = grow(ctx, &ctx->mt_dist, &ctx->mt_dist_cap, N1 * N1, "distances");
        if (!rc && ctx->mt_dist_host_cap < N1 * N1) {
            if (ctx->mt_dist_host) cudaFreeHost(ctx->mt_dist_host);
            ctx->mt_dist_host = nullptr;
            ctx->mt_dist_host_cap = 0;
            if (host_alloc(ctx, &ctx->mt_dist_host, sizeof(int32_t) * N1 * N1) != cudaSuccess) {
                cudaGetLastError();
                rc = fail(ctx, CVRPSD_ERR_NOMEM, "pinned distances");
            } else {
                ctx->mt_dist_host_cap = N1 * N1;
            }
        }
    }
    ctx->mt_descs_cap = (int)dcap;
    ctx->mt_acc_cap = (int)acap;
    if (rc) return rc;
    if (!same_dist) {
        if (!ctx->ev_dist) CK(cudaEventCreateWithFlags(&ctx->ev_dist, cudaEventDisableTiming), "cudaEventCreate");
        // The pinned copy may still feed the previous upload (on any stream).
        CK(cudaEventSynchronize(ctx->ev_dist), "cudaEventSynchronize");
        memcpy(ctx->mt_dist_host, dist, sizeof(int32_t) * N1 * N1);
        CK(cudaMemcpyAsync(ctx->mt_dist, ctx->mt_dist_host, sizeof(int32_t) * N1 * N1, cudaMemcpyHostToDevice,
                           stream),
           "upload distances");
        CK(cudaEventRecord(ctx->ev_dist, stream), "cudaEventRecord");
        ctx->mt_dist_key = key;
        ctx->mt_dist_n = n;
    }
    CK(cudaMemsetAsync(ctx->mt_acc, 0, sizeof(unsigned long long) * (BACC_WORDS + 3LL * T), stream),
       "clear accumulators");
    CK(launch_tour_tables(d_tours, T, n, ctx->mt_dist, nullptr, ctx->mt_tabs, ctx->mt_descs, demand, ld, Q,
                          L < n ? L : n + 1, K, stream),
       "tour tables");
    BatchParams bp{};
    bp.tours = ctx->mt_descs;
    bp.items = nullptr;
    bp.tiles = (int)tiles;
    bp.n_items = (int)(tiles * T);
    bp.S = S;
    bp.acc = ctx->mt_acc;
    bp.list = ctx->mt_list;
    bp.list_cap = ctx->mt_list_cap;
    bp.max_n = n;
    bp.walk2 = demand_dtype == CVRPSD_I16 && batch2_keys_fit(n, Q, K);
    int per_sm = 0;
    CK(launch_split_batch(bp, demand_dtype, L < n, shape, 0, true, &per_sm, stream), "configure batch kernel");
    CK(launch_split_batch(bp, demand_dtype, L < n, shape, ctx->sm_count * (per_sm > 0 ? per_sm : 1), false, nullptr,
                          stream),
       "split kernel");
    CK(launch_split_warp_batch(bp, demand_dtype, 2 * ctx->sm_count, ctx->max_smem, true, stream), "configure warp");
    CK(launch_split_warp_batch(bp, demand_dtype, 2 * ctx->sm_count, ctx->max_smem, false, stream), "warp kernel");
    CK(launch_tour_means(ctx->mt_acc, T, S, d_mean, reinterpret_cast<long long *>(d_sum),
                         reinterpret_cast<long long *>(d_infeasible), stream),
       "tour means");
    ctx->stats = cvrpsd_stats{};
    ctx->stats.kernel = CVRPSD_KERNEL_DEQUE;
    ctx->stats.threads = shape.threads;
    ctx->stats.spt = 1;
    ctx->stats.ring = shape.ring;
    ctx->stats.overflow = -1;
    ctx->stats.launches = 4;
    ctx->stats.kernel_ms = ctx->stats.fallback_ms = -1.0f;
    return CVRPSD_OK;
}

int cvrpsd_neighbors(cvrpsd_ctx *ctx, const int32_t *d_base, int32_t n, const int32_t *d_moves, int32_t M,
                     int32_t *d_out, void *stream)
{
    CVRPSD_TRACE("cvrpsd_neighbors");
    if (!ctx) return CVRPSD_ERR_ARG;
    if (n < 1 || M < 0) return fail(ctx, CVRPSD_ERR_ARG, "n = %d, M = %d", n, M);
    if (M == 0) return CVRPSD_OK;
    CK(cudaSetDevice(ctx->device), "cudaSetDevice");
    if (!is_device_ptr(d_base, ctx->device) || !is_device_ptr(d_moves, ctx->device) ||
        !is_device_ptr(d_out, ctx->device))
        return fail(ctx, CVRPSD_ERR_ARG, "base, moves and out must be device memory");
    CK(launch_neighbors(d_base, n, d_moves, M, d_out, reinterpret_cast<cudaStream_t>(stream)), "neighbors");
    return CVRPSD_OK;
}

int cvrpsd_topk(cvrpsd_ctx *ctx, const float *d_scores, int32_t M, int32_t k, int32_t *d_idx, void *stream)
{
    CVRPSD_TRACE("cvrpsd_topk");
    if (!ctx) return CVRPSD_ERR_ARG;
    if (M < 1 || M > 16384 || k < 1 || k > M) return fail(ctx, CVRPSD_ERR_ARG, "M = %d, k = %d", M, k);
    CK(cudaSetDevice(ctx->device), "cudaSetDevice");
    if (!is_device_ptr(d_scores, ctx->device) || !is_device_ptr(d_idx, ctx->device))
        return fail(ctx, CVRPSD_ERR_ARG, "scores and idx must be device memory");
    CK(launch_topk(d_scores, M, k, d_idx, reinterpret_cast<cudaStream_t>(stream)), "topk");
    return CVRPSD_OK;
}

int cvrpsd_gather_tours(cvrpsd_ctx *ctx, const int32_t *d_tours, int32_t rows, int32_t n, const int32_t *d_idx,
                        int32_t R, int32_t *d_out, void *stream)
{
    CVRPSD_TRACE("cvrpsd_gather_tours");
    if (!ctx) return CVRPSD_ERR_ARG;
    if (n < 1 || R < 0 || rows < 1) return fail(ctx, CVRPSD_ERR_ARG, "rows = %d, n = %d, R = %d", rows, n, R);
    if (R == 0) return CVRPSD_OK;
    CK(cudaSetDevice(ctx->device), "cudaSetDevice");
    if (!is_device_ptr(d_tours, ctx->device) || !is_device_ptr(d_idx, ctx->device) ||
        !is_device_ptr(d_out, ctx->device))
        return fail(ctx, CVRPSD_ERR_ARG, "tours, idx and out must be device memory");
    CK(launch_gather_rows(d_tours, rows, n, d_idx, R, d_out, reinterpret_cast<cudaStream_t>(stream)), "gather");
    return CVRPSD_OK;
}

int cvrpsd_accept_best(cvrpsd_ctx *ctx, const int32_t *d_tours, int32_t T, int32_t n, const double *d_cost,
                       int32_t *d_cur, double *d_cur_cost, double *d_trace, void *stream)
{
    CVRPSD_TRACE("cvrpsd_accept_best");
    if (!ctx) return CVRPSD_ERR_ARG;
    if (T < 1 || n < 1) return fail(ctx, CVRPSD_ERR_ARG, "T = %d, n = %d", T, n);
    CK(cudaSetDevice(ctx->device), "cudaSetDevice");
    if (!is_device_ptr(d_tours, ctx->device) || !is_device_ptr(d_cost, ctx->device) ||
        !is_device_ptr(d_cur, ctx->device) || !is_device_ptr(d_cur_cost, ctx->device) ||
        (d_trace && !is_device_ptr(d_trace, ctx->device)))
        return fail(ctx, CVRPSD_ERR_ARG, "tours, cost, cur, cur_cost and trace must be device memory");
    const uintptr_t t0 = (uintptr_t)d_tours, t1 = t0 + (uintptr_t)T * (uintptr_t)n * sizeof(int32_t);
    const uintptr_t c0 = (uintptr_t)d_cur, c1 = c0 + (uintptr_t)n * sizeof(int32_t);
    if (c0 < t1 && t0 < c1) return fail(ctx, CVRPSD_ERR_ARG, "cur overlaps the candidate tours");
    CK(launch_accept_best(d_tours, T, n, d_cost, d_cur, d_cur_cost, d_trace, reinterpret_cast<cudaStream_t>(stream)),
       "accept");
    return CVRPSD_OK;
}

}  // extern "C"

// ------------------------------------------------------------ surrogate

struct cvrpsd_surrogate {
    cvrpsd_ctx *ctx = nullptr;
    int n = 0;
    float *d_cust = nullptr;       // [n][4] normalised
    int32_t *d_dist = nullptr;     // (n+1)^2
    float *d_p = nullptr, *d_g = nullptr, *d_m = nullptr, *d_v = nullptr;
    __nv_bfloat16 *d_pb = nullptr;
    long long cap = 0;             // workspace rows
    float *d_zt = nullptr, *d_U = nullptr, *d_y = nullptr, *d_dy = nullptr, *d_dU = nullptr, *d_dzt = nullptr;
    float *d_loss = nullptr;
    unsigned int *d_err = nullptr;  // set by a tensor-core kernel whose wait gave up
    int step = 0;
    float len_mean = 0.0f, len_inv_sd = 1.0f;
};

namespace {

void sur_free(cvrpsd_surrogate *s)
{
    if (!s) return;
    for (void *p : {(void *)s->d_cust, (void *)s->d_dist, (void *)s->d_p, (void *)s->d_g, (void *)s->d_m,
                    (void *)s->d_v, (void *)s->d_pb, (void *)s->d_zt, (void *)s->d_U, (void *)s->d_y,
                    (void *)s->d_dy, (void *)s->d_dU, (void *)s->d_dzt, (void *)s->d_loss, (void *)s->d_err})
        if (p) cudaFree(p);
    delete s;
}

int sur_workspace(cvrpsd_surrogate *s, long long T)
{
    cvrpsd_ctx *ctx = s->ctx;
    if (T <= s->cap) return CVRPSD_OK;
    // The old buffers go first; until all new ones exist the capacity is 0,
    // so a failed call leaves nothing that a later call could mistake for room.
    s->cap = 0;
    for (float **p : {&s->d_zt, &s->d_U, &s->d_y, &s->d_dy, &s->d_dU, &s->d_dzt}) {
        if (*p) cudaFree(*p);
        *p = nullptr;
    }
    CK(dev_alloc(ctx, &s->d_zt, sizeof(float) * T * kMlpIn2), "surrogate workspace");
    CK(dev_alloc(ctx, &s->d_U, sizeof(float) * T * kMlpH), "surrogate workspace");
    CK(dev_alloc(ctx, &s->d_y, sizeof(float) * T), "surrogate workspace");
    CK(dev_alloc(ctx, &s->d_dy, sizeof(float) * T), "surrogate workspace");
    CK(dev_alloc(ctx, &s->d_dU, sizeof(float) * T * kMlpH), "surrogate workspace");
    CK(dev_alloc(ctx, &s->d_dzt, sizeof(float) * T * kMlpIn2), "surrogate workspace");
    s->cap = T;
    return CVRPSD_OK;
}

MlpWeights weights_of(const cvrpsd_surrogate *s)
{
    MlpWeights w;
    w.w1 = s->d_pb + kOffW1;
    w.b1 = s->d_pb + kOffB1;
    w.w2 = s->d_pb + kOffW2;
    w.b2 = s->d_pb + kOffB2;
    w.w3 = s->d_pb + kOffW3;
    w.b3 = s->d_pb + kOffB3;
    return w;
}

MlpLayer1Args layer1_of(const cvrpsd_surrogate *s, const int32_t *tours, int T)
{
    MlpLayer1Args a{};
    a.tours = tours;
    a.T = T;
    a.n = s->n;
    a.cust = s->d_cust;
    a.dist = s->d_dist;
    a.w1 = s->d_pb + kOffW1;
    a.b1 = s->d_pb + kOffB1;
    a.len_mean = s->len_mean;
    a.len_inv_sd = s->len_inv_sd;
    a.zt = s->d_zt;
    a.err = s->d_err;
    a.sm_count = s->ctx->sm_count > 0 ? s->ctx->sm_count : 1;
    return a;
}

// A tensor-core kernel of an earlier call on this network gave up waiting
// for its MMAs (read after the device has finished that work).
int sur_device_error(cvrpsd_surrogate *s)
{
    cvrpsd_ctx *ctx = s->ctx;
    unsigned int h = 0;
    CK(cudaMemcpy(&h, s->d_err, sizeof(h), cudaMemcpyDeviceToHost), "read status");
    if (h) return fail(ctx, CVRPSD_ERR_TIMEOUT, "a tensor-core wait of the surrogate gave up");
    return CVRPSD_OK;
}

int sur_check(cvrpsd_surrogate *s, const int32_t *d_tours, int32_t T)
{
    cvrpsd_ctx *ctx = s->ctx;
    if (T < 1) return fail(ctx, CVRPSD_ERR_ARG, "T = %d", T);
    CK(cudaSetDevice(ctx->device), "cudaSetDevice");
    if (!is_device_ptr(d_tours, ctx->device)) return fail(ctx, CVRPSD_ERR_ARG, "tours must be device memory");
    return sur_workspace(s, T);
}

}  // namespace

extern "C" {

int cvrpsd_surrogate_create(cvrpsd_ctx *ctx, int32_t n, const float *cust, const int32_t *dist, float Q, uint64_t seed,
                            cvrpsd_surrogate **out)
{
    CVRPSD_TRACE("cvrpsd_surrogate_create");
    if (!ctx || !out) return CVRPSD_ERR_ARG;
    *out = nullptr;
    if (n < 1 || n > 4096 || !cust || !dist || !(Q > 0))
        return fail(ctx, CVRPSD_ERR_ARG, "surrogate needs 1 <= n <= 4096, features, distances and Q > 0");
    CK(cudaSetDevice(ctx->device), "cudaSetDevice");
    cvrpsd_surrogate *s = new (std::nothrow) cvrpsd_surrogate();
    if (!s) return CVRPSD_ERR_NOMEM;
    s->ctx = ctx;
    s->n = n;
    s->len_mean = 0.0f;
    s->len_inv_sd = 1.0f / (500.0f * (float)n);
    std::vector<float> c((size_t)n * 4);
    for (int k = 0; k < n; ++k) {
        c[4 * k + 0] = cust[4 * k + 0] / 1000.0f;
        c[4 * k + 1] = cust[4 * k + 1] / 1000.0f;
        c[4 * k + 2] = cust[4 * k + 2] / Q;
        c[4 * k + 3] = cust[4 * k + 3] / Q;
    }
    // Parameters: uniform(-1/sqrt(fan_in), 1/sqrt(fan_in)) from a SplitMix64 stream.
    std::vector<float> p((size_t)kMlpParams);
    uint64_t st = seed;
    auto uni = [&st]() {
        st += 0x9E3779B97F4A7C15ull;
        uint64_t z = st;
        z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
        z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
        z ^= z >> 31;
        return (double)(z >> 11) * (1.0 / 9007199254740992.0) * 2.0 - 1.0;
    };
    auto fill = [&](long long off, long long cnt, int fan_in) {
        const double bound = 1.0 / std::sqrt((double)fan_in);
        for (long long i = 0; i < cnt; ++i) p[off + i] = (float)(uni() * bound);
    };
    fill(kOffW1, (long long)kMlpH * kMlpIn1, kMlpIn1);
    fill(kOffB1, kMlpH, kMlpIn1);
    fill(kOffW2, (long long)kMlpH * kMlpIn2, kMlpIn2);
    fill(kOffB2, kMlpH, kMlpIn2);
    fill(kOffW3, kMlpH, kMlpH);
    fill(kOffB3, 1, kMlpH);
    const long long N1 = (long long)n + 1;
#define SK(call, what)                          \
    do {                                        \
        cudaError_t e_ = (call);                \
        if (e_ != cudaSuccess) {                \
            cudaGetLastError();                 \
            sur_free(s);                        \
            return cuda_fail(ctx, e_, what);    \
        }                                       \
    } while (0)
    SK(dev_alloc(ctx, &s->d_cust, sizeof(float) * n * 4), "cudaMalloc");
    SK(dev_alloc(ctx, &s->d_dist, sizeof(int32_t) * N1 * N1), "cudaMalloc");
    SK(dev_alloc(ctx, &s->d_p, sizeof(float) * kMlpParams), "cudaMalloc");
    SK(dev_alloc(ctx, &s->d_g, sizeof(float) * kMlpParams), "cudaMalloc");
    SK(dev_alloc(ctx, &s->d_m, sizeof(float) * kMlpParams), "cudaMalloc");
    SK(dev_alloc(ctx, &s->d_v, sizeof(float) * kMlpParams), "cudaMalloc");
    SK(dev_alloc(ctx, &s->d_pb, sizeof(__nv_bfloat16) * kMlpParams), "cudaMalloc");
    SK(dev_alloc(ctx, &s->d_loss, sizeof(float)), "cudaMalloc");
    SK(dev_alloc(ctx, &s->d_err, sizeof(unsigned int)), "cudaMalloc");
    SK(cudaMemset(s->d_err, 0, sizeof(unsigned int)), "memset");
    SK(cudaMemcpy(s->d_cust, c.data(), sizeof(float) * n * 4, cudaMemcpyHostToDevice), "upload");
    SK(cudaMemcpy(s->d_dist, dist, sizeof(int32_t) * N1 * N1, cudaMemcpyHostToDevice), "upload");
    SK(cudaMemcpy(s->d_p, p.data(), sizeof(float) * kMlpParams, cudaMemcpyHostToDevice), "upload");
    SK(cudaMemset(s->d_m, 0, sizeof(float) * kMlpParams), "memset");
    SK(cudaMemset(s->d_v, 0, sizeof(float) * kMlpParams), "memset");
    SK(mlp_to_bf16(s->d_p, s->d_pb, nullptr), "bf16 copy");
    SK(cudaDeviceSynchronize(), "synchronize");
#undef SK
    *out = s;
    return CVRPSD_OK;
}

int cvrpsd_surrogate_destroy(cvrpsd_surrogate *s)
{
    if (!s) return CVRPSD_ERR_ARG;
    cudaSetDevice(s->ctx->device);
    sur_free(s);
    return CVRPSD_OK;
}

int cvrpsd_surrogate_predict(cvrpsd_surrogate *s, const int32_t *d_tours, int32_t T, float *d_pred, void *stream_ptr)
{
    CVRPSD_TRACE("cvrpsd_surrogate_predict");
    if (!s) return CVRPSD_ERR_ARG;
    cvrpsd_ctx *ctx = s->ctx;
    int rc = sur_check(s, d_tours, T);
    if (rc) return rc;
    if (!is_device_ptr(d_pred, ctx->device)) return fail(ctx, CVRPSD_ERR_ARG, "pred must be device memory");
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream_ptr);
    CK(mlp_forward(layer1_of(s, d_tours, T), weights_of(s), s->d_U, d_pred, nullptr, nullptr, nullptr, st),
       "surrogate forward");
    return CVRPSD_OK;
}

static int sur_grad(cvrpsd_surrogate *s, const int32_t *d_tours, int32_t T, const float *d_target, cudaStream_t st)
{
    cvrpsd_ctx *ctx = s->ctx;
    CK(cudaMemsetAsync(s->d_g, 0, sizeof(float) * kMlpParams, st), "clear gradient");
    CK(cudaMemsetAsync(s->d_loss, 0, sizeof(float), st), "clear loss");
    const MlpLayer1Args l1 = layer1_of(s, d_tours, T);
    const MlpWeights w = weights_of(s);
    CK(mlp_forward(l1, w, s->d_U, s->d_y, d_target, s->d_dy, s->d_loss, st), "surrogate forward");
    CK(mlp_backward(l1, w, s->d_U, s->d_dy, s->d_dU, s->d_dzt, s->d_g, st), "surrogate backward");
    return CVRPSD_OK;
}

int cvrpsd_surrogate_train_step(cvrpsd_surrogate *s, const int32_t *d_tours, int32_t T, const float *d_target,
                                float lr, float *d_loss, void *stream_ptr)
{
    CVRPSD_TRACE("cvrpsd_surrogate_train_step");
    if (!s) return CVRPSD_ERR_ARG;
    cvrpsd_ctx *ctx = s->ctx;
    int rc = sur_check(s, d_tours, T);
    if (rc) return rc;
    if (!is_device_ptr(d_target, ctx->device)) return fail(ctx, CVRPSD_ERR_ARG, "targets must be device memory");
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream_ptr);
    rc = sur_grad(s, d_tours, T, d_target, st);
    if (rc) return rc;
    s->step += 1;
    CK(mlp_adam(s->d_p, s->d_g, s->d_m, s->d_v, s->d_pb, lr, s->step, st), "adam");
    if (d_loss) CK(cudaMemcpyAsync(d_loss, s->d_loss, sizeof(float), cudaMemcpyDeviceToDevice, st), "loss");
    return CVRPSD_OK;
}

int cvrpsd_surrogate_gradients(cvrpsd_surrogate *s, const int32_t *d_tours, int32_t T, const float *d_target,
                               float *h_grad, float *h_loss)
{
    CVRPSD_TRACE("cvrpsd_surrogate_gradients");
    if (!s || !h_grad) return CVRPSD_ERR_ARG;
    cvrpsd_ctx *ctx = s->ctx;
    int rc = sur_check(s, d_tours, T);
    if (rc) return rc;
    if (!is_device_ptr(d_target, ctx->device)) return fail(ctx, CVRPSD_ERR_ARG, "targets must be device memory");
    rc = sur_grad(s, d_tours, T, d_target, nullptr);
    if (rc) return rc;
    CK(cudaMemcpy(h_grad, s->d_g, sizeof(float) * kMlpParams, cudaMemcpyDeviceToHost), "read gradient");
    if (h_loss) CK(cudaMemcpy(h_loss, s->d_loss, sizeof(float), cudaMemcpyDeviceToHost), "read loss");
    return sur_device_error(s);
}

int cvrpsd_surrogate_set_scale(cvrpsd_surrogate *s, float len_mean, float len_sd)
{
    if (!s) return CVRPSD_ERR_ARG;
    if (!(len_sd > 0.0f)) return fail(s->ctx, CVRPSD_ERR_ARG, "len_sd must be > 0");
    s->len_mean = len_mean;
    s->len_inv_sd = 1.0f / len_sd;
    return CVRPSD_OK;
}

int cvrpsd_surrogate_params(cvrpsd_surrogate *s, float *h_get, const float *h_set, int64_t *count)
{
    if (!s) return CVRPSD_ERR_ARG;
    cvrpsd_ctx *ctx = s->ctx;
    CK(cudaSetDevice(ctx->device), "cudaSetDevice");
    if (count) *count = kMlpParams;
    if (h_set) {
        CK(cudaMemcpy(s->d_p, h_set, sizeof(float) * kMlpParams, cudaMemcpyHostToDevice), "set parameters");
        CK(mlp_to_bf16(s->d_p, s->d_pb, nullptr), "bf16 copy");
        CK(cudaDeviceSynchronize(), "synchronize");
    }
    if (h_get) CK(cudaMemcpy(h_get, s->d_p, sizeof(float) * kMlpParams, cudaMemcpyDeviceToHost), "get parameters");
    return CVRPSD_OK;
}

// Layout of a surrogate checkpoint (host memory, native byte order).
struct SurrogateStateHeader {
    uint32_t magic;       // kSurrogateStateMagic
    uint32_t version;     // 1
    int32_t n;            // customers of the instance the network was built for
    int32_t params;       // kMlpParams
    int32_t step;         // Adam steps taken
    float len_mean;       // tour-length input scale
    float len_inv_sd;
    int32_t reserved;
};
constexpr uint32_t kSurrogateStateMagic = 0x53504443u;

int cvrpsd_surrogate_state(cvrpsd_surrogate *s, void *h_get, const void *h_set, int64_t *bytes)
{
    CVRPSD_TRACE("cvrpsd_surrogate_state");
    if (!s) return CVRPSD_ERR_ARG;
    cvrpsd_ctx *ctx = s->ctx;
    const size_t arr = sizeof(float) * (size_t)kMlpParams;
    const size_t total = sizeof(SurrogateStateHeader) + 3 * arr;
    if (bytes) *bytes = (int64_t)total;
    CK(cudaSetDevice(ctx->device), "cudaSetDevice");
    if (h_set) {
        SurrogateStateHeader h;
        memcpy(&h, h_set, sizeof(h));
        if (h.magic != kSurrogateStateMagic || h.version != 1)
            return fail(ctx, CVRPSD_ERR_ARG, "not a surrogate checkpoint (magic %08x, version %u)", h.magic, h.version);
        if (h.n != s->n || h.params != kMlpParams)
            return fail(ctx, CVRPSD_ERR_ARG, "checkpoint of a network for n = %d (%d parameters), this one has n = %d",
                        h.n, h.params, s->n);
        if (h.step < 0 || !(h.len_inv_sd > 0.0f))
            return fail(ctx, CVRPSD_ERR_ARG, "checkpoint header out of range");
        const char *src = static_cast<const char *>(h_set) + sizeof(h);
        CK(cudaMemcpy(s->d_p, src, arr, cudaMemcpyHostToDevice), "restore parameters");
        CK(cudaMemcpy(s->d_m, src + arr, arr, cudaMemcpyHostToDevice), "restore first moments");
        CK(cudaMemcpy(s->d_v, src + 2 * arr, arr, cudaMemcpyHostToDevice), "restore second moments");
        CK(mlp_to_bf16(s->d_p, s->d_pb, nullptr), "bf16 copy");
        CK(cudaDeviceSynchronize(), "synchronize");
        s->step = h.step;
        s->len_mean = h.len_mean;
        s->len_inv_sd = h.len_inv_sd;
    }
    if (h_get) {
        CK(cudaDeviceSynchronize(), "synchronize");
        SurrogateStateHeader h{kSurrogateStateMagic, 1u, s->n, (int32_t)kMlpParams, s->step, s->len_mean,
                               s->len_inv_sd, 0};
        char *dst = static_cast<char *>(h_get);
        memcpy(dst, &h, sizeof(h));
        CK(cudaMemcpy(dst + sizeof(h), s->d_p, arr, cudaMemcpyDeviceToHost), "save parameters");
        CK(cudaMemcpy(dst + sizeof(h) + arr, s->d_m, arr, cudaMemcpyDeviceToHost), "save first moments");
        CK(cudaMemcpy(dst + sizeof(h) + 2 * arr, s->d_v, arr, cudaMemcpyDeviceToHost), "save second moments");
    }
    return CVRPSD_OK;
}

}  // extern "C"
