// C ABI of the scenario-batched Split (include/cvrpsd.h): argument checks,
// the per-tour position table, the launch plan and the exact host outputs.
#include <cuda.h>
#include <cuda_runtime.h>
#include <stdarg.h>
#include <stdio.h>
#include <string.h>

#include <algorithm>
#include <cmath>
#include <mutex>
#include <string>
#include <vector>

#include "../../include/cvrpsd.h"
#include "ctx.h"
#include "deque2.h"
#include "kernels.h"
#include "trace.h"
#include "tour_table.h"

using namespace cvrpsd;

namespace {

#define CK(call, what)                                     \
    do {                                                   \
        cudaError_t e_ = (call);                           \
        if (e_ != cudaSuccess) return cuda_fail(ctx, e_, what); \
    } while (0)

typedef CUresult (*GetRangeFn)(CUdeviceptr *, size_t *, CUdeviceptr);

GetRangeFn get_range_fn()
{
    static GetRangeFn fn = nullptr;
    static std::once_flag once;
    std::call_once(once, [] {
        void *p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuMemGetAddressRange", &p, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<GetRangeFn>(p);
        else
            cudaGetLastError();
    });
    return fn;
}

// The buffer [ptr, ptr + bytes) must be device memory of ctx->device inside one
// allocation, so that no kernel of this library can read or write past it.
int check_device_buffer(cvrpsd_ctx *ctx, const void *ptr, unsigned long long bytes, const char *what)
{
    if (!ptr) return fail(ctx, CVRPSD_ERR_ARG, "%s is NULL", what);
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, ptr) != cudaSuccess) {
        cudaGetLastError();
        return fail(ctx, CVRPSD_ERR_ARG, "%s is not a CUDA pointer", what);
    }
    if (a.type != cudaMemoryTypeDevice && a.type != cudaMemoryTypeManaged)
        return fail(ctx, CVRPSD_ERR_ARG, "%s must be device memory", what);
    if (a.type == cudaMemoryTypeDevice && a.device != ctx->device)
        return fail(ctx, CVRPSD_ERR_ARG, "%s lives on device %d, context is on %d", what, a.device, ctx->device);
    if (GetRangeFn fn = get_range_fn()) {
        CUdeviceptr base = 0;
        size_t size = 0;
        if (fn(&base, &size, (CUdeviceptr)ptr) == CUDA_SUCCESS) {
            const unsigned long long end = (unsigned long long)(uintptr_t)ptr + bytes;
            if (end > (unsigned long long)base + size)
                return fail(ctx, CVRPSD_ERR_ARG, "%s: %llu bytes needed, allocation ends after %llu", what, bytes,
                            (unsigned long long)(base + size - (CUdeviceptr)ptr));
        }
    }
    return CVRPSD_OK;
}

// The buffer [ptr, ptr + bytes) must be page-locked host memory mapped into
// the device's address space (cudaHostAlloc, cudaMallocHost, or
// cudaHostRegister with cudaHostRegisterMapped); *dev gets the address the
// kernels use. The extent is checked wherever the driver reports the
// allocation's range.
int check_host_buffer(cvrpsd_ctx *ctx, const void *ptr, unsigned long long bytes, const char *what, void **dev)
{
    if (!ptr) return fail(ctx, CVRPSD_ERR_ARG, "%s is NULL", what);
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, ptr) != cudaSuccess) {
        cudaGetLastError();
        return fail(ctx, CVRPSD_ERR_ARG, "%s is not known to CUDA", what);
    }
    if (a.type != cudaMemoryTypeHost || !a.devicePointer)
        return fail(ctx, CVRPSD_ERR_ARG, "%s must be page-locked, mapped host memory (cudaHostAlloc or "
                                         "cudaHostRegister)", what);
    if (GetRangeFn fn = get_range_fn()) {
        CUdeviceptr base = 0;
        size_t size = 0;
        if (fn(&base, &size, (CUdeviceptr)a.devicePointer) == CUDA_SUCCESS) {
            const unsigned long long end = (unsigned long long)(uintptr_t)a.devicePointer + bytes;
            if (end > (unsigned long long)base + size)
                return fail(ctx, CVRPSD_ERR_ARG, "%s: %llu bytes needed, allocation ends after %llu", what, bytes,
                            (unsigned long long)(base + size - (CUdeviceptr)a.devicePointer));
        }
    }
    *dev = a.devicePointer;
    return CVRPSD_OK;
}

int ensure_scratch(cvrpsd_ctx *ctx, long long S)
{
    // Each resource on its own: after a failed allocation the next call
    // retries only what is still missing.
    if (!ctx->d_acc) {
        CK(dev_alloc(ctx, &ctx->d_acc, ACC_ALLOC_WORDS * sizeof(unsigned long long)), "cudaMalloc(acc)");
        // the sticky status word starts clear and is never zeroed per call
        CK(cudaMemset(ctx->d_acc, 0, ACC_ALLOC_WORDS * sizeof(unsigned long long)), "clear accumulators");
    }
    if (!ctx->h_acc) CK(host_alloc(ctx, &ctx->h_acc, ACC_ALLOC_WORDS * sizeof(unsigned long long)), "cudaMallocHost(acc)");
    if (!ctx->d_tab) CK(dev_alloc(ctx, &ctx->d_tab, (CVRPSD_MAX_N + 1) * sizeof(TourStep)), "cudaMalloc(tab)");
    if (!ctx->h_tab) CK(host_alloc(ctx, &ctx->h_tab, (CVRPSD_MAX_N + 1) * sizeof(TourStep)), "cudaMallocHost(tab)");
    if (!ctx->ev_tab) CK(cudaEventCreateWithFlags(&ctx->ev_tab, cudaEventDisableTiming), "cudaEventCreate");
    if (S > ctx->list_cap) {
        if (ctx->d_list) cudaFree(ctx->d_list);
        ctx->d_list = nullptr;
        ctx->list_cap = 0;
        long long cap = S < 4096 ? 4096 : S;
        cudaError_t e = dev_alloc(ctx, &ctx->d_list, (size_t)cap * sizeof(int32_t));
        if (e != cudaSuccess) {
            cudaGetLastError();
            return fail(ctx, CVRPSD_ERR_NOMEM, "overflow list of %lld entries: %s", cap, cudaGetErrorString(e));
        }
        ctx->list_cap = cap;
    }
    return CVRPSD_OK;
}

// Table of one tour (see tour_table.h), with the message kept on the context.
int build_tour_table(cvrpsd_ctx *ctx, const int32_t *tour, int n, const int32_t *dist, int Q, TourStep *tab,
                     int32_t *g0)
{
    char msg[256] = {0};
    const int rc = fill_tour_table(tour, n, dist, Q, tab, g0, msg, sizeof(msg));
    return rc ? fail(ctx, rc, "%s", msg) : CVRPSD_OK;
}

bool valid_shape(int threads, int spt, int ring)
{
    return (threads == 64 || threads == 128 || threads == 256 || threads == 512) && (spt == 1 || spt == 2) &&
           (ring == 8 || ring == 16 || ring == 32 || ring == 64);
}

}  // namespace

extern "C" {

const char *cvrpsd_version(void) { return "cvrpsd-gb300 0.1 (sm_103a)"; }

const char *cvrpsd_strerror(int code)
{
    switch (code) {
    case CVRPSD_OK: return "ok";
    case CVRPSD_WARN_INFEASIBLE: return "some scenarios have no feasible split";
    case CVRPSD_ERR_ARG: return "invalid argument";
    case CVRPSD_ERR_DTYPE: return "unsupported demand type";
    case CVRPSD_ERR_OVERFLOW: return "costs could overflow int32";
    case CVRPSD_ERR_CUDA: return "CUDA error";
    case CVRPSD_ERR_DEVICE_STATUS: return "a kernel reported invalid input";
    case CVRPSD_ERR_NOMEM: return "out of device memory";
    case CVRPSD_ERR_UNSUPPORTED: return "size beyond the library's limits";
    case CVRPSD_ERR_TIMEOUT: return "a device-side wait gave up";
    default: return "unknown status";
    }
}

const char *cvrpsd_last_error(const cvrpsd_ctx *ctx) { return ctx ? ctx->err : "no context"; }

int cvrpsd_create(cvrpsd_ctx **out, int device)
{
    CVRPSD_TRACE("cvrpsd_create");
    if (!out) return CVRPSD_ERR_ARG;
    *out = nullptr;
    int count = 0;
    cudaError_t e = cudaGetDeviceCount(&count);
    if (e != cudaSuccess || device < 0 || device >= count) {
        cudaGetLastError();
        return CVRPSD_ERR_CUDA;
    }
    cvrpsd_ctx *ctx = new (std::nothrow) cvrpsd_ctx();
    if (!ctx) return CVRPSD_ERR_NOMEM;
    ctx->device = device;
    if (cudaSetDevice(device) != cudaSuccess ||
        cudaDeviceGetAttribute(&ctx->sm_count, cudaDevAttrMultiProcessorCount, device) != cudaSuccess ||
        cudaDeviceGetAttribute(&ctx->max_smem, cudaDevAttrMaxSharedMemoryPerBlockOptin, device) != cudaSuccess) {
        cudaGetLastError();
        delete ctx;
        return CVRPSD_ERR_CUDA;
    }
    *out = ctx;
    return CVRPSD_OK;
}

int cvrpsd_destroy(cvrpsd_ctx *ctx)
{
    CVRPSD_TRACE("cvrpsd_destroy");
    if (!ctx) return CVRPSD_ERR_ARG;
    cudaSetDevice(ctx->device);
    if (ctx->d_acc) cudaFree(ctx->d_acc);
    if (ctx->d_list) cudaFree(ctx->d_list);
    if (ctx->d_tab) cudaFree(ctx->d_tab);
    if (ctx->d_gen) cudaFree(ctx->d_gen);
    if (ctx->h_tab) cudaFreeHost(ctx->h_tab);
    if (ctx->h_acc) cudaFreeHost(ctx->h_acc);
    if (ctx->h_gen) cudaFreeHost(ctx->h_gen);
    if (ctx->ev_tab) cudaEventDestroy(ctx->ev_tab);
    if (ctx->ev_gen) cudaEventDestroy(ctx->ev_gen);
    if (ctx->ev_dist) cudaEventDestroy(ctx->ev_dist);
    for (cudaEvent_t e : ctx->ev_t)
        if (e) cudaEventDestroy(e);
    if (ctx->mt_tabs) cudaFree(ctx->mt_tabs);
    if (ctx->mt_descs) cudaFree(ctx->mt_descs);
    if (ctx->mt_acc) cudaFree(ctx->mt_acc);
    if (ctx->mt_list) cudaFree(ctx->mt_list);
    if (ctx->mt_dist) cudaFree(ctx->mt_dist);
    if (ctx->mt_dist_host) cudaFreeHost(ctx->mt_dist_host);
    if (ctx->seq_lo) cudaFree(ctx->seq_lo);
    if (ctx->seq_flags) cudaFree(ctx->seq_flags);
    if (ctx->seq_mats) cudaFree(ctx->seq_mats);
    delete ctx;
    return CVRPSD_OK;
}

int cvrpsd_set_config(cvrpsd_ctx *ctx, const cvrpsd_config *cfg)
{
    if (!ctx || !cfg) return CVRPSD_ERR_ARG;
    if (cfg->kernel < CVRPSD_KERNEL_AUTO || cfg->kernel > CVRPSD_KERNEL_SEQPAR)
        return fail(ctx, CVRPSD_ERR_ARG, "kernel %d unknown", cfg->kernel);
    const bool any_shape = cfg->threads || cfg->spt || cfg->ring;
    if (any_shape && !valid_shape(cfg->threads, cfg->spt, cfg->ring))
        return fail(ctx, CVRPSD_ERR_ARG, "shape threads=%d spt=%d ring=%d not supported", cfg->threads, cfg->spt,
                    cfg->ring);
    if (cfg->variant < CVRPSD_WALK_AUTO || cfg->variant > CVRPSD_WALK_PARAM_TABLE)
        return fail(ctx, CVRPSD_ERR_ARG, "walk variant %d unknown", cfg->variant);
    if (cfg->rounds < 0 || cfg->rounds > 1024) return fail(ctx, CVRPSD_ERR_ARG, "rounds = %d outside 0..1024", cfg->rounds);
    ctx->cfg = *cfg;
    return CVRPSD_OK;
}

int cvrpsd_get_config(const cvrpsd_ctx *ctx, cvrpsd_config *cfg)
{
    if (!ctx || !cfg) return CVRPSD_ERR_ARG;
    *cfg = ctx->cfg;
    return CVRPSD_OK;
}

int cvrpsd_last_stats(const cvrpsd_ctx *ctx, cvrpsd_stats *stats)
{
    if (!ctx || !stats) return CVRPSD_ERR_ARG;
    *stats = ctx->stats;
    return CVRPSD_OK;
}

int cvrpsd_debug_fail_alloc(cvrpsd_ctx *ctx, int32_t after)
{
    if (!ctx) return CVRPSD_ERR_ARG;
    ctx->fail_alloc_after = after < 0 ? -1 : after;
    return CVRPSD_OK;
}

int cvrpsd_set_profiling(cvrpsd_ctx *ctx, int32_t on)
{
    if (!ctx) return CVRPSD_ERR_ARG;
    if (on && !ctx->ev_t[0]) {
        CK(cudaSetDevice(ctx->device), "cudaSetDevice");
        for (cudaEvent_t &e : ctx->ev_t) CK(cudaEventCreate(&e), "cudaEventCreate");
    }
    ctx->profiling = on ? 1 : 0;
    return CVRPSD_OK;
}

int cvrpsd_set_log(cvrpsd_ctx *ctx, cvrpsd_log_fn fn, void *user, int32_t max_level)
{
    if (!ctx) return CVRPSD_ERR_ARG;
    ctx->log_fn = fn;
    ctx->log_user = user;
    ctx->log_level = fn ? max_level : -1;
    return CVRPSD_OK;
}

int cvrpsd_check_inputs(cvrpsd_ctx *ctx, void *stream_ptr)
{
    CVRPSD_TRACE("cvrpsd_check_inputs");
    if (!ctx) return CVRPSD_ERR_ARG;
    ctx->err[0] = 0;
    if (!ctx->d_acc || !ctx->h_acc) return CVRPSD_OK;   // no Split has run on this context
    cudaStream_t stream = reinterpret_cast<cudaStream_t>(stream_ptr);
    CK(cudaSetDevice(ctx->device), "cudaSetDevice");
    CK(cudaMemcpyAsync(ctx->h_acc + ACC_STICKY, ctx->d_acc + ACC_STICKY, sizeof(unsigned long long),
                       cudaMemcpyDeviceToHost, stream),
       "read status");
    CK(cudaMemsetAsync(ctx->d_acc + ACC_STICKY, 0, sizeof(unsigned long long), stream), "clear status");
    CK(cudaStreamSynchronize(stream), "cudaStreamSynchronize");
    if (ctx->h_acc[ACC_STICKY] & ST_NEGATIVE_DEMAND)
        return fail(ctx, CVRPSD_ERR_DEVICE_STATUS, "negative demand found by a Split since the last check");
    return CVRPSD_OK;
}

}  // extern "C"

namespace {

int split_eval_impl(cvrpsd_ctx *ctx, const int32_t *tour, int32_t n, const int32_t *dist, const void *demand,
                    int32_t demand_dtype, int64_t S, int64_t ld, int32_t Q, int32_t L, int32_t *out_cost,
                    int64_t *out_sum, int64_t *out_infeasible, double *out_mean, void *stream_ptr, int16_t *pred,
                    int64_t ldp, bool host_buffers = false)
{
    if (!ctx) return CVRPSD_ERR_ARG;
    ctx->err[0] = 0;
    cudaStream_t stream = reinterpret_cast<cudaStream_t>(stream_ptr);
    if (n < 1 || n > CVRPSD_MAX_N) return fail(ctx, CVRPSD_ERR_ARG, "n = %d outside 1..%d", n, CVRPSD_MAX_N);
    if (demand_dtype != CVRPSD_I16 && demand_dtype != CVRPSD_I32)
        return fail(ctx, CVRPSD_ERR_DTYPE, "demand_dtype %d (use CVRPSD_I16 or CVRPSD_I32)", demand_dtype);
    if (S < 0 || S > INT32_MAX) return fail(ctx, CVRPSD_ERR_ARG, "S = %lld outside 0..2^31-1", (long long)S);
    if (ld < S || ld < 1) return fail(ctx, CVRPSD_ERR_ARG, "ld = %lld must be >= max(S, 1)", (long long)ld);
    if ((unsigned long long)ld * demand_dtype > 0xFFFFFFFFull)
        return fail(ctx, CVRPSD_ERR_UNSUPPORTED, "row pitch of %lld bytes exceeds 4 GiB", (long long)ld * demand_dtype);
    if (Q < 0) return fail(ctx, CVRPSD_ERR_ARG, "Q = %d must be >= 0", Q);
    if (L < 1) return fail(ctx, CVRPSD_ERR_ARG, "L = %d must be >= 1", L);
    if (L > n) L = n;
    CK(cudaSetDevice(ctx->device), "cudaSetDevice");
    if (S > 0 && host_buffers) {
        // the kernels read the demands (and write the costs) in place, across
        // the host link: each value crosses it once
        void *dd = nullptr, *od = nullptr;
        int rc = check_host_buffer(ctx, demand, ((unsigned long long)(n - 1) * ld + S) * demand_dtype, "demand", &dd);
        if (rc) return rc;
        demand = dd;
        if (out_cost) {
            rc = check_host_buffer(ctx, out_cost, (unsigned long long)S * 4, "out_cost", &od);
            if (rc) return rc;
            out_cost = static_cast<int32_t *>(od);
        }
    } else if (S > 0) {
        int rc = check_device_buffer(ctx, demand, ((unsigned long long)(n - 1) * ld + S) * demand_dtype, "demand");
        if (rc) return rc;
        if (out_cost) {
            rc = check_device_buffer(ctx, out_cost, (unsigned long long)S * 4, "out_cost");
            if (rc) return rc;
        }
        if (pred) {
            if (ldp < S) return fail(ctx, CVRPSD_ERR_ARG, "pred pitch %lld < S", (long long)ldp);
            rc = check_device_buffer(ctx, pred, ((unsigned long long)(n - 1) * ldp + S) * 2, "pred");
            if (rc) return rc;
        }
    }
    int rc = ensure_scratch(ctx, S);
    if (rc) return rc;

    // The pinned table may still be feeding the previous call's copy.
    CK(cudaEventSynchronize(ctx->ev_tab), "cudaEventSynchronize");
    int32_t g0 = 0;
    rc = build_tour_table(ctx, tour, n, dist, Q, ctx->h_tab, &g0);
    if (rc) return rc;
    CK(cudaMemcpyAsync(ctx->d_tab, ctx->h_tab, (size_t)n * sizeof(TourStep), cudaMemcpyHostToDevice, stream),
       "upload tour table");
    CK(cudaEventRecord(ctx->ev_tab, stream), "cudaEventRecord");
    CK(cudaMemsetAsync(ctx->d_acc, 0, ACC_WORDS * sizeof(unsigned long long), stream), "clear accumulators");

    SplitParams p{};
    p.tab = ctx->d_tab;
    p.demand = demand;
    p.ld = ld;
    p.S = S;
    p.n = n;
    p.Q = Q;
    p.L = L;
    p.g0 = g0;
    p.K = key_scale(n);
    p.out_cost = out_cost;
    p.acc = ctx->d_acc;
    p.ovf_list = ctx->d_list;
    p.pred = pred;
    p.ldp = ldp;

    cvrpsd_stats st{};
    st.overflow = -1;
    st.kernel_ms = st.fallback_ms = -1.0f;
    const bool timed = ctx->profiling && (out_sum || out_infeasible || out_mean || host_buffers) && S > 0;
    bool fallback_launched = false;
    if (S > 0) {
        // Automatic choice: for a handful of scenarios on a long tour the
        // sequence-parallel kernel has the lowest latency (it parallelises
        // along the tour); otherwise scenario parallelism wins.
        int kernel = ctx->cfg.kernel;
        if (kernel == CVRPSD_KERNEL_AUTO)
            kernel = (S <= 256 && n >= 128 && !pred) ? CVRPSD_KERNEL_SEQPAR : CVRPSD_KERNEL_DEQUE;
        const int warp_grid = 2 * (ctx->sm_count > 0 ? ctx->sm_count : 152);
        if (kernel == CVRPSD_KERNEL_SEQPAR && !pred) {
            if (S > 4096) return fail(ctx, CVRPSD_ERR_UNSUPPORTED, "the sequence-parallel kernel takes S <= 4096");
            const int blocks = seqpar_blocks(n), W = seqpar_width();
            int rc2 = 0;
            auto grow = [&](int32_t **buf, long long *cap, long long need, const char *what) {
                if (rc2 || need <= *cap) return;
                if (*buf) cudaFree(*buf);
                *buf = nullptr;
                *cap = 0;
                if (dev_alloc(ctx, buf, sizeof(int32_t) * need) != cudaSuccess) {
                    cudaGetLastError();
                    rc2 = fail(ctx, CVRPSD_ERR_NOMEM, "%s", what);
                    return;
                }
                *cap = need;
            };
            grow(&ctx->seq_lo, &ctx->seq_lo_cap, S * (long long)n, "window starts");
            grow(&ctx->seq_flags, &ctx->seq_flags_cap, S, "flags");
            grow(&ctx->seq_mats, &ctx->seq_mats_cap, S * (long long)blocks * W * W, "transfer matrices");
            if (rc2) return rc2;
            SeqParParams a{};
            a.tab = ctx->d_tab;
            a.demand = demand;
            a.ld = ld;
            a.S = (int)S;
            a.n = n;
            a.Q = Q;
            a.L = L;
            a.g0 = g0;
            a.blocks = blocks;
            a.lo = ctx->seq_lo;
            a.flags = ctx->seq_flags;
            a.mats = ctx->seq_mats;
            a.out_cost = out_cost;
            a.acc = ctx->d_acc;
            a.list = ctx->d_list;
            if (timed) CK(cudaEventRecord(ctx->ev_t[0], stream), "cudaEventRecord");
            CK(launch_seqpar(a, demand_dtype, stream), "seqpar launch");
            if (timed) CK(cudaEventRecord(ctx->ev_t[1], stream), "cudaEventRecord");
            CK(launch_split_warp(p, demand_dtype, ctx->d_list, ctx->d_acc + ACC_OVERFLOW, warp_grid, ctx->max_smem,
                                 stream),
               "split_warp (set-aside scenarios) launch");
            if (timed) CK(cudaEventRecord(ctx->ev_t[2], stream), "cudaEventRecord");
            fallback_launched = true;
            st.kernel = CVRPSD_KERNEL_SEQPAR;
            st.launches = 4;
        } else if (kernel == CVRPSD_KERNEL_WARP) {
            long long need = (S + 3) / 4;
            const int grid = (int)(need < 8LL * warp_grid ? need : 8LL * warp_grid);
            if (timed) CK(cudaEventRecord(ctx->ev_t[0], stream), "cudaEventRecord");
            CK(launch_split_warp(p, demand_dtype, nullptr, nullptr, grid, ctx->max_smem, stream),
               "split_warp launch");
            if (timed) CK(cudaEventRecord(ctx->ev_t[1], stream), "cudaEventRecord");
            st.kernel = CVRPSD_KERNEL_WARP;
            st.launches = 1;
        } else {
            DequeShape shape{128, 1, 16};
            if (ctx->cfg.threads) shape = DequeShape{ctx->cfg.threads, ctx->cfg.spt, ctx->cfg.ring};
            if (shape.threads > 256) shape.threads = 256;   // 512 threads: batched path only
            // The parameter-table walk wherever it applies (one scenario per
            // thread, no predecessor output, n <= 4032, ...).
            // Host buffers keep the global-table walk: its prefetch runs twice
            // as far ahead, which the host link's latency wants.
            const bool v2_ok = deque2_supported(p, demand_dtype) && !host_buffers;
            const int variant = ctx->cfg.variant == CVRPSD_WALK_GLOBAL_TABLE || !v2_ok ? CVRPSD_WALK_GLOBAL_TABLE
                              : (ctx->cfg.variant == CVRPSD_WALK_PARAM_TABLE || !ctx->cfg.threads || shape.spt == 1)
                                  ? CVRPSD_WALK_PARAM_TABLE
                                  : CVRPSD_WALK_GLOBAL_TABLE;
            if (variant == CVRPSD_WALK_PARAM_TABLE) {
                if (timed) CK(cudaEventRecord(ctx->ev_t[0], stream), "cudaEventRecord");
                DequeShape ran{};
                const int rounds = ctx->cfg.rounds;
                // untuned default: 128 threads, rings of 16 (13 blocks fill an SM's
                // shared memory; rings of 8 need a ring-overflow test on every push
                // and set aside more scenarios, and measured 20 % slower at n = 1000)
                const DequeShape want = ctx->cfg.threads ? DequeShape{shape.threads, 1, shape.ring}
                                                         : DequeShape{128, 1, 16};
                CK(launch_split_deque2(p, ctx->h_tab, demand_dtype, want, rounds, &ran, stream),
                   "split_deque2 launch");
                if (timed) CK(cudaEventRecord(ctx->ev_t[1], stream), "cudaEventRecord");
                st.kernel = CVRPSD_KERNEL_DEQUE;
                st.threads = ran.threads;
                st.spt = 1;
                st.ring = ran.ring;
                st.variant = CVRPSD_WALK_PARAM_TABLE;
                st.rounds = rounds;
                CK(launch_split_warp(p, demand_dtype, ctx->d_list, ctx->d_acc + ACC_OVERFLOW, warp_grid,
                                     ctx->max_smem, stream),
                   "split_warp (set-aside scenarios) launch");
                st.launches = 2;
                fallback_launched = true;
                if (timed) CK(cudaEventRecord(ctx->ev_t[2], stream), "cudaEventRecord");
                goto launched;
            }
            if (host_buffers && !ctx->cfg.threads) shape = DequeShape{128, 1, 16};
            if (shape.ring == 8 && (shape.spt != 1 || shape.threads == 64 || pred))
                shape.ring = 16;   // rings of 8 exist for one scenario per thread, 128 or 256 threads
            if (pred && (shape.spt != 1 || shape.threads == 64 || shape.ring == 64))
                shape = DequeShape{128, 1, 16};      // route recovery shapes
            // Vector loads of spt demands need spt-aligned rows and base.
            while (shape.spt > 1 && (ld % shape.spt != 0 ||
                                     (uintptr_t)demand % ((uintptr_t)shape.spt * demand_dtype) != 0))
                shape.spt >>= 1;
            // Fit the block's rings in the device's shared-memory limit.
            while (split_deque_smem(p, shape) > (size_t)ctx->max_smem) {
                if (shape.spt > 1) shape.spt >>= 1;
                else if (shape.threads > 64) shape.threads >>= 1;
                else if (shape.ring > 16) shape.ring >>= 1;
                else return fail(ctx, CVRPSD_ERR_UNSUPPORTED, "no deque shape fits %d bytes of shared memory",
                                 ctx->max_smem);
            }
            if (timed) CK(cudaEventRecord(ctx->ev_t[0], stream), "cudaEventRecord");
            CK(launch_split_deque(p, demand_dtype, shape, stream), "split_deque launch");
            if (timed) CK(cudaEventRecord(ctx->ev_t[1], stream), "cudaEventRecord");
            st.kernel = CVRPSD_KERNEL_DEQUE;
            st.threads = shape.threads;
            st.spt = shape.spt;
            st.ring = shape.ring;
            st.variant = CVRPSD_WALK_GLOBAL_TABLE;
            st.launches = 1;
            // Scenarios the deque kernel set aside (ring too small, a demand above
            // Q, a negative demand) are evaluated by the warp kernel; with none
            // set aside its blocks exit at once.
            CK(launch_split_warp(p, demand_dtype, ctx->d_list, ctx->d_acc + ACC_OVERFLOW, warp_grid,
                                 ctx->max_smem, stream),
               "split_warp (set-aside scenarios) launch");
            st.launches = 2;
            fallback_launched = true;
            if (timed) CK(cudaEventRecord(ctx->ev_t[2], stream), "cudaEventRecord");
        }
    }
launched:
    ctx->stats = st;
    log_msg(ctx, CVRPSD_LOG_DEBUG, "split n=%d S=%lld: kernel %d walk %d threads %d spt %d ring %d rounds %d", n,
            (long long)S, st.kernel, st.variant, st.threads, st.spt, st.ring, st.rounds);
    if (!out_sum && !out_infeasible && !out_mean && !host_buffers) return CVRPSD_OK;

    CK(cudaMemcpyAsync(ctx->h_acc, ctx->d_acc, ACC_WORDS * sizeof(unsigned long long), cudaMemcpyDeviceToHost,
                       stream),
       "read accumulators");
    CK(cudaStreamSynchronize(stream), "cudaStreamSynchronize");
    const unsigned long long *a = ctx->h_acc;
    ctx->stats.overflow = (int64_t)a[ACC_OVERFLOW];
    if (timed) {
        float ms = 0;
        CK(cudaEventElapsedTime(&ms, ctx->ev_t[0], ctx->ev_t[1]), "cudaEventElapsedTime");
        ctx->stats.kernel_ms = ms;
        if (fallback_launched) {
            CK(cudaEventElapsedTime(&ms, ctx->ev_t[1], ctx->ev_t[2]), "cudaEventElapsedTime");
            ctx->stats.fallback_ms = ms;
        }
    }
    if (a[ACC_STATUS] & ST_INDEX)
        return fail(ctx, CVRPSD_ERR_DEVICE_STATUS, "a kernel index check failed (checked build)");
    if (a[ACC_STATUS] & ST_NEGATIVE_DEMAND)
        return fail(ctx, CVRPSD_ERR_DEVICE_STATUS, "negative demand found in the scenario matrix");
    const long long sum = (long long)a[ACC_SUM];
    const long long inf = (long long)a[ACC_INFEASIBLE];
    if (out_sum) *out_sum = sum;
    if (out_infeasible) *out_infeasible = inf;
    if (out_mean) *out_mean = (S - inf) > 0 ? (double)sum / (double)(S - inf) : NAN;
    return inf > 0 ? CVRPSD_WARN_INFEASIBLE : CVRPSD_OK;
}

}  // namespace

extern "C" {

int cvrpsd_split_eval(cvrpsd_ctx *ctx, const int32_t *tour, int32_t n, const int32_t *dist, const void *demand,
                      int32_t demand_dtype, int64_t S, int64_t ld, int32_t Q, int32_t L, int32_t *out_cost,
                      int64_t *out_sum, int64_t *out_infeasible, double *out_mean, void *stream)
{
    CVRPSD_TRACE("cvrpsd_split_eval");
    return split_eval_impl(ctx, tour, n, dist, demand, demand_dtype, S, ld, Q, L, out_cost, out_sum, out_infeasible,
                           out_mean, stream, nullptr, 0);
}

int cvrpsd_split_eval_host(cvrpsd_ctx *ctx, const int32_t *tour, int32_t n, const int32_t *dist,
                           const void *demand, int32_t demand_dtype, int64_t S, int64_t ld, int32_t Q, int32_t L,
                           int32_t *out_cost, int64_t *out_sum, int64_t *out_infeasible, double *out_mean,
                           void *stream)
{
    CVRPSD_TRACE("cvrpsd_split_eval_host");
    if (!ctx) return CVRPSD_ERR_ARG;
    return split_eval_impl(ctx, tour, n, dist, demand, demand_dtype, S, ld, Q, L, out_cost, out_sum, out_infeasible,
                           out_mean, stream, nullptr, 0, true);
}

int cvrpsd_split_routes(cvrpsd_ctx *ctx, const int32_t *tour, int32_t n, const int32_t *dist, const void *demand,
                        int32_t demand_dtype, int64_t S, int64_t ld, int32_t Q, int32_t L, int32_t *out_cost,
                        int16_t *pred, int64_t ldp, int64_t *out_sum, int64_t *out_infeasible, double *out_mean,
                        void *stream)
{
    CVRPSD_TRACE("cvrpsd_split_routes");
    if (!ctx) return CVRPSD_ERR_ARG;
    if (!pred) return fail(ctx, CVRPSD_ERR_ARG, "pred is required");
    return split_eval_impl(ctx, tour, n, dist, demand, demand_dtype, S, ld, Q, L, out_cost, out_sum, out_infeasible,
                           out_mean, stream, pred, ldp);
}

}  // extern "C"

namespace {

// One split with the given shape; the main-kernel + set-aside device time.
int timed_split(cvrpsd_ctx *ctx, const cvrpsd_config &cfg, const int32_t *tour, int32_t n, const int32_t *dist,
                const void *demand, int32_t dtype, int64_t S, int64_t ld, int32_t Q, int32_t L, void *stream,
                long long *sum, long long *inf, float *ms)
{
    ctx->cfg = cfg;
    int64_t s64 = 0, i64 = 0;
    double mean = 0;
    const int rc = cvrpsd_split_eval(ctx, tour, n, dist, demand, dtype, S, ld, Q, L, nullptr, &s64, &i64, &mean,
                                     stream);
    if (rc < 0) return rc;
    *sum = s64;
    *inf = i64;
    *ms = ctx->stats.kernel_ms + (ctx->stats.fallback_ms > 0 ? ctx->stats.fallback_ms : 0.0f);
    return CVRPSD_OK;
}

std::string tune_key(cvrpsd_ctx *ctx, int n, long long S, int dtype, bool lcap)
{
    cudaDeviceProp prop;
    std::string name = cudaGetDeviceProperties(&prop, ctx->device) == cudaSuccess ? prop.name : "unknown";
    for (char &c : name)
        if (c == ' ' || c == '"') c = '_';
    long long nb = 1, sb = 1;
    while (nb < n) nb <<= 1;
    while (sb * 2 <= S) sb <<= 1;
    char buf[256];
    snprintf(buf, sizeof(buf), "%s/n%lld/S%lld/%s/%s", name.c_str(), nb, sb, dtype == CVRPSD_I16 ? "i16" : "i32",
             lcap ? "cap" : "nocap");
    return buf;
}

bool tune_cache_lookup(const char *path, const std::string &key, cvrpsd_tune_result *r)
{
    FILE *f = fopen(path, "r");
    if (!f) return false;
    char line[512], k[256];
    bool found = false;
    while (fgets(line, sizeof(line), f)) {
        cvrpsd_tune_result t{};
        if (sscanf(line, "{\"key\": \"%255[^\"]\", \"threads\": %d, \"spt\": %d, \"ring\": %d, \"variant\": %d, "
                         "\"rounds\": %d, \"ms\": %f, \"dtype\": %d}",
                   k, &t.best.threads, &t.best.spt, &t.best.ring, &t.best.variant, &t.best.rounds, &t.best_ms,
                   &t.best_dtype) == 8 &&
            key == k && valid_shape(t.best.threads, t.best.spt, t.best.ring)) {
            t.best.kernel = CVRPSD_KERNEL_DEQUE;
            *r = t;
            found = true;   // the last entry for a key wins
        }
    }
    fclose(f);
    return found;
}

}  // namespace

extern "C" int cvrpsd_autotune(cvrpsd_ctx *ctx, const int32_t *tour, int32_t n, const int32_t *dist,
                               const void *demand, int32_t demand_dtype, int64_t S, int64_t ld, int32_t Q, int32_t L,
                               const char *cache_path, cvrpsd_tune_result *result, void *stream_ptr)
{
    CVRPSD_TRACE("cvrpsd_autotune");
    if (!ctx || !result) return CVRPSD_ERR_ARG;
    if (S < 1) return fail(ctx, CVRPSD_ERR_ARG, "autotune needs S >= 1");
    const cvrpsd_config saved = ctx->cfg;
    const int saved_prof = ctx->profiling;
    int rc = cvrpsd_set_profiling(ctx, 1);
    if (rc) return rc;
    const bool lcap = L < n;
    const std::string key = tune_key(ctx, n, S, demand_dtype, lcap);
    cvrpsd_tune_result best{};
    long long ref_sum = 0, ref_inf = 0, s_ = 0, i_ = 0;
    float ms = 0;
    // reference: the global-table walk in its default shape (also validates
    // every argument); every candidate must reproduce its sums
    rc = timed_split(ctx, cvrpsd_config{CVRPSD_KERNEL_DEQUE, 128, 1, 16, CVRPSD_WALK_GLOBAL_TABLE, 0}, tour, n, dist,
                     demand, demand_dtype, S, ld,
                     Q, L, stream_ptr, &ref_sum, &ref_inf, &ms);
    if (rc < 0) {
        ctx->cfg = saved;
        ctx->profiling = saved_prof;
        return rc;
    }
    if (cache_path && tune_cache_lookup(cache_path, key, &best)) {
        best.shapes_timed = 0;
        ctx->cfg = best.best;
        ctx->profiling = saved_prof;
        *result = best;
        return CVRPSD_OK;
    }
    best.best_ms = 1e30f;
    int timed = 0;
    // Candidates: the parameter-table walk (where it applies) over threads x
    // ring, one scenario per thread (grids of several rounds per block
    // measured slower on GB300 and are not swept), then the global-table walk
    // over threads x spt x ring.
    std::vector<cvrpsd_config> cands;
    SplitParams probe{};
    probe.n = n;
    probe.ld = ld;
    probe.S = S;
    probe.Q = Q;
    probe.L = L < n ? L : n;
    probe.K = key_scale(n);
    if (deque2_supported(probe, demand_dtype)) {
        for (int threads : {64, 128, 256})
            for (int ring : {8, 16})
                cands.push_back(cvrpsd_config{CVRPSD_KERNEL_DEQUE, threads, 1, ring, CVRPSD_WALK_PARAM_TABLE, 0});
    }
    for (int threads : {64, 128, 256})
        for (int spt : {1, 2})
            for (int ring : {16, 32, 64})
                cands.push_back(cvrpsd_config{CVRPSD_KERNEL_DEQUE, threads, spt, ring, CVRPSD_WALK_GLOBAL_TABLE, 0});
    for (const cvrpsd_config &cfg : cands) {
        const int threads = cfg.threads, spt = cfg.spt, ring = cfg.ring;
        float t_best = 1e30f;
        for (int rep = 0; rep < 4; ++rep) {
            rc = timed_split(ctx, cfg, tour, n, dist, demand, demand_dtype, S, ld, Q, L, stream_ptr, &s_,
                             &i_, &ms);
            if (rc < 0) break;
            if (s_ != ref_sum || i_ != ref_inf) {
                ctx->cfg = saved;
                ctx->profiling = saved_prof;
                return fail(ctx, CVRPSD_ERR_DEVICE_STATUS,
                            "shape %d/%d/%d walk %d rounds %d gives sum %lld, default %lld", threads, spt,
                            ring, cfg.variant, cfg.rounds, s_, ref_sum);
            }
            if (rep > 0 && ms < t_best) t_best = ms;   // first run warms up
        }
        if (rc < 0) continue;                            // shape not launchable here
        ++timed;
        // the shape the library actually ran (it may shrink spt / threads to fit)
        const cvrpsd_config ran{CVRPSD_KERNEL_DEQUE, ctx->stats.threads, ctx->stats.spt, ctx->stats.ring,
                                ctx->stats.variant, ctx->stats.rounds};
        if (t_best < best.best_ms) {
            best.best_ms = t_best;
            best.best = ran;
        }
    }
    if (!timed) {
        ctx->cfg = saved;
        ctx->profiling = saved_prof;
        return fail(ctx, CVRPSD_ERR_UNSUPPORTED, "no launch shape could run this workload");
    }
    best.shapes_timed = timed;
    best.best_dtype = demand_dtype;

    // Demand storage: time the best shape on int16 and int32 copies of a sample.
    const long long Ss = S < 65536 ? S : 65536;
    void *tmp[2] = {nullptr, nullptr};
    unsigned int *sat = nullptr;
    cudaStream_t stream = reinterpret_cast<cudaStream_t>(stream_ptr);
    if (dev_alloc(ctx, &tmp[0], (size_t)n * Ss * 2) == cudaSuccess &&
        dev_alloc(ctx, &tmp[1], (size_t)n * Ss * 4) == cudaSuccess &&
        dev_alloc(ctx, &sat, sizeof(unsigned int)) == cudaSuccess && cudaMemsetAsync(sat, 0, 4, stream) == cudaSuccess &&
        launch_convert_demand(demand, demand_dtype, ld, tmp[0], 2, Ss, n, Ss, sat, stream) == cudaSuccess &&
        launch_convert_demand(demand, demand_dtype, ld, tmp[1], 4, Ss, n, Ss, sat, stream) == cudaSuccess) {
        unsigned int h_sat = 1;
        cudaMemcpyAsync(&h_sat, sat, 4, cudaMemcpyDeviceToHost, stream);
        cudaStreamSynchronize(stream);
        float t16 = 1e30f, t32 = 1e30f;
        for (int rep = 0; rep < 4; ++rep) {
            if (!h_sat && timed_split(ctx, best.best, tour, n, dist, tmp[0], CVRPSD_I16, Ss, Ss, Q, L, stream_ptr,
                                      &s_, &i_, &ms) == CVRPSD_OK && rep > 0)
                t16 = std::min(t16, ms);
            if (timed_split(ctx, best.best, tour, n, dist, tmp[1], CVRPSD_I32, Ss, Ss, Q, L, stream_ptr, &s_, &i_,
                            &ms) == CVRPSD_OK && rep > 0)
                t32 = std::min(t32, ms);
        }
        best.best_dtype = (!h_sat && t16 <= t32) ? CVRPSD_I16 : CVRPSD_I32;
    } else {
        cudaGetLastError();
    }
    for (void *p : tmp)
        if (p) cudaFree(p);
    if (sat) cudaFree(sat);

    ctx->cfg = best.best;
    ctx->profiling = saved_prof;
    log_msg(ctx, CVRPSD_LOG_INFO, "autotune n=%d S=%lld: %d shapes, best walk %d threads %d spt %d ring %d "
            "(%.4f ms), demand type %s", n, (long long)S, best.shapes_timed, best.best.variant, best.best.threads,
            best.best.spt, best.best.ring, best.best_ms, best.best_dtype == CVRPSD_I16 ? "int16" : "int32");
    if (cache_path) {
        if (FILE *f = fopen(cache_path, "a")) {
            fprintf(f, "{\"key\": \"%s\", \"threads\": %d, \"spt\": %d, \"ring\": %d, \"variant\": %d, "
                       "\"rounds\": %d, \"ms\": %.6f, \"dtype\": %d}\n",
                    key.c_str(), best.best.threads, best.best.spt, best.best.ring, best.best.variant,
                    best.best.rounds, best.best_ms, best.best_dtype);
            fclose(f);
        }
    }
    *result = best;
    return CVRPSD_OK;
}

struct cvrpsd_batch {
    cvrpsd_ctx *ctx = nullptr;
    int T = 0;
    long long S = 0;
    BatchParams bp{};
    TourDev *d_tours = nullptr;
    TourStep *d_tabs = nullptr;
    int2 *d_items = nullptr;
    unsigned long long *d_acc = nullptr;
    int2 *d_list = nullptr;
    unsigned long long *h_acc = nullptr;   // pinned: header + 3 words per tour
    size_t acc_words = 0;
    cudaStream_t cap_stream = nullptr;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    cudaEvent_t done = nullptr;
    bool ran = false;
};

namespace {

void batch_free(cvrpsd_batch *b)
{
    if (!b) return;
    if (b->exec) cudaGraphExecDestroy(b->exec);
    if (b->graph) cudaGraphDestroy(b->graph);
    if (b->cap_stream) cudaStreamDestroy(b->cap_stream);
    if (b->done) cudaEventDestroy(b->done);
    if (b->d_tours) cudaFree(b->d_tours);
    if (b->d_tabs) cudaFree(b->d_tabs);
    if (b->d_items) cudaFree(b->d_items);
    if (b->d_acc) cudaFree(b->d_acc);
    if (b->d_list) cudaFree(b->d_list);
    if (b->h_acc) cudaFreeHost(b->h_acc);
    delete b;
}

bool valid_batch_shape(const DequeShape &s) { return batch_shape_compiled(s); }

}  // namespace

extern "C" {

int cvrpsd_batch_create(cvrpsd_ctx *ctx, int32_t T, const cvrpsd_tour_desc *tours, int64_t S, int32_t demand_dtype,
                        cvrpsd_batch **out)
{
    CVRPSD_TRACE("cvrpsd_batch_create");
    if (!ctx || !out) return CVRPSD_ERR_ARG;
    *out = nullptr;
    ctx->err[0] = 0;
    if (T < 1 || !tours) return fail(ctx, CVRPSD_ERR_ARG, "T = %d tours (need >= 1)", T);
    if (demand_dtype != CVRPSD_I16 && demand_dtype != CVRPSD_I32)
        return fail(ctx, CVRPSD_ERR_DTYPE, "demand_dtype %d", demand_dtype);
    if (S < 1 || S > INT32_MAX) return fail(ctx, CVRPSD_ERR_ARG, "S = %lld outside 1..2^31-1", (long long)S);
    CK(cudaSetDevice(ctx->device), "cudaSetDevice");

    std::vector<TourDev> hd((size_t)T);
    std::vector<long long> tab_off((size_t)T);
    long long total_n = 0;
    int max_n = 0;
    bool lcap = false;
    for (int t = 0; t < T; ++t) {
        const cvrpsd_tour_desc &d = tours[t];
        if (d.n < 1 || d.n > CVRPSD_MAX_N) return fail(ctx, CVRPSD_ERR_ARG, "tour %d: n = %d", t, d.n);
        if (d.Q < 0 || d.L < 1) return fail(ctx, CVRPSD_ERR_ARG, "tour %d: Q = %d, L = %d", t, d.Q, d.L);
        if (d.ld < S) return fail(ctx, CVRPSD_ERR_ARG, "tour %d: ld = %lld < S", t, (long long)d.ld);
        if ((unsigned long long)d.ld * demand_dtype > 0xFFFFFFFFull)
            return fail(ctx, CVRPSD_ERR_UNSUPPORTED, "tour %d: row pitch exceeds 4 GiB", t);
        int rc = check_device_buffer(ctx, d.demand, ((unsigned long long)(d.n - 1) * d.ld + S) * demand_dtype,
                                     "demand");
        if (rc) return fail(ctx, rc, "tour %d: %s", t, std::string(ctx->err).c_str());
        if (d.out_cost) {
            rc = check_device_buffer(ctx, d.out_cost, (unsigned long long)S * 4, "out_cost");
            if (rc) return fail(ctx, rc, "tour %d: %s", t, std::string(ctx->err).c_str());
        }
        tab_off[t] = total_n;
        total_n += d.n;
        if (d.n > max_n) max_n = d.n;
        const int L = d.L > d.n ? d.n : d.L;
        if (L < d.n) lcap = true;
    }
    std::vector<TourStep> htab((size_t)total_n);
    for (int t = 0; t < T; ++t) {
        const cvrpsd_tour_desc &d = tours[t];
        int32_t g0 = 0;
        int rc = build_tour_table(ctx, d.tour, d.n, d.dist, d.Q, htab.data() + tab_off[t], &g0);
        if (rc) return fail(ctx, rc, "tour %d: %s", t, std::string(ctx->err).c_str());
        TourDev &td = hd[t];
        td.tab = nullptr;   // set after upload
        td.demand = d.demand;
        td.ld = d.ld;
        td.out_cost = d.out_cost;
        td.n = d.n;
        td.Q = d.Q;
        td.L = d.L > d.n ? d.n : d.L;
        if (!lcap) td.L = d.n + 1;
        td.g0 = g0;
        td.K = key_scale(d.n);
        td.pad = 0;
    }

    DequeShape shape{256, 1, 16};
    if (ctx->cfg.threads) {
        DequeShape want{ctx->cfg.threads, ctx->cfg.spt, ctx->cfg.ring};
        if (valid_batch_shape(want)) shape = want;
    }
    while (split_batch_smem(max_n, shape) > (size_t)ctx->max_smem) {
        if (shape.spt > 1) shape.spt = 1;
        else if (shape.ring > 16) shape.ring = 16;
        else if (shape.threads > 128) shape.threads = 128;
        else return fail(ctx, CVRPSD_ERR_UNSUPPORTED, "no batch shape fits %d bytes of shared memory", ctx->max_smem);
    }
    const long long per_tile = (long long)shape.threads * shape.spt;
    const long long tiles = (S + per_tile - 1) / per_tile;
    if (tiles * T > INT32_MAX) return fail(ctx, CVRPSD_ERR_UNSUPPORTED, "too many work items");
    // Work items: tours by decreasing n (longest first), all tiles of a tour together.
    std::vector<int> order((size_t)T);
    for (int t = 0; t < T; ++t) order[t] = t;
    std::stable_sort(order.begin(), order.end(), [&](int a, int b) { return tours[a].n > tours[b].n; });
    std::vector<int2> items((size_t)(tiles * T));
    size_t k = 0;
    for (int t : order)
        for (long long j = 0; j < tiles; ++j) items[k++] = make_int2(t, (int)j);

    cvrpsd_batch *b = new (std::nothrow) cvrpsd_batch();
    if (!b) return CVRPSD_ERR_NOMEM;
    b->ctx = ctx;
    b->T = T;
    b->S = S;
    b->acc_words = BACC_WORDS + 3 * (size_t)T;
    const long long list_cap = std::min<long long>((long long)T * S, 1LL << 24);
#define BK(call, what)                              do {                                                cudaError_t e_ = (call);                        if (e_ != cudaSuccess) {                            int rc_ = cuda_fail(ctx, e_, what);             cudaGetLastError();                             batch_free(b);                                  return rc_;                                 }                                           } while (0)
    BK(dev_alloc(ctx, &b->d_tours, sizeof(TourDev) * T), "cudaMalloc(tours)");
    BK(dev_alloc(ctx, &b->d_tabs, sizeof(TourStep) * total_n), "cudaMalloc(tables)");
    BK(dev_alloc(ctx, &b->d_items, sizeof(int2) * items.size()), "cudaMalloc(items)");
    BK(dev_alloc(ctx, &b->d_acc, sizeof(unsigned long long) * b->acc_words), "cudaMalloc(acc)");
    BK(dev_alloc(ctx, &b->d_list, sizeof(int2) * list_cap), "cudaMalloc(list)");
    BK(host_alloc(ctx, &b->h_acc, sizeof(unsigned long long) * b->acc_words), "cudaMallocHost(acc)");
    for (int t = 0; t < T; ++t) hd[t].tab = b->d_tabs + tab_off[t];
    BK(cudaMemcpy(b->d_tours, hd.data(), sizeof(TourDev) * T, cudaMemcpyHostToDevice), "upload tours");
    BK(cudaMemcpy(b->d_tabs, htab.data(), sizeof(TourStep) * total_n, cudaMemcpyHostToDevice), "upload tables");
    BK(cudaMemcpy(b->d_items, items.data(), sizeof(int2) * items.size(), cudaMemcpyHostToDevice), "upload items");

    BatchParams &bp = b->bp;
    bp.tours = b->d_tours;
    bp.items = b->d_items;
    bp.tiles = (int)tiles;
    bp.n_items = (int)items.size();
    bp.S = S;
    bp.acc = b->d_acc;
    bp.list = b->d_list;
    bp.list_cap = list_cap;
    bp.max_n = max_n;
    bp.walk2 = demand_dtype == CVRPSD_I16;
    for (int t = 0; t < T; ++t) bp.walk2 &= batch2_keys_fit(hd[t].n, hd[t].Q, hd[t].K);
    int per_sm = 0;
    BK(launch_split_batch(bp, demand_dtype, lcap, shape, 0, true, &per_sm, nullptr), "configure batch kernel");
    if (per_sm < 1) per_sm = 1;
    const int grid = ctx->sm_count * per_sm;
    const int warp_grid = 2 * ctx->sm_count;
    BK(launch_split_warp_batch(bp, demand_dtype, warp_grid, ctx->max_smem, true, nullptr), "configure warp kernel");

    BK(cudaStreamCreateWithFlags(&b->cap_stream, cudaStreamNonBlocking), "cudaStreamCreate");
    BK(cudaEventCreateWithFlags(&b->done, cudaEventDisableTiming), "cudaEventCreate");
    BK(cudaStreamBeginCapture(b->cap_stream, cudaStreamCaptureModeThreadLocal), "begin capture");
    cudaError_t e1 = cudaMemsetAsync(b->d_acc, 0, sizeof(unsigned long long) * b->acc_words, b->cap_stream);
    cudaError_t e2 = launch_split_batch(bp, demand_dtype, lcap, shape, grid, false, nullptr, b->cap_stream);
    cudaError_t e3 = launch_split_warp_batch(bp, demand_dtype, warp_grid, ctx->max_smem, false, b->cap_stream);
    cudaError_t e4 = cudaMemcpyAsync(b->h_acc, b->d_acc, sizeof(unsigned long long) * b->acc_words,
                                     cudaMemcpyDeviceToHost, b->cap_stream);
    cudaError_t e5 = cudaStreamEndCapture(b->cap_stream, &b->graph);
    BK(e1 != cudaSuccess ? e1 : e2 != cudaSuccess ? e2 : e3 != cudaSuccess ? e3 : e4 != cudaSuccess ? e4 : e5,
       "capture batch graph");
    BK(cudaGraphInstantiate(&b->exec, b->graph, 0), "instantiate batch graph");
#undef BK
    ctx->stats = cvrpsd_stats{};
    ctx->stats.kernel = CVRPSD_KERNEL_DEQUE;
    ctx->stats.threads = shape.threads;
    ctx->stats.spt = shape.spt;
    ctx->stats.ring = shape.ring;
    ctx->stats.overflow = -1;
    ctx->stats.launches = 2;
    ctx->stats.kernel_ms = ctx->stats.fallback_ms = -1.0f;
    *out = b;
    return CVRPSD_OK;
}

int cvrpsd_batch_run(cvrpsd_batch *b, void *stream_ptr)
{
    CVRPSD_TRACE("cvrpsd_batch_run");
    if (!b) return CVRPSD_ERR_ARG;
    cvrpsd_ctx *ctx = b->ctx;
    cudaStream_t stream = reinterpret_cast<cudaStream_t>(stream_ptr);
    CK(cudaSetDevice(ctx->device), "cudaSetDevice");
    CK(cudaGraphLaunch(b->exec, stream), "cudaGraphLaunch");
    CK(cudaEventRecord(b->done, stream), "cudaEventRecord");
    b->ran = true;
    return CVRPSD_OK;
}

int cvrpsd_batch_results(cvrpsd_batch *b, int64_t *out_sum, int64_t *out_infeasible, double *out_mean,
                         int32_t *out_status)
{
    CVRPSD_TRACE("cvrpsd_batch_results");
    if (!b) return CVRPSD_ERR_ARG;
    cvrpsd_ctx *ctx = b->ctx;
    if (!b->ran) return fail(ctx, CVRPSD_ERR_ARG, "batch has not been run");
    CK(cudaEventSynchronize(b->done), "cudaEventSynchronize");
    const unsigned long long *h = b->h_acc;
    if (h[BACC_STATUS] & ST_INDEX)
        return fail(ctx, CVRPSD_ERR_DEVICE_STATUS, "a kernel index check failed (checked build)");
    if (h[BACC_STATUS] & BST_LIST_FULL)
        return fail(ctx, CVRPSD_ERR_UNSUPPORTED, "more than %lld set-aside scenarios", (long long)b->bp.list_cap);
    ctx->stats.overflow = (int64_t)h[BACC_LIST];
    int worst = CVRPSD_OK;
    for (int t = 0; t < b->T; ++t) {
        const unsigned long long *w = h + BACC_WORDS + 3 * t;
        const long long sum = (long long)w[0], inf = (long long)w[1];
        int st = CVRPSD_OK;
        if (w[2] & ST_NEGATIVE_DEMAND) st = CVRPSD_ERR_DEVICE_STATUS;
        else if (inf > 0) st = CVRPSD_WARN_INFEASIBLE;
        if (out_sum) out_sum[t] = sum;
        if (out_infeasible) out_infeasible[t] = inf;
        if (out_mean) out_mean[t] = (b->S - inf) > 0 ? (double)sum / (double)(b->S - inf) : NAN;
        if (out_status) out_status[t] = st;
        if (st < 0) worst = st;
        else if (worst >= 0 && st > worst) worst = st;
    }
    if (worst == CVRPSD_ERR_DEVICE_STATUS) fail(ctx, worst, "negative demand in at least one tour's matrix");
    return worst;
}

int cvrpsd_batch_destroy(cvrpsd_batch *b)
{
    if (!b) return CVRPSD_ERR_ARG;
    cudaSetDevice(b->ctx->device);
    batch_free(b);
    return CVRPSD_OK;
}

}  // extern "C"

namespace {

// Device time of one graph run of a batch in shape `cfg` (best of three after
// a warm-up), with the per-tour sums and infeasible counts of the last run.
int time_batch(cvrpsd_ctx *ctx, const cvrpsd_config &cfg, int32_t T, const cvrpsd_tour_desc *tours, int64_t S,
               int32_t dtype, cudaEvent_t ev0, cudaEvent_t ev1, cudaStream_t stream, float *ms_out,
               std::vector<int64_t> &sum, std::vector<int64_t> &inf, cvrpsd_config *ran)
{
    ctx->cfg = cfg;
    cvrpsd_batch *b = nullptr;
    int rc = cvrpsd_batch_create(ctx, T, tours, S, dtype, &b);
    if (rc) return rc;
    // the shape the batch actually runs (it may shrink to fit)
    *ran = cvrpsd_config{CVRPSD_KERNEL_DEQUE, ctx->stats.threads, ctx->stats.spt, ctx->stats.ring, 0, 0};
    float t_best = 1e30f;
    for (int rep = 0; rep < 4 && rc >= 0; ++rep) {
        cudaEventRecord(ev0, stream);
        rc = cvrpsd_batch_run(b, stream);
        cudaEventRecord(ev1, stream);
        if (rc >= 0) rc = cvrpsd_batch_results(b, sum.data(), inf.data(), nullptr, nullptr);
        float ms = 0;
        if (rc >= 0 && cudaEventElapsedTime(&ms, ev0, ev1) == cudaSuccess && rep > 0 && ms < t_best)
            t_best = ms;   // the first run warms up
    }
    cvrpsd_batch_destroy(b);
    *ms_out = t_best;
    return rc;
}

}  // namespace

extern "C" {

int cvrpsd_batch_autotune(cvrpsd_ctx *ctx, int32_t T, const cvrpsd_tour_desc *tours, int64_t S,
                          int32_t demand_dtype, cvrpsd_tune_result *result, void *stream_ptr)
{
    CVRPSD_TRACE("cvrpsd_batch_autotune");
    if (!ctx || !result) return CVRPSD_ERR_ARG;
    ctx->err[0] = 0;
    if (T < 1 || !tours) return fail(ctx, CVRPSD_ERR_ARG, "T = %d", T);
    cudaStream_t stream = reinterpret_cast<cudaStream_t>(stream_ptr);
    const cvrpsd_config saved = ctx->cfg;
    std::vector<int64_t> ref_sum((size_t)T), ref_inf((size_t)T), sum((size_t)T), inf((size_t)T);
    cudaEvent_t ev[2] = {nullptr, nullptr};
    CK(cudaSetDevice(ctx->device), "cudaSetDevice");
    CK(cudaEventCreate(&ev[0]), "cudaEventCreate");
    if (cudaEventCreate(&ev[1]) != cudaSuccess) {
        cudaEventDestroy(ev[0]);
        return fail(ctx, CVRPSD_ERR_CUDA, "cudaEventCreate");
    }
    cvrpsd_tune_result best{};
    best.best_ms = 1e30f;
    best.best_dtype = demand_dtype;
    int rc = CVRPSD_OK;
    bool have_ref = false;
    // Scenarios per block 32..512 (threads x scenarios per thread) x deque
    // ring 16 / 32 / 64 (the window tile), every shape the kernel is compiled for.
    for (int threads : {32, 64, 128, 256, 512})
        for (int spt : {1, 2})
            for (int ring : {16, 32, 64}) {
                if (rc < 0 || !batch_shape_compiled(DequeShape{threads, spt, ring})) continue;
                const cvrpsd_config cfg{CVRPSD_KERNEL_DEQUE, threads, spt, ring, 0, 0};
                cvrpsd_config ran{};
                float t = 0;
                rc = time_batch(ctx, cfg, T, tours, S, demand_dtype, ev[0], ev[1], stream, &t, sum, inf, &ran);
                if (rc < 0) break;
                if (!have_ref) {
                    ref_sum = sum;
                    ref_inf = inf;
                    have_ref = true;
                } else if (sum != ref_sum || inf != ref_inf) {
                    rc = fail(ctx, CVRPSD_ERR_DEVICE_STATUS, "batch shape %d/%d/%d changes a tour's result", threads,
                              spt, ring);
                    break;
                }
                ++best.shapes_timed;
                if (t < best.best_ms) {
                    best.best_ms = t;
                    best.best = ran;
                }
            }
    // Demand storage: the best shape on int16 and int32 copies of a sample of
    // every tour's scenarios (at most 2 GB of copies), bit-checked against
    // each other; int16 only if every demand fits.
    const long long total_n = [&] {
        long long t = 0;
        for (int k = 0; k < T; ++k) t += tours[k].n;
        return t;
    }();
    long long Ss = std::min<long long>(S, 8192);
    Ss = std::min<long long>(Ss, std::max<long long>(32, (2000000000LL / (6 * std::max<long long>(total_n, 1))) / 32 * 32));
    void *tmp16 = nullptr, *tmp32 = nullptr;
    unsigned int *sat = nullptr;
    if (rc >= 0 && Ss >= 1 && dev_alloc(ctx, &tmp16, (size_t)total_n * Ss * 2) == cudaSuccess &&
        dev_alloc(ctx, &tmp32, (size_t)total_n * Ss * 4) == cudaSuccess &&
        dev_alloc(ctx, &sat, sizeof(unsigned int)) == cudaSuccess && cudaMemsetAsync(sat, 0, 4, stream) == cudaSuccess) {
        std::vector<cvrpsd_tour_desc> d16(tours, tours + T), d32(tours, tours + T);
        long long row = 0;
        bool ok = true;
        for (int k = 0; k < T && ok; ++k) {
            char *p16 = static_cast<char *>(tmp16) + row * Ss * 2, *p32 = static_cast<char *>(tmp32) + row * Ss * 4;
            ok = launch_convert_demand(tours[k].demand, demand_dtype, tours[k].ld, p16, 2, Ss, tours[k].n, Ss, sat,
                                       stream) == cudaSuccess &&
                 launch_convert_demand(tours[k].demand, demand_dtype, tours[k].ld, p32, 4, Ss, tours[k].n, Ss, sat,
                                       stream) == cudaSuccess;
            d16[k].demand = p16;
            d32[k].demand = p32;
            d16[k].ld = d32[k].ld = Ss;
            d16[k].out_cost = d32[k].out_cost = nullptr;
            row += tours[k].n;
        }
        unsigned int h_sat = 1;
        if (ok && cudaMemcpyAsync(&h_sat, sat, 4, cudaMemcpyDeviceToHost, stream) == cudaSuccess &&
            cudaStreamSynchronize(stream) == cudaSuccess) {
            std::vector<int64_t> s16((size_t)T), i16((size_t)T);
            cvrpsd_config ran{};
            float t16 = 1e30f, t32 = 1e30f;
            const bool r32 = time_batch(ctx, best.best, T, d32.data(), Ss, CVRPSD_I32, ev[0], ev[1], stream, &t32,
                                        sum, inf, &ran) >= 0;
            const bool r16 = !h_sat && time_batch(ctx, best.best, T, d16.data(), Ss, CVRPSD_I16, ev[0], ev[1], stream,
                                                  &t16, s16, i16, &ran) >= 0;
            if (r16 && r32 && (s16 != sum || i16 != inf))
                rc = fail(ctx, CVRPSD_ERR_DEVICE_STATUS, "int16 and int32 copies of the demands disagree");
            else if (r32 || r16)
                best.best_dtype = (r16 && t16 <= t32) ? CVRPSD_I16 : CVRPSD_I32;
        }
    }
    cudaGetLastError();
    if (tmp16) cudaFree(tmp16);
    if (tmp32) cudaFree(tmp32);
    if (sat) cudaFree(sat);
    cudaEventDestroy(ev[0]);
    cudaEventDestroy(ev[1]);
    if (rc < 0) {
        ctx->cfg = saved;
        return rc;
    }
    ctx->cfg = best.best;
    *result = best;
    log_msg(ctx, CVRPSD_LOG_INFO, "batch autotune T=%d S=%lld: %d shapes, best threads %d spt %d ring %d "
            "(%.4f ms), demand type %s", T, (long long)S, best.shapes_timed, best.best.threads, best.best.spt,
            best.best.ring, best.best_ms, best.best_dtype == CVRPSD_I16 ? "int16" : "int32");
    return CVRPSD_OK;
}

int cvrpsd_split_eval_batch(cvrpsd_ctx *ctx, int32_t T, const cvrpsd_tour_desc *tours, int64_t S,
                            int32_t demand_dtype, int64_t *out_sum, int64_t *out_infeasible, double *out_mean,
                            int32_t *out_status, void *stream)
{
    CVRPSD_TRACE("cvrpsd_split_eval_batch");
    cvrpsd_batch *b = nullptr;
    int rc = cvrpsd_batch_create(ctx, T, tours, S, demand_dtype, &b);
    if (rc) return rc;
    rc = cvrpsd_batch_run(b, stream);
    if (rc == CVRPSD_OK) rc = cvrpsd_batch_results(b, out_sum, out_infeasible, out_mean, out_status);
    cvrpsd_batch_destroy(b);
    return rc;
}

int cvrpsd_gen_demand(cvrpsd_ctx *ctx, uint64_t seed, int32_t kind, const int32_t *mu, const int32_t *region,
                      int32_t n, int64_t S, int64_t ld, int32_t dtype, void *out, void *stream_ptr)
{
    CVRPSD_TRACE("cvrpsd_gen_demand");
    if (!ctx) return CVRPSD_ERR_ARG;
    ctx->err[0] = 0;
    cudaStream_t stream = reinterpret_cast<cudaStream_t>(stream_ptr);
    if (kind != CVRPSD_GEN_NORMAL && kind != CVRPSD_GEN_CORRELATED)
        return fail(ctx, CVRPSD_ERR_ARG, "generator kind %d unknown", kind);
    if (dtype != CVRPSD_I16 && dtype != CVRPSD_I32) return fail(ctx, CVRPSD_ERR_DTYPE, "dtype %d", dtype);
    if (n < 1 || n > CVRPSD_MAX_N) return fail(ctx, CVRPSD_ERR_ARG, "n = %d outside 1..%d", n, CVRPSD_MAX_N);
    if (S < 0 || S > 0xFFFFFFFFLL) return fail(ctx, CVRPSD_ERR_ARG, "S = %lld outside 0..2^32-1", (long long)S);
    if (ld < S || ld < 1) return fail(ctx, CVRPSD_ERR_ARG, "ld must be >= max(S, 1)");
    if (!mu || (kind == CVRPSD_GEN_CORRELATED && !region))
        return fail(ctx, CVRPSD_ERR_ARG, "mu (and region for correlated demands) are required");
    for (int k = 0; k < n; ++k) {
        if (mu[k] < 0) return fail(ctx, CVRPSD_ERR_ARG, "mu[%d] < 0", k);
        if (region && (region[k] < 0 || region[k] > 3)) return fail(ctx, CVRPSD_ERR_ARG, "region[%d] not in 0..3", k);
    }
    CK(cudaSetDevice(ctx->device), "cudaSetDevice");
    if (S == 0) return CVRPSD_OK;
    int rc = check_device_buffer(ctx, out, ((unsigned long long)(n - 1) * ld + S) * dtype, "out");
    if (rc) return rc;
    if (!ctx->d_gen) CK(dev_alloc(ctx, &ctx->d_gen, 2 * (CVRPSD_MAX_N + 1) * sizeof(int32_t)), "cudaMalloc(gen)");
    if (!ctx->h_gen) CK(host_alloc(ctx, &ctx->h_gen, 2 * (CVRPSD_MAX_N + 1) * sizeof(int32_t)), "cudaMallocHost(gen)");
    if (!ctx->ev_gen) CK(cudaEventCreateWithFlags(&ctx->ev_gen, cudaEventDisableTiming), "cudaEventCreate");
    CK(cudaEventSynchronize(ctx->ev_gen), "cudaEventSynchronize");
    for (int k = 0; k < n; ++k) {
        ctx->h_gen[k] = mu[k];
        ctx->h_gen[n + k] = region ? region[k] : 0;
    }
    CK(cudaMemcpyAsync(ctx->d_gen, ctx->h_gen, 2 * (size_t)n * sizeof(int32_t), cudaMemcpyHostToDevice, stream),
       "upload mu/region");
    CK(cudaEventRecord(ctx->ev_gen, stream), "cudaEventRecord");
    GenParams g{seed, kind, ctx->d_gen, ctx->d_gen + n, n, S, ld, out};
    CK(launch_gen_demand(g, dtype, stream), "gen_demand launch");
    return CVRPSD_OK;
}

}  // extern "C"
