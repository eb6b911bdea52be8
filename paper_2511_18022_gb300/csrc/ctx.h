// Internal: the library context and its error helpers (shared by the C ABI
// translation units).
#pragma once

#include <cuda_runtime.h>
#include <stdarg.h>
#include <stdio.h>

#include "../../include/cvrpsd.h"
#include "kernels.h"

using cvrpsd::TourDev;
using cvrpsd::TourStep;

struct cvrpsd_ctx {
    int device = 0;
    int sm_count = 0;
    int max_smem = 48 * 1024;              // opt-in shared memory per block
    unsigned long long *d_acc = nullptr;   // ACC_WORDS
    int32_t *d_list = nullptr;             // overflow list
    long long list_cap = 0;
    TourStep *d_tab = nullptr;
    TourStep *h_tab = nullptr;             // pinned
    unsigned long long *h_acc = nullptr;   // pinned
    int32_t *d_gen = nullptr;              // mu[n], region[n]
    int32_t *h_gen = nullptr;              // pinned
    cudaEvent_t ev_tab = nullptr;          // tab upload done
    cudaEvent_t ev_gen = nullptr;          // gen upload done
    cudaEvent_t ev_t[3] = {nullptr, nullptr, nullptr};   // kernel timing (profiling)
    int profiling = 0;
    cvrpsd_config cfg{0, 0, 0, 0};
    cvrpsd_stats stats{};
    char err[512] = {0};
    // many tours of one instance (cvrpsd_split_eval_tours), grown on demand
    TourStep *mt_tabs = nullptr;
    long long mt_tabs_cap = 0;
    TourDev *mt_descs = nullptr;
    int mt_descs_cap = 0;
    unsigned long long *mt_acc = nullptr;
    int mt_acc_cap = 0;
    int2 *mt_list = nullptr;
    long long mt_list_cap = 0;
    int32_t *mt_dist = nullptr;
    long long mt_dist_cap = 0;
    int32_t *mt_dist_host = nullptr;       // pinned staging copy of the last distances uploaded
    long long mt_dist_host_cap = 0;
    unsigned long long mt_dist_key = 0;    // hash of those distances (with n); 0 = none
    int mt_dist_n = 0;
    cudaEvent_t ev_dist = nullptr;         // their upload done (the pinned copy is free again)
    // sequence-parallel Split scratch
    int32_t *seq_lo = nullptr;
    long long seq_lo_cap = 0;
    int32_t *seq_flags = nullptr;
    long long seq_flags_cap = 0;
    int32_t *seq_mats = nullptr;
    long long seq_mats_cap = 0;
    // test hook (cvrpsd_debug_fail_alloc): allocations left before one fails; -1 = off
    int fail_alloc_after = -1;
    // caller's log sink (cvrpsd_set_log)
    cvrpsd_log_fn log_fn = nullptr;
    void *log_user = nullptr;
    int log_level = -1;
};

namespace cvrpsd {

// A message to the context's log sink, if one takes this level.
inline void log_msg(cvrpsd_ctx *ctx, int level, const char *fmt, ...)
{
    if (!ctx || !ctx->log_fn || level > ctx->log_level) return;
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof(buf), fmt, ap);
    va_end(ap);
    ctx->log_fn(level, buf, ctx->log_user);
}

inline int fail(cvrpsd_ctx *ctx, int code, const char *fmt, ...)
{
    if (ctx) {
        va_list ap;
        va_start(ap, fmt);
        vsnprintf(ctx->err, sizeof(ctx->err), fmt, ap);
        va_end(ap);
        log_msg(ctx, CVRPSD_LOG_ERROR, "error %d: %s", code, ctx->err);
    }
    return code;
}

inline int cuda_fail(cvrpsd_ctx *ctx, cudaError_t e, const char *what)
{
    return fail(ctx, e == cudaErrorMemoryAllocation ? CVRPSD_ERR_NOMEM : CVRPSD_ERR_CUDA, "%s: %s", what,
                cudaGetErrorString(e));
}

// Every device and pinned-host allocation of a context goes through these, so
// that the test hook can make one of them fail as if memory had run out.
inline bool injected_alloc_failure(cvrpsd_ctx *ctx)
{
    if (!ctx || ctx->fail_alloc_after < 0) return false;
    if (ctx->fail_alloc_after == 0) {
        ctx->fail_alloc_after = -1;
        return true;
    }
    --ctx->fail_alloc_after;
    return false;
}
template <typename T>
inline cudaError_t dev_alloc(cvrpsd_ctx *ctx, T **p, size_t bytes)
{
    if (injected_alloc_failure(ctx)) {
        *p = nullptr;
        return cudaErrorMemoryAllocation;
    }
    return cudaMalloc(reinterpret_cast<void **>(p), bytes);
}
template <typename T>
inline cudaError_t host_alloc(cvrpsd_ctx *ctx, T **p, size_t bytes)
{
    if (injected_alloc_failure(ctx)) {
        *p = nullptr;
        return cudaErrorMemoryAllocation;
    }
    return cudaMallocHost(reinterpret_cast<void **>(p), bytes);
}

}  // namespace cvrpsd
