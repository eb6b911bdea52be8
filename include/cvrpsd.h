/*
 * cvrpsd.h - C ABI of the GB300 scenario-batched Split for the CVRP with
 * stochastic demands.
 *
 * Method: Zhao, Yang, Zhang, Ding, "GPU-based Split algorithm for Large-Scale
 * CVRPSD". Given a giant tour sigma_1..sigma_n of customers (Section 3) and S
 * demand scenarios, the Split of scenario w is the dynamic program of Eq. 1:
 *
 *   f(0) = 0,  f(i) = min_{p <= i-1} f(p) + c(0, sigma_{p+1})
 *                    + sum_{k=p+1}^{i-1} c(sigma_k, sigma_{k+1}) + c(sigma_i, 0)
 *   over the p whose route sigma_{p+1}..sigma_i carries load <= Q,
 *
 * which Eq. 2 and Eq. 3 restate as a min over the window
 * [mask_w(i), i-1] of candidates. The scenario cost is f(n); Appendix A's
 * sample-average estimate is the mean of f(n) over the scenarios.
 *
 * Conventions shared by every entry point:
 *  - Node 0 of `dist` is the depot and also the paper's return depot n+1.
 *    `dist` is (n+1) x (n+1) int32, row-major, row = from, column = to, on the
 *    HOST, all used entries >= 0.
 *  - `tour` is a HOST array of n int32 customer ids, a permutation of 1..n.
 *  - Demands live on the DEVICE as a [n][ld] matrix: row k-1 holds customer k
 *    (by id, not by tour position), scenario s is column s, scenarios are
 *    contiguous. Element type int16 (CVRPSD_I16) or int32 (CVRPSD_I32),
 *    values >= 0. `ld` >= S is the row pitch in elements.
 *  - Q >= 0 is the vehicle capacity. L is the largest number of customers on
 *    one route (this library's reading of the optional route-length limit of
 *    Section 3); L >= n means no limit. The fleet is unlimited.
 *  - A scenario in which some customer's demand exceeds Q has no feasible
 *    split (Eq. 2's window is empty): its cost is INT32_MAX, it is left out
 *    of the sum and the mean, and it is counted as infeasible; the call then
 *    returns CVRPSD_WARN_INFEASIBLE (outputs are still valid).
 *  - Costs are exact integers. Per-scenario costs are int32; sums are int64.
 *  - The caller owns every buffer; the library never frees caller memory.
 *    Work is enqueued on `stream` (a cudaStream_t, NULL = legacy default).
 *  - Return value: 0 on success, CVRPSD_WARN_INFEASIBLE (> 0), or a negative
 *    error code; cvrpsd_strerror() names it and cvrpsd_last_error() gives the
 *    detail of the last failure on that context. On error no output is
 *    written unless stated otherwise.
 *  - A context may be used by one host thread at a time.
 */
#ifndef CVRPSD_H
#define CVRPSD_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define CVRPSD_OK                  0
#define CVRPSD_WARN_INFEASIBLE     1
#define CVRPSD_ERR_ARG            -1   /* bad size, pointer, Q, L, or tour */
#define CVRPSD_ERR_DTYPE          -2   /* demand element type not supported */
#define CVRPSD_ERR_OVERFLOW       -3   /* costs could exceed int32 */
#define CVRPSD_ERR_CUDA           -4   /* a CUDA runtime call failed */
#define CVRPSD_ERR_DEVICE_STATUS  -5   /* a kernel reported a bad input */
#define CVRPSD_ERR_NOMEM          -6   /* scratch allocation failed */
#define CVRPSD_ERR_UNSUPPORTED    -7   /* size beyond the library's limits */
#define CVRPSD_ERR_TIMEOUT        -8   /* a device-side wait gave up (bounded polls) */

#define CVRPSD_I16  2
#define CVRPSD_I32  4

/* Largest tour the library accepts. */
#define CVRPSD_MAX_N 8191

/* Kernel choice for the Split (see cvrpsd_config). AUTO takes SEQPAR for
 * S <= 256 scenarios on tours of n >= 128 (lowest latency there) and DEQUE
 * otherwise. */
#define CVRPSD_KERNEL_AUTO   0
#define CVRPSD_KERNEL_DEQUE  1   /* one thread per scenario, monotone deque */
#define CVRPSD_KERNEL_WARP   2   /* one warp per scenario, parallel window min */
#define CVRPSD_KERNEL_SEQPAR 3   /* few scenarios: min-plus matrix products over blocks of
                                    positions, parallel along the tour (S <= 4096) */

/* Demand kinds of the scenario generator. */
#define CVRPSD_GEN_NORMAL      0
#define CVRPSD_GEN_CORRELATED  1

typedef struct cvrpsd_ctx cvrpsd_ctx;

/* Walks of the deque kernel (cvrpsd_config.variant). */
#define CVRPSD_WALK_AUTO          0   /* PARAM_TABLE where it applies, else GLOBAL_TABLE */
#define CVRPSD_WALK_GLOBAL_TABLE  1   /* tour table in global memory; any n, spt 1 or 2 */
#define CVRPSD_WALK_PARAM_TABLE   2   /* tour table in the launch's parameters: n <= 4032, spt 1,
                                         int16 demands need Q < 32768; rings of 8 or 16 */

/* Launch shape of the Split. threads in {64,128,256} per block (512 for the
 * batched path; single-tour calls then run 256), spt
 * (scenarios per thread) in {1,2}, ring (deque capacity per scenario) in
 * {8,16,32,64} (8 only with the parameter-table walk), variant one of
 * CVRPSD_WALK_*, rounds >= 0: with rounds = 0 every thread walks one
 * scenario; with rounds = r >= 1 (parameter-table walk) the grid has
 * ceil(tiles / r) blocks and each walks up to r tiles of `threads`
 * scenarios, one after the other. Zero fields mean "library default /
 * autotuned". A shape or walk that does not apply to a call is replaced by
 * the nearest one that does (cvrpsd_last_stats reports what ran). */
typedef struct {
    int32_t kernel;
    int32_t threads;
    int32_t spt;
    int32_t ring;
    int32_t variant;
    int32_t rounds;
} cvrpsd_config;

/* What the last Split call on a context did. */
typedef struct {
    int32_t kernel;            /* kernel that evaluated the scenarios */
    int32_t threads, spt, ring;
    int64_t overflow;          /* scenarios the warp kernel re-evaluated (deque ring too
                                  small, demand above Q or negative), -1 if not read back */
    int32_t launches;          /* kernels launched by the call */
    float kernel_ms;           /* device time of the main Split kernel, -1 unless profiling */
    float fallback_ms;         /* device time of the overflow pass, -1 unless profiling */
    int32_t variant;           /* deque walk that ran (CVRPSD_WALK_*), 0 for other kernels */
    int32_t rounds;            /* tiles per block of that walk (0: one scenario per thread) */
} cvrpsd_stats;

/* Create a context bound to CUDA device `device`. Allocates small scratch
 * lazily on first use. Returns CVRPSD_ERR_CUDA if the device is unusable. */
int cvrpsd_create(cvrpsd_ctx **ctx, int device);

/* Release a context and its scratch. Waits for nothing: the caller must not
 * destroy a context while work it enqueued is still running. */
int cvrpsd_destroy(cvrpsd_ctx *ctx);

const char *cvrpsd_strerror(int code);
const char *cvrpsd_last_error(const cvrpsd_ctx *ctx);
const char *cvrpsd_version(void);

/* Fix the launch shape used by later Split calls on `ctx` (testing and
 * tuning). Returns CVRPSD_ERR_ARG for values outside the listed sets. */
int cvrpsd_set_config(cvrpsd_ctx *ctx, const cvrpsd_config *cfg);
int cvrpsd_get_config(const cvrpsd_ctx *ctx, cvrpsd_config *cfg);
int cvrpsd_last_stats(const cvrpsd_ctx *ctx, cvrpsd_stats *stats);

/* With on != 0, later Split calls that return host outputs also time their
 * kernels with CUDA events recorded on the call's stream and report the
 * durations in cvrpsd_stats. Off by default. */
int cvrpsd_set_profiling(cvrpsd_ctx *ctx, int32_t on);

/* Messages of a context go to a caller-supplied function and nowhere else
 * (the library never prints). Levels: */
#define CVRPSD_LOG_ERROR 0   /* the detail of every failing call (also cvrpsd_last_error) */
#define CVRPSD_LOG_INFO  1   /* tuning results, batch set-up */
#define CVRPSD_LOG_DEBUG 2   /* per call: the kernel, walk and launch shape a Split ran */
typedef void (*cvrpsd_log_fn)(int32_t level, const char *message, void *user);

/* Route messages of level <= max_level to fn(level, message, user), called
 * on the thread that makes the library call; fn = NULL turns logging off
 * (the default). The message is valid only during the call. */
int cvrpsd_set_log(cvrpsd_ctx *ctx, cvrpsd_log_fn fn, void *user, int32_t max_level);

/* Input errors of calls that did not wait. A Split call that requests no
 * host output returns once its work is enqueued, before the kernels have
 * looked at the demands; a negative demand found there (that scenario's
 * cost is then evaluated with it read as zero) cannot be returned by the
 * call itself. Every Split on
 * the context also records such findings in a status word that only this
 * function clears: it waits for `stream` (which must be ordered after the
 * calls to check), returns CVRPSD_ERR_DEVICE_STATUS if any Split since the
 * previous check found a negative demand (CVRPSD_OK otherwise), and clears
 * the record. Calls that return host outputs report the error themselves as
 * well. */
int cvrpsd_check_inputs(cvrpsd_ctx *ctx, void *stream);

/* Test hook for the error paths: after `after` more device or pinned-host
 * allocations made for `ctx` (its scratch, batches, surrogates), the next one
 * fails as if memory had run out (the call returns CVRPSD_ERR_NOMEM and
 * leaves the context usable); after < 0 turns the hook off. The hook fires
 * once. Not for production use. */
int cvrpsd_debug_fail_alloc(cvrpsd_ctx *ctx, int32_t after);

/*
 * Split one giant tour under S scenarios (Section 3, Eq. 1-3) and reduce the
 * costs to the sample-average of Appendix A.
 *
 *  tour[n], dist[(n+1)^2]  HOST, see conventions; 1 <= n <= CVRPSD_MAX_N.
 *  demand                  DEVICE [n][ld], element type demand_dtype.
 *  S >= 0, ld >= S         scenarios and row pitch (elements).
 *  Q >= 0, L >= 1          capacity and route-length limit.
 *  out_cost                DEVICE int32[S] or NULL: f(n) per scenario,
 *                          INT32_MAX where infeasible.
 *  out_sum, out_infeasible HOST int64 or NULL: exact sum of feasible costs,
 *                          number of infeasible scenarios.
 *  out_mean                HOST double or NULL: out_sum / (S - infeasible),
 *                          NaN when no scenario is feasible or S == 0.
 *  stream                  cudaStream_t.
 *
 * If any host output is requested the call waits for `stream` to finish its
 * work; otherwise it returns once the work is enqueued. Rejects device
 * buffers too small for [n][ld] / [S] with CVRPSD_ERR_ARG, and inputs whose
 * costs could overflow int32 with CVRPSD_ERR_OVERFLOW.
 */
int cvrpsd_split_eval(cvrpsd_ctx *ctx, const int32_t *tour, int32_t n,
                      const int32_t *dist, const void *demand,
                      int32_t demand_dtype, int64_t S, int64_t ld, int32_t Q,
                      int32_t L, int32_t *out_cost, int64_t *out_sum,
                      int64_t *out_infeasible, double *out_mean, void *stream);

/*
 * cvrpsd_split_eval on HOST buffers: the scenario matrix stays in host
 * memory (an addition of this library, not a step of the paper's method).
 *
 *  demand    HOST [n][ld], page-locked and mapped into the device's address
 *            space (cudaHostAlloc / cudaMallocHost, or cudaHostRegister with
 *            cudaHostRegisterMapped). The kernels read it in place across
 *            the host link: every demand crosses the link exactly once, with
 *            no staging copy in device memory.
 *  out_cost  HOST int32[S] or NULL, page-locked and mapped like `demand`;
 *            written in place by the kernels.
 *  other arguments as for cvrpsd_split_eval.
 *
 * Always waits for `stream` before returning (the kernels use the host
 * buffers until then), so the caller may reuse or free them afterwards.
 * Pageable or unknown memory is rejected with CVRPSD_ERR_ARG; so is a buffer
 * smaller than [n][ld] / [S] wherever the driver reports the allocation's
 * extent (the caller guarantees the extent otherwise).
 */
int cvrpsd_split_eval_host(cvrpsd_ctx *ctx, const int32_t *tour, int32_t n,
                           const int32_t *dist, const void *demand,
                           int32_t demand_dtype, int64_t S, int64_t ld,
                           int32_t Q, int32_t L, int32_t *out_cost,
                           int64_t *out_sum, int64_t *out_infeasible,
                           double *out_mean, void *stream);

/*
 * cvrpsd_split_eval that also recovers the optimal routes (the Section 2
 * Example lists a scenario's routes). For every scenario s and position
 * i = 1..n, pred[(i-1) * ldp + s] (DEVICE int16, [n][ldp], ldp >= S) receives
 * the p that attains f(i) in Eq. 1 -- the route ending at sigma_i starts at
 * sigma_{p+1} -- taking the smallest such p on ties. The routes of scenario
 * s follow by walking p = pred[n-1][s], pred[p-1][s], ... down to 0.
 * Entries of infeasible scenarios are unspecified. Writing 2 bytes per
 * (scenario, position) doubles the HBM traffic of the Split.
 */
int cvrpsd_split_routes(cvrpsd_ctx *ctx, const int32_t *tour, int32_t n,
                        const int32_t *dist, const void *demand,
                        int32_t demand_dtype, int64_t S, int64_t ld, int32_t Q,
                        int32_t L, int32_t *out_cost, int16_t *pred, int64_t ldp,
                        int64_t *out_sum, int64_t *out_infeasible,
                        double *out_mean, void *stream);

/*
 * Seeded scenario generator (workload synthesis, not part of the paper's
 * method). Writes demand[k-1][s] for customers k = 1..n and scenarios
 * s = 0..S-1 into the DEVICE [n][ld] matrix `out` of type `dtype`:
 *   CVRPSD_GEN_NORMAL:     max(0, round(mu_k + 0.3 mu_k Z_sk))
 *   CVRPSD_GEN_CORRELATED: max(0, round(mu_k exp(0.3 (0.6 F_{s,r_k}
 *                                                  + 0.8 E_sk) - 0.045)))
 * with Z, E, F standard normals from Philox4x32-10 (counter (s, index,
 * domain, 0), key = seed halves) by Box-Muller in float64, round half away
 * from zero, clamped to the type's maximum. mu[n], region[n] (quadrant
 * 0..3 of customer k at [k-1]) are HOST arrays. Asynchronous on `stream`.
 */
int cvrpsd_gen_demand(cvrpsd_ctx *ctx, uint64_t seed, int32_t kind,
                      const int32_t *mu, const int32_t *region, int32_t n,
                      int64_t S, int64_t ld, int32_t dtype, void *out,
                      void *stream);

/* ---- Autotuning the launch shape ---- */
typedef struct {
    cvrpsd_config best;     /* fastest shape; also set as the context's configuration */
    float best_ms;          /* its device time per Split (main kernel + set-aside pass) */
    int32_t best_dtype;     /* CVRPSD_I16 or CVRPSD_I32: the faster demand storage, timed on a
                               sample of min(S, 65536) scenarios (int16 only if every demand fits) */
    int32_t shapes_timed;   /* shapes swept by this call; 0 when the result came from the cache */
} cvrpsd_tune_result;

/*
 * Time every launch shape of the scenario-parallel kernel (threads x spt x
 * ring, see cvrpsd_config) on this workload with CUDA events on `stream`,
 * check that each shape gives exactly the sum and infeasible count of the
 * default shape (CVRPSD_ERR_DEVICE_STATUS otherwise), and keep the fastest.
 * Arguments as for cvrpsd_split_eval; out_cost is not written. With
 * cache_path != NULL, a result stored under the same key (GPU name, n rounded
 * up to a power of two, S rounded down to a power of two, demand type,
 * whether L limits routes) is reused, and a new result is appended to that
 * file (one JSON object per line). Allocates temporary device buffers for the
 * demand-type comparison. Synchronous.
 */
int cvrpsd_autotune(cvrpsd_ctx *ctx, const int32_t *tour, int32_t n, const int32_t *dist, const void *demand,
                    int32_t demand_dtype, int64_t S, int64_t ld, int32_t Q, int32_t L, const char *cache_path,
                    cvrpsd_tune_result *result, void *stream);

/* ---- Batches of tours: one persistent launch, captured in a CUDA graph ----
 *
 * Many giant tours (Section 3; in the paper's setting, the candidate tours a
 * metaheuristic evaluates), each with its own customers, distances, demand
 * matrix, Q and L, all under S scenarios. The library packs the tours'
 * tables, orders the work (largest tours first) and captures the whole
 * evaluation -- clearing the accumulators, one persistent Split kernel whose
 * blocks take (tour, scenario tile) items from an atomic counter, the warp
 * kernel for set-aside scenarios, and the copy of the per-tour sums to pinned
 * host memory -- into one CUDA graph at creation. */
typedef struct {
    const int32_t *tour;   /* HOST [n]: customer ids, a permutation of 1..n */
    int32_t n;             /* 1 <= n <= CVRPSD_MAX_N */
    const int32_t *dist;   /* HOST [(n+1)^2], node 0 = depot */
    const void *demand;    /* DEVICE [n][ld], the batch's demand type */
    int64_t ld;            /* row pitch in elements, >= S */
    int32_t Q;             /* capacity >= 0 */
    int32_t L;             /* route-length limit >= 1 (>= n: none) */
    int32_t *out_cost;     /* DEVICE [S] or NULL */
} cvrpsd_tour_desc;

typedef struct cvrpsd_batch cvrpsd_batch;

/* Validate and pack T >= 1 tours, allocate the batch's device scratch and
 * capture its graph (the launch shape is the context's configuration, or the
 * default). The host arrays are read only during this call; the device
 * buffers must stay valid for the batch's lifetime. Errors as for
 * cvrpsd_split_eval; a bad tour is reported with its index in
 * cvrpsd_last_error. */
int cvrpsd_batch_create(cvrpsd_ctx *ctx, int32_t T, const cvrpsd_tour_desc *tours, int64_t S,
                        int32_t demand_dtype, cvrpsd_batch **batch);

/* Enqueue one evaluation of the batch (a graph launch) on `stream`. The
 * demand matrices may change between runs; the tours may not. Runs of one
 * batch must not overlap. */
int cvrpsd_batch_run(cvrpsd_batch *batch, void *stream);

/* Wait for the last run and return per-tour results (arrays of T, each may be
 * NULL): exact sum of feasible costs, infeasible count, mean (NaN if no
 * scenario is feasible), and a status (0, CVRPSD_WARN_INFEASIBLE or
 * CVRPSD_ERR_DEVICE_STATUS for a negative demand). Returns the worst
 * status. */
int cvrpsd_batch_results(cvrpsd_batch *batch, int64_t *out_sum, int64_t *out_infeasible, double *out_mean,
                         int32_t *out_status);

int cvrpsd_batch_destroy(cvrpsd_batch *batch);

/*
 * Autotuner of the batched path: for every launch shape of the persistent
 * batch kernel -- scenarios per block 32 to 512 (threads {32, 64, 128, 256}
 * x scenarios per thread {1, 2}) x deque ring (window tile) {16, 32, 64},
 * rings of 64 up to 128 threads, plus 512 threads with rings of 16: 21
 * shapes -- create this batch, time its
 * graph with CUDA events on `stream` (best of three runs after one warm-up),
 * and check that every tour's sum and infeasible count equal those of the
 * first shape (CVRPSD_ERR_DEVICE_STATUS otherwise). The fastest shape becomes
 * the context's configuration, so the next cvrpsd_batch_create uses it. Then
 * the demand storage: the best shape runs on int16 and int32 copies of a
 * sample of every tour's scenarios (at most 8192 columns and 2 GB of
 * copies), both must give the same results, and result->best_dtype names the
 * faster (int16 only if every demand fits). Arguments as for
 * cvrpsd_batch_create. Synchronous; allocates the sample copies.
 */
int cvrpsd_batch_autotune(cvrpsd_ctx *ctx, int32_t T, const cvrpsd_tour_desc *tours, int64_t S,
                          int32_t demand_dtype, cvrpsd_tune_result *result, void *stream);

/* One-shot batch: create, run on `stream`, read the results, destroy. */
int cvrpsd_split_eval_batch(cvrpsd_ctx *ctx, int32_t T, const cvrpsd_tour_desc *tours, int64_t S,
                            int32_t demand_dtype, int64_t *out_sum, int64_t *out_infeasible,
                            double *out_mean, int32_t *out_status, void *stream);

/* ---- Local search around the Split, on device-resident candidate tours ----
 *
 * The paper embeds the Split in a metaheuristic that evaluates many candidate
 * giant tours of one instance (Section 1; the fixed-budget search of Section
 * 4.3). These entry points keep the candidates on the device: they build
 * neighbours, split all of them under the scenario set, pick the best, and
 * screen neighbours with a learned surrogate. All are asynchronous on
 * `stream`; every pointer named d_* is DEVICE memory. */

/* SAA evaluation of T tours of one instance: d_tours [T][n] (each a
 * permutation of 1..n; other values are clamped into range and give
 * meaningless results), dist HOST (n+1)^2, demand DEVICE [n][ld] shared by all
 * tours. Writes per tour d_mean (double, NaN if no scenario is feasible),
 * d_sum and d_infeasible (int64); any of them may be NULL. Same arithmetic
 * and bit-exact results as cvrpsd_split_eval per tour. */
int cvrpsd_split_eval_tours(cvrpsd_ctx *ctx, const int32_t *d_tours, int32_t T, int32_t n,
                            const int32_t *dist, const void *demand, int32_t demand_dtype,
                            int64_t S, int64_t ld, int32_t Q, int32_t L, double *d_mean,
                            int64_t *d_sum, int64_t *d_infeasible, void *stream);

/* Neighbours of d_base [n] under M moves d_moves [M][3] = (type, a, b) with
 * 0 <= a, b < n (values outside are clamped): type 0 reverses positions a..b
 * (2-opt), type 1 moves the customer at position a so that it ends at
 * position b (relocate). Writes d_out [M][n]. */
int cvrpsd_neighbors(cvrpsd_ctx *ctx, const int32_t *d_base, int32_t n, const int32_t *d_moves,
                     int32_t M, int32_t *d_out, void *stream);

/* Indices of the k smallest of d_scores [M] (1 <= k <= M <= 16384),
 * ascending, ties to the smaller index, NaN last. Writes d_idx [k]. */
int cvrpsd_topk(cvrpsd_ctx *ctx, const float *d_scores, int32_t M, int32_t k, int32_t *d_idx,
                void *stream);

/* d_out[r] = d_tours[d_idx[r]] for R rows of n ints; d_tours has `rows`
 * rows and indices outside 0..rows-1 are clamped. */
int cvrpsd_gather_tours(cvrpsd_ctx *ctx, const int32_t *d_tours, int32_t rows, int32_t n,
                        const int32_t *d_idx, int32_t R, int32_t *d_out, void *stream);

/* The search's improvement step (the fixed-budget search of Section 4.3):
 * among T candidate tours d_tours [T][n] with exact costs d_cost [T] (e.g.
 * the d_mean of cvrpsd_split_eval_tours), take the cheapest, the smallest
 * index among equal costs (a NaN cost is never taken), and accept it if it
 * is strictly cheaper than *d_cur_cost: then it is copied to d_cur [n] and
 * its cost stored in *d_cur_cost. d_trace (optional, one double) receives
 * *d_cur_cost after the step. d_cur must not overlap d_tours
 * (CVRPSD_ERR_ARG). One kernel on `stream`; nothing waits. */
int cvrpsd_accept_best(cvrpsd_ctx *ctx, const int32_t *d_tours, int32_t T, int32_t n,
                       const double *d_cost, int32_t *d_cur, double *d_cur_cost, double *d_trace,
                       void *stream);

/* Surrogate of a tour's SAA cost for screening neighbours (not part of the
 * paper's method). Per position k it sees (x, y, mean demand, demand sd,
 * fractional part of the cumulative mean demand / Q) of the customer there;
 * layer 1 (256 units, ReLU) runs per position and is mean-pooled, the tour's
 * closed length joins (see cvrpsd_surrogate_set_scale), layer 2 (256, ReLU)
 * and layer 3 (scalar) follow. BF16 weights and per-position features, FP32
 * accumulation, Adam on FP32 master weights. Layer 1's forward pass runs on
 * the tensor cores (tcgen05 MMAs, accumulators in tensor memory). */
typedef struct cvrpsd_surrogate cvrpsd_surrogate;
#define CVRPSD_SURROGATE_PARAMS 67841

/* cust: HOST [n][4] = (x, y, mean demand, demand sd) of customer k at k-1
 * (coordinates on the 0..1000 scale); dist HOST (n+1)^2; Q > 0; 1 <= n <= 4096;
 * parameters drawn from `seed`. */
int cvrpsd_surrogate_create(cvrpsd_ctx *ctx, int32_t n, const float *cust, const int32_t *dist,
                            float Q, uint64_t seed, cvrpsd_surrogate **sur);
int cvrpsd_surrogate_destroy(cvrpsd_surrogate *sur);
/* d_pred [T] = network output for d_tours [T][n]. */
int cvrpsd_surrogate_predict(cvrpsd_surrogate *sur, const int32_t *d_tours, int32_t T, float *d_pred,
                             void *stream);
/* One Adam step (rate lr) on the mean squared error to d_target [T]; the
 * batch loss goes to d_loss (device float) if not NULL. */
int cvrpsd_surrogate_train_step(cvrpsd_surrogate *sur, const int32_t *d_tours, int32_t T,
                                const float *d_target, float lr, float *d_loss, void *stream);
/* Gradient of that loss w.r.t. all parameters, without updating them
 * (synchronous): h_grad HOST [CVRPSD_SURROGATE_PARAMS], h_loss HOST or NULL.
 * Also reports CVRPSD_ERR_TIMEOUT if a tensor-core kernel of this network
 * (this or an earlier call) gave up waiting for its MMAs. */
int cvrpsd_surrogate_gradients(cvrpsd_surrogate *sur, const int32_t *d_tours, int32_t T,
                               const float *d_target, float *h_grad, float *h_loss);
/* The tour-length input becomes (closed tour length - len_mean) / len_sd
 * (default len_mean = 0, len_sd = 500 n); set it from the training tours so
 * that the small length differences between neighbours are visible. */
int cvrpsd_surrogate_set_scale(cvrpsd_surrogate *sur, float len_mean, float len_sd);

/* Read (h_get) and/or replace (h_set) the FP32 parameters (HOST arrays of
 * CVRPSD_SURROGATE_PARAMS: W1 [256][5], b1 [256], W2 [256][257], b2 [256],
 * w3 [256], b3); *count receives the size. Synchronous. */
int cvrpsd_surrogate_params(cvrpsd_surrogate *sur, float *h_get, const float *h_set, int64_t *count);

/*
 * Checkpoint of the surrogate trainer: a flat host blob of *bytes bytes
 * (header: magic, version, n, parameter count, Adam step, tour-length scale;
 * then the fp32 parameters and Adam's first and second moments). With h_get
 * the current state is written there; with h_set the state is restored from
 * a blob taken from a network of the same n (CVRPSD_ERR_ARG otherwise), so
 * that training resumes where it stopped. Synchronous (waits for the device).
 * An addition of this library: the paper trains no network.
 */
int cvrpsd_surrogate_state(cvrpsd_surrogate *sur, void *h_get, const void *h_set, int64_t *bytes);

/*
 * Measured rate of 32-bit integer min/max instructions on `device` (the
 * operation of Eq. 3's window minimum: one min per candidate predecessor),
 * for the integer-ALU roofline of a Split launch. Runs one kernel of eight
 * independent min/max chains per thread on a full grid (every SM at full
 * occupancy), `iters` x 64 min/max per thread, timed with CUDA events on
 * `stream`. *ops_per_s receives thread-level operations per second (one warp
 * instruction = 32 operations), *ms (may be NULL) the kernel time.
 * Synchronous; allocates 4 bytes of device memory. Not a step of the paper's
 * method: a measurement helper.
 */
int cvrpsd_int_rate(int32_t device, int32_t iters, double *ops_per_s, double *ms, void *stream);

/* Largest S accepted by cvrpsd_split_eval_noalloc. */
#define CVRPSD_NOALLOC_MAX_S 1048576

/*
 * cvrpsd_split_eval for callers that cannot allocate device memory when they
 * call: programs that hand all device memory to their own pool at start-up,
 * and loops where a cudaMalloc could block on the device or fail under memory
 * pressure. The paper has no counterpart; this is a deployment variant.
 *
 * Same inputs, outputs, conventions and results as cvrpsd_split_eval, on the
 * current CUDA device and without a context. Its scratch (accumulators, the
 * tour table, the list of scenarios handed to the warp kernel) is one
 * file-scope device array of about 4.1 MiB. Every device that loads the
 * library holds it until the library is unloaded. The call allocates no device memory
 * (no cudaMalloc, no cudaFree). Limits: 1 <= n <= CVRPSD_MAX_N and
 * 0 <= S <= CVRPSD_NOALLOC_MAX_S; a larger S returns CVRPSD_ERR_UNSUPPORTED.
 *
 * The first call on a device looks up the array's device address
 * (cudaGetSymbolAddress) and the device limits; make that first call before
 * any stream capture. Every call on a device shares the one array: each call
 * clears the accumulators it needs, but two calls whose work overlaps on the
 * GPU (different streams, or host threads) race on it and must be serialised
 * by the caller. Errors are returned as codes only (no message).
 *
 * The tour table travels through one process-wide host staging buffer, so a
 * call on a stream that is being captured into a CUDA graph is refused with
 * CVRPSD_ERR_UNSUPPORTED (a recorded copy would read that buffer when the
 * graph runs, after later calls have changed it). Without host outputs the
 * call returns before its kernels run, so a negative demand (read as zero by
 * the kernels) is not reported; request a host output to have it reported
 * as CVRPSD_ERR_DEVICE_STATUS.
 */
int cvrpsd_split_eval_noalloc(const int32_t *tour, int32_t n,
                              const int32_t *dist, const void *demand,
                              int32_t demand_dtype, int64_t S, int64_t ld,
                              int32_t Q, int32_t L, int32_t *out_cost,
                              int64_t *out_sum, int64_t *out_infeasible,
                              double *out_mean, void *stream);

#ifdef __cplusplus
}
#endif

#endif /* CVRPSD_H */
