/*
 * Oracle for the scenario-batched Split of a CVRPSD giant tour.
 *
 * TEST INFRASTRUCTURE ONLY. Only the tests, the smoke check and the CPU
 * baseline of the benchmark may load this library; the product path never
 * does, and it shares no code with the CUDA implementation.
 *
 * What it computes (Zhao, Yang, Zhang, Ding, "GPU-based Split algorithm for
 * Large-Scale CVRPSD", Section 3, Eq. 1): for one demand scenario w and a giant
 * tour sigma_1..sigma_n between depot nodes sigma_0 = 0 and sigma_{n+1},
 *
 *   f(0) = 0,
 *   f(i) = min over 0 <= p <= i-1 of
 *            f(p) + c(0, sigma_{p+1}) + sum_{k=p+1}^{i-1} c(sigma_k, sigma_{k+1})
 *                 + c(sigma_i, n+1)
 *          subject to sum_{k=p+1}^{i} q(sigma_k) <= Q,
 *
 * and the scenario's cost is f(n). Readings taken where the paper is silent:
 *   - the return depot n+1 is node 0 of the distance matrix (same place);
 *   - demands are stored by customer id (row k-1 holds customer k), not by
 *     tour position;
 *   - the optional route limit of Section 3 is "at most L customers per route",
 *     i.e. p >= i - L (L >= n means no limit);
 *   - a scenario in which some customer's demand exceeds Q has no feasible
 *     split: its cost is reported as INT32_MAX and it is left out of the
 *     sample-average sum (Appendix A) and counted separately;
 *   - the fleet is unlimited (Eq. 1 has no vehicle bound).
 *
 * The candidate p walks down from i-1, adding one customer's demand and one
 * tour edge per step, so load and segment length are the sums in Eq. 1 for
 * that p. Demands are non-negative, so once the load exceeds Q (or the route
 * exceeds L customers) every smaller p does too, and the walk stops there.
 * All arithmetic is 64-bit integer; nothing is rounded.
 *
 * It uses neither the earliest-feasible-split masks of Eq. 2 nor any
 * rearrangement of the segment cost: each candidate is costed as written.
 */
#include <pthread.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define ORACLE_INF INT64_MAX

/* Demand of customer id c (1..n) in the scenario column `s` of a [n][ld]
 * matrix whose elements are `esize` bytes (2 = int16, 4 = int32). */
static int64_t demand_at(const void *demand, int esize, int64_t ld, int32_t c,
                         int64_t s)
{
    int64_t off = (int64_t)(c - 1) * ld + s;
    if (esize == 2) return (int64_t)((const int16_t *)demand)[off];
    return (int64_t)((const int32_t *)demand)[off];
}

/* Eq. 1 for one scenario. f must hold n+1 entries. Returns f(n), or -1 when
 * no feasible split exists. *relax (if not NULL) is incremented by the number
 * of feasible (p, i) pairs examined. If pred is not NULL, pred[i] receives the
 * smallest p attaining the minimum for f(i). */
int64_t oracle_split_scenario(int32_t n, const int32_t *tour, const int32_t *dist,
                              const void *demand, int esize, int64_t ld,
                              int64_t s, int64_t Q, int32_t L, int64_t *f,
                              int64_t *relax, int32_t *pred)
{
    const int64_t N1 = (int64_t)n + 1;
    int64_t count = 0;
    f[0] = 0;
    for (int32_t i = 1; i <= n; ++i) {
        const int32_t last = tour[i - 1];               /* sigma_i */
        int64_t best = ORACLE_INF;
        int32_t best_p = -1;
        int64_t load = 0;
        int64_t inner = 0;                              /* sum of tour edges inside the route */
        for (int32_t p = i - 1; p >= 0; --p) {
            if (i - p > L) break;                       /* route would exceed L customers */
            const int32_t first = tour[p];              /* sigma_{p+1} */
            load += demand_at(demand, esize, ld, first, s);
            if (load > Q) break;                        /* capacity constraint of Eq. 1 */
            if (p < i - 1) inner += dist[(int64_t)tour[p] * N1 + tour[p + 1]];
            ++count;
            if (f[p] == ORACLE_INF) continue;
            int64_t cost = f[p] + dist[0 * N1 + first] + inner + dist[(int64_t)last * N1 + 0];
            if (cost < best || (cost == best && p < best_p)) {
                best = cost;
                best_p = p;
            }
        }
        f[i] = best;
        if (pred) pred[i] = best_p;
    }
    if (relax) *relax += count;
    return f[n] == ORACLE_INF ? -1 : f[n];
}

typedef struct {
    int32_t n;
    const int32_t *tour;
    const int32_t *dist;
    const void *demand;
    int esize;
    int64_t ld;
    int64_t s_begin, s_end;       /* scenario columns [s_begin, s_end) */
    int64_t Q;
    int32_t L;
    int32_t *out_cost;            /* indexed by s - s_first */
    int64_t s_first;
    int64_t relax;
    int64_t sum;
    int64_t infeasible;
    int status;
} oracle_job;

static void *oracle_worker(void *arg)
{
    oracle_job *j = (oracle_job *)arg;
    int64_t *f = (int64_t *)malloc(sizeof(int64_t) * ((size_t)j->n + 1));
    if (!f) { j->status = -1; return NULL; }
    for (int64_t s = j->s_begin; s < j->s_end; ++s) {
        int64_t c = oracle_split_scenario(j->n, j->tour, j->dist, j->demand, j->esize,
                                          j->ld, s, j->Q, j->L, f, &j->relax, NULL);
        int32_t out;
        if (c < 0) {
            out = INT32_MAX;
            j->infeasible += 1;
        } else if (c >= INT32_MAX) {
            out = INT32_MAX;
            j->status = -2;       /* cost does not fit the int32 output */
        } else {
            out = (int32_t)c;
            j->sum += c;
        }
        if (j->out_cost) j->out_cost[s - j->s_first] = out;
    }
    free(f);
    return NULL;
}

/* Split of scenarios [s0, s0+count) of a [n][ld] demand matrix, spread over
 * `nthreads` POSIX threads by contiguous scenario ranges.
 * out_cost[count] gets per-scenario costs (INT32_MAX = infeasible),
 * out3[0] = sum of feasible costs, out3[1] = number of infeasible scenarios,
 * out3[2] = number of feasible (p, i) pairs examined.
 * Returns 0, or a negative value on allocation failure / int32 overflow. */
int oracle_split_many(int32_t n, const int32_t *tour, const int32_t *dist,
                      const void *demand, int esize, int64_t ld, int64_t s0,
                      int64_t count, int64_t Q, int32_t L, int32_t *out_cost,
                      int64_t *out3, int nthreads)
{
    if (nthreads < 1) nthreads = 1;
    if (count < nthreads) nthreads = count > 0 ? (int)count : 1;
    oracle_job *jobs = (oracle_job *)calloc((size_t)nthreads, sizeof(oracle_job));
    pthread_t *th = (pthread_t *)calloc((size_t)nthreads, sizeof(pthread_t));
    if (!jobs || !th) { free(jobs); free(th); return -1; }
    for (int t = 0; t < nthreads; ++t) {
        oracle_job *j = &jobs[t];
        j->n = n; j->tour = tour; j->dist = dist; j->demand = demand;
        j->esize = esize; j->ld = ld; j->Q = Q; j->L = L;
        j->out_cost = out_cost; j->s_first = s0;
        j->s_begin = s0 + count * t / nthreads;
        j->s_end = s0 + count * (t + 1) / nthreads;
    }
    int rc = 0;
    if (nthreads == 1) {
        oracle_worker(&jobs[0]);
    } else {
        int started = 0;
        for (int t = 0; t < nthreads; ++t) {
            if (pthread_create(&th[t], NULL, oracle_worker, &jobs[t]) != 0) break;
            ++started;
        }
        for (int t = 0; t < started; ++t) pthread_join(th[t], NULL);
        for (int t = started; t < nthreads; ++t) oracle_worker(&jobs[t]);
    }
    int64_t sum = 0, inf = 0, relax = 0;
    for (int t = 0; t < nthreads; ++t) {
        sum += jobs[t].sum;
        inf += jobs[t].infeasible;
        relax += jobs[t].relax;
        if (jobs[t].status) rc = jobs[t].status;
    }
    out3[0] = sum;
    out3[1] = inf;
    out3[2] = relax;
    free(jobs);
    free(th);
    return rc;
}

/* Optimal routes of one scenario, recovered from the predecessor of Eq. 1
 * (smallest p on ties). route_end receives the tour positions at which routes
 * end, in increasing order; returns the route count, or -1 if infeasible. */
int32_t oracle_split_routes(int32_t n, const int32_t *tour, const int32_t *dist,
                            const void *demand, int esize, int64_t ld, int64_t s,
                            int64_t Q, int32_t L, int32_t *pred, int32_t *route_end,
                            int64_t *cost)
{
    int64_t *f = (int64_t *)malloc(sizeof(int64_t) * ((size_t)n + 1));
    if (!f) return -2;
    int64_t c = oracle_split_scenario(n, tour, dist, demand, esize, ld, s, Q, L, f,
                                      NULL, pred);
    free(f);
    *cost = c;
    if (c < 0) return -1;
    int32_t k = 0;
    int32_t stack_i = n;
    /* walk predecessors back from n, then reverse */
    while (stack_i > 0) {
        route_end[k++] = stack_i;
        stack_i = pred[stack_i];
    }
    for (int32_t a = 0, b = k - 1; a < b; ++a, --b) {
        int32_t t = route_end[a]; route_end[a] = route_end[b]; route_end[b] = t;
    }
    return k;
}
