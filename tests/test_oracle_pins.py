"""Pins for the CPU oracle (Section 3, Eq. 1), independent of the oracle itself.

Each check rests on something other than the oracle's code: values worked by
hand, the paper's Example (Section 2), exhaustive enumeration of all 2^(n-1)
partitions, a second published algorithm (the linear-time Split of Vidal,
"Split algorithm in O(n) for the capacitated vehicle routing problem",
Computers & Operations Research 69, 2016, restated here in our own words), a
closed form on an exact-metric instance, and monotonicity invariants. The
mutation test at the end checks that plausible slips in the oracle (a dropped
term, a transposed operand, an off-by-one bound) break at least one pin.
"""
import collections
import json
import os
import subprocess

import numpy as np
import pytest

import oracle
from synth import instance_from_coords, make_instance, demand_matrix, workload

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")
INT32_MAX = 2**31 - 1


# ---------------------------------------------------------------- references

def brute_force(tour, dist, q_by_id, Q, L):
    """Minimum over every set of cut points of the summed route costs, with
    each route's load <= Q and at most L customers; None if none is feasible."""
    n = len(tour)
    best = None
    for mask in range(1 << (n - 1)):
        cost, ok, start = 0, True, 0
        for k in range(n):
            if k == n - 1 or (mask >> k) & 1:
                route = [int(c) for c in tour[start:k + 1]]
                if len(route) > L or sum(int(q_by_id[c - 1]) for c in route) > Q:
                    ok = False
                    break
                cost += int(dist[0][route[0]]) + int(dist[route[-1]][0])
                cost += sum(int(dist[route[j]][route[j + 1]]) for j in range(len(route) - 1))
                start = k + 1
        if ok and (best is None or cost < best):
            best = cost
    return best


def linear_split(tour, dist, q_by_id, Q, L):
    """Vidal's O(n) Split with a route-length bound: the cost of a route
    sigma_{p+1}..sigma_i separates into a part depending on p and a part
    depending on i through cumulative tour distance, so the best predecessor
    over the sliding feasible window comes from a monotone double-ended queue
    of candidates ordered by that p-part."""
    n = len(tour)
    sig = [0] + [int(c) for c in tour]
    load = [0] * (n + 1)
    cum = [0] * (n + 1)           # cum[k]: tour distance from sigma_1 to sigma_k
    for k in range(1, n + 1):
        load[k] = load[k - 1] + int(q_by_id[sig[k] - 1])
        if k >= 2:
            cum[k] = cum[k - 1] + int(dist[sig[k - 1]][sig[k]])
    INF = None
    pot = [INF] * (n + 1)
    pot[0] = 0

    def start_value(p):           # potential of p plus the route's opening leg
        return pot[p] + int(dist[0][sig[p + 1]]) - cum[p + 1]

    dq = collections.deque([0])
    for i in range(1, n + 1):
        while dq and (load[i] - load[dq[0]] > Q or i - dq[0] > L):
            dq.popleft()
        if not dq:
            return None
        pot[i] = start_value(dq[0]) + cum[i] + int(dist[sig[i]][0])
        if i < n:
            v = start_value(i)
            while dq and start_value(dq[-1]) >= v:
                dq.pop()
            dq.append(i)
    return pot[n]


def costs(inst_tour, dist, D, Q, L, **kw):
    c, total, inf, _ = oracle.split_costs(inst_tour, dist, D, Q, L, **kw)
    return c, total, inf


def as_opt(c):
    return None if c == INT32_MAX else int(c)


# ---------------------------------------------------------------- golden pins

def test_hand_worked_tour(oracle_lib):
    g = json.load(open(os.path.join(GOLDEN, "hand_tour_3.json")))
    coords = [g["depot"]] + g["customers"]
    inst = instance_from_coords(coords, g["tour"], g["Q"])
    d = inst.dist
    assert (d[0, 1], d[0, 2], d[0, 3], d[1, 2], d[2, 3]) == tuple(g["distances"].values())
    names = list(g["scenarios"])
    D = np.array([g["scenarios"][k]["demand_by_customer_id"] for k in names]).T
    for L, key in ((3, "cost_L3"), (2, "cost_L2")):
        c, total, inf = costs(inst.tour, d, D, g["Q"], L)
        assert [as_opt(x) for x in c] == [g["scenarios"][k][key] for k in names]
    c, total, inf = costs(inst.tour, d, D, g["Q"], 3)
    assert (total, inf) == (g["saa_L3_feasible"]["sum"], g["saa_L3_feasible"]["infeasible"])
    assert oracle.saa(c)[2] == g["saa_L3_feasible"]["mean"]
    c, _, _ = costs(inst.tour, d, D, 10**9, 3)
    assert set(int(x) for x in c) == {g["unlimited_capacity_cost"]}


@pytest.mark.parametrize("by_position", [False, True])
def test_paper_example_route_counts(oracle_lib, by_position):
    """Section 2 Example: with every route costing exactly 2 (unit depot legs,
    free travel between customers) the Split cost is twice the minimum number
    of routes; the paper's listed splits are feasible and use that many."""
    g = json.load(open(os.path.join(GOLDEN, "paper_example_q17.json")))
    tour, Q = g["tour"], g["Q"]
    n = len(tour)
    dist = np.zeros((n + 1, n + 1), dtype=np.int32)
    dist[0, 1:] = 1
    dist[1:, 0] = 1
    for sc in g["scenarios"]:
        dem = sc["demands"]
        if by_position:   # the vector lists demands in tour order
            q = [0] * n
            for pos, cust in enumerate(tour):
                q[cust - 1] = dem[pos]
        else:
            q = dem
        for route in sc["routes"]:
            assert sum(q[c - 1] for c in route) <= Q
        assert [c for r in sc["routes"] for c in r] == tour
        c, _, _ = costs(tour, dist, np.array(q).reshape(n, 1), Q, n)
        assert int(c[0]) == 2 * len(sc["routes"])
        cost, routes, _ = oracle.split_routes(tour, dist, q, Q, n)
        assert cost == 2 * len(sc["routes"])
        assert all(sum(q[x - 1] for x in r) <= Q for r in routes)


# ---------------------------------------------------------------- brute force

def random_case(rng, n, asym):
    if asym:
        dist = rng.integers(0, 60, size=(n + 1, n + 1)).astype(np.int32)
    else:
        pts = rng.integers(0, 100, size=(n + 1, 2))
        dist = np.floor(np.sqrt(((pts[:, None] - pts[None]) ** 2).sum(-1)) + 0.5).astype(np.int32)
    tour = rng.permutation(np.arange(1, n + 1)).astype(np.int32)
    Q = int(rng.integers(1, 30))
    L = int(rng.integers(1, n + 1))
    S = 4
    D = rng.integers(0, 12, size=(n, S)).astype(np.int32)
    return tour, dist, D, Q, L


def brute_cases(seed=11, count=60, nmax=9):
    rng = np.random.default_rng(seed)
    out = []
    for t in range(count):
        n = int(rng.integers(1, nmax + 1))
        out.append(random_case(rng, n, asym=(t % 2 == 0)))
    return out


def test_brute_force_small(oracle_lib):
    for tour, dist, D, Q, L in brute_cases():
        c, total, inf = costs(tour, dist, D, Q, L)
        for s in range(D.shape[1]):
            assert as_opt(c[s]) == brute_force(tour, dist, D[:, s], Q, L)


def test_brute_force_n14(oracle_lib):
    rng = np.random.default_rng(5)
    for asym in (False, True):
        tour, dist, D, Q, L = random_case(rng, 14, asym)
        D = rng.integers(0, 6, size=(14, 2)).astype(np.int32)
        Q, L = 17, 9
        c, _, _ = costs(tour, dist, D, Q, L)
        for s in range(2):
            assert as_opt(c[s]) == brute_force(tour, dist, D[:, s], Q, L)


# ------------------------------------------------------- route recovery

def route_cost(tour, dist, a, b):
    """Cost of the route serving tour positions a+1..b (customers tour[a:b])."""
    r = [int(c) for c in tour[a:b]]
    inner = sum(int(dist[r[j]][r[j + 1]]) for j in range(len(r) - 1))
    return int(dist[0][r[0]]) + inner + int(dist[r[-1]][0])


def route_ok(tour, q_by_id, Q, L, a, b):
    return b - a <= L and sum(int(q_by_id[int(c) - 1]) for c in tour[a:b]) <= Q


def brute_prefix_pred(tour, dist, q_by_id, Q, L):
    """Predecessors by enumeration, owing nothing to the oracle: F[i] is the
    cheapest feasible cut of the first i customers, found over all 2^(i-1)
    cut sets of that prefix; pred[i] is the smallest p whose route p+1..i is
    feasible and closes a cheapest cut, F[p] + cost(p+1..i) = F[i] (-1 when
    the prefix has no feasible cut)."""
    n = len(tour)
    F = [0] + [None] * n
    for i in range(1, n + 1):
        for mask in range(1 << (i - 1)):
            cost, start, ok = 0, 0, True
            for k in range(i):
                if k == i - 1 or (mask >> k) & 1:
                    if not route_ok(tour, q_by_id, Q, L, start, k + 1):
                        ok = False
                        break
                    cost += route_cost(tour, dist, start, k + 1)
                    start = k + 1
            if ok and (F[i] is None or cost < F[i]):
                F[i] = cost
    pred = [-1] * (n + 1)
    for i in range(1, n + 1):
        if F[i] is None:
            continue
        for p in range(i):
            if (F[p] is not None and route_ok(tour, q_by_id, Q, L, p, i)
                    and F[p] + route_cost(tour, dist, p, i) == F[i]):
                pred[i] = p
                break
    return F, pred


def routes_from_pred(tour, pred):
    """Walk the predecessors back from position n: the routes in tour order."""
    ends, i = [], len(tour)
    while i > 0:
        ends.append(i)
        i = pred[i]
    routes, start = [], 0
    for e in reversed(ends):
        routes.append([int(c) for c in tour[start:e]])
        start = e
    return routes


def tie_cases():
    """Instances with many equal-cost cuts, where the tie rule decides."""
    out = []
    for n in (4, 6, 8):
        # free travel between customers, unit depot legs: every cut with the
        # same number of routes costs the same
        dist = np.zeros((n + 1, n + 1), dtype=np.int32)
        dist[0, 1:] = 1
        dist[1:, 0] = 1
        tour = np.arange(1, n + 1, dtype=np.int32)
        out.append((tour, dist, np.ones((n, 3), np.int32) * [[1, 2, 3]], 4, n))
        # collinear, symmetric about the depot: customers at -k and +k on a line
        pts = [[0, 0]] + [[(k // 2 + 1) * (1 if k % 2 else -1), 0] for k in range(n)]
        pts = np.array(pts)
        dist = np.abs(pts[:, None, 0] - pts[None, :, 0]).astype(np.int32)
        out.append((np.arange(1, n + 1, dtype=np.int32)[::-1].copy(), dist,
                    np.array([[2, 1, 3]] * n, np.int32), 5, 3))
        # duplicate coordinates: pairs of customers at the same point
        pts = np.array([[50, 50]] + [[10 * (k // 2), 7 * (k // 2)] for k in range(n)])
        dist = np.floor(np.sqrt(((pts[:, None] - pts[None]) ** 2).sum(-1)) + 0.5).astype(np.int32)
        out.append((np.arange(1, n + 1, dtype=np.int32), dist,
                    np.array([[1, 0, 2]] * n, np.int32), 3, n))
    return out


def route_pin_cases():
    return brute_cases() + tie_cases()


def check_routes(tour, dist, D, Q, L, lib=None):
    """Oracle predecessors and routes against enumeration; returns the first
    mismatch as a string, or None."""
    for s in range(D.shape[1]):
        q = D[:, s]
        F, want_pred = brute_prefix_pred(tour, dist, q, Q, L)
        cost, routes, pred = oracle.split_routes(tour, dist, q, Q, L, lib=lib)
        if list(pred[1:]) != want_pred[1:]:
            return f"pred {list(pred[1:])} != {want_pred[1:]}"
        n = len(tour)
        if F[n] is None:
            if cost is not None:
                return "infeasible scenario given a cost"
            continue
        if cost != F[n] or routes != routes_from_pred(tour, want_pred):
            return f"routes {routes} (cost {cost}) != {routes_from_pred(tour, want_pred)} ({F[n]})"
    return None


def test_route_recovery_matches_enumeration(oracle_lib):
    """Whole predecessor array (smallest optimal p, Section 3 reading 7) and
    the routes walked back from it, on the random brute-force cases and on
    tie-heavy instances."""
    for tour, dist, D, Q, L in route_pin_cases():
        assert check_routes(tour, dist, D, Q, L) is None


def test_tie_cases_have_ties(oracle_lib):
    """The tie-heavy instances really have several optimal predecessors at
    some position (else they would not test the tie rule)."""
    seen = 0
    for tour, dist, D, Q, L in tie_cases():
        q = D[:, 0]
        F, pred = brute_prefix_pred(tour, dist, q, Q, L)
        for i in range(1, len(tour) + 1):
            if F[i] is None:
                continue
            opt = [p for p in range(i) if F[p] is not None and route_ok(tour, q, Q, L, p, i)
                   and F[p] + route_cost(tour, dist, p, i) == F[i]]
            seen += len(opt) > 1
    assert seen >= 10


# ------------------------------------------------------- second algorithm

@pytest.mark.parametrize("name,S", [("plain-n50", 1000), ("corr-n200", 1500)])
def test_linear_split_matches(oracle_lib, name, S):
    w = workload(name, S=S)
    inst = w.instances[0]
    D = demand_matrix(inst.mu, inst.region, w.kind, w.scen_seeds[0], S, dtype=w.dtype)
    c, total, inf = costs(inst.tour, inst.dist, D, inst.Q, inst.L, nthreads=4)
    dist = inst.dist.tolist()
    for s in range(S):
        assert as_opt(c[s]) == linear_split(inst.tour, dist, D[:, s], inst.Q, inst.L)


# ------------------------------------------------------------- closed form

def ray_cost(n, cap):
    """Customers k at (3k, 4k), depot at the origin, tour 1..n, unit demands:
    every distance is 5|a-b|, a route ending at customer b costs 10b, and the
    optimum uses R = ceil(n/cap) routes ending as early as the cap allows."""
    R = -(-n // cap)
    return 10 * sum(max(k, n - cap * (R - k)) for k in range(1, R + 1))


@pytest.mark.parametrize("n", [1, 2, 7, 10, 31])
def test_ray_closed_form(oracle_lib, n):
    coords = [[0, 0]] + [[3 * k, 4 * k] for k in range(1, n + 1)]
    for reverse in (False, True):
        tour = list(range(n, 0, -1)) if reverse else list(range(1, n + 1))
        inst = instance_from_coords(coords, tour, Q=1)
        for Q in range(1, n + 2):
            for L in sorted({1, 2, 3, n}):
                D = np.ones((n, 1), dtype=np.int32)
                c, _, _ = costs(inst.tour, inst.dist, D, Q, L)
                assert int(c[0]) == ray_cost(n, min(Q, L))
        c, _, _ = costs(inst.tour, inst.dist, np.zeros((n, 1), np.int32), 0, n)
        assert int(c[0]) == 10 * n     # one route: the tour itself


# -------------------------------------------------------------- invariants

def test_rounding_breaks_triangle(oracle_lib):
    """Rounded Euclidean distances need not satisfy the triangle inequality:
    depot (500,500), customers (499,499), (501,501) give c01 = c02 = 1 and
    c12 = 3, so two routes (cost 4) beat the single route (cost 5)."""
    inst = instance_from_coords([[500, 500], [499, 499], [501, 501]], [1, 2], Q=100)
    assert (inst.dist[0, 1], inst.dist[0, 2], inst.dist[1, 2]) == (1, 1, 3)
    c, _, _ = costs(inst.tour, inst.dist, np.ones((2, 1), np.int32), 100, 2)
    assert int(c[0]) == 4


def test_monotone_invariants(oracle_lib):
    rng = np.random.default_rng(3)
    inst = make_instance(40, 1, 10, seed=9, Q=30, L=12)
    D = rng.integers(0, 9, size=(40, 64)).astype(np.int32)
    base, _, _ = costs(inst.tour, inst.dist, D, 30, 12)
    assert (base != INT32_MAX).all()
    moreQ, _, _ = costs(inst.tour, inst.dist, D, 35, 12)
    moreL, _, _ = costs(inst.tour, inst.dist, D, 30, 20)
    assert (moreQ <= base).all() and (moreL <= base).all()
    D2 = D.copy()
    D2[rng.integers(0, 40, 10), rng.integers(0, 64, 10)] += 3
    more_dem, _, _ = costs(inst.tour, inst.dist, D2, 30, 12)
    assert (more_dem >= base).all()
    # every customer served alone is always feasible when all q <= Q
    trips = int(sum(inst.dist[0, c] + inst.dist[c, 0] for c in inst.tour))
    assert (base <= trips).all()
    solo, _, _ = costs(inst.tour, inst.dist, D, 30, 1)
    assert (solo == trips).all()


def test_infeasible_and_saa(oracle_lib):
    inst = make_instance(20, 1, 10, seed=4, Q=15)
    rng = np.random.default_rng(8)
    D = rng.integers(0, 8, size=(20, 50)).astype(np.int32)
    D[5, 7] = 16                        # one customer above capacity
    D[0, 9] = 15                        # exactly at capacity: still feasible
    c, total, inf = costs(inst.tour, inst.dist, D, 15, 20)
    assert c[7] == INT32_MAX and c[9] != INT32_MAX and inf == 1
    perm = rng.permutation(50)
    c2, total2, inf2 = costs(inst.tour, inst.dist, D[:, perm], 15, 20)
    assert (total2, inf2) == (total, inf) and (c2 == c[perm]).all()
    rep = np.repeat(D[:, 3:4], 33, axis=1)
    c3, total3, inf3 = costs(inst.tour, inst.dist, rep, 15, 20)
    assert total3 == 33 * int(c[3]) and oracle.saa(c3)[2] == float(c[3])


def test_threads_agree(oracle_lib):
    w = workload("corr-n200", S=3000)
    inst = w.instances[0]
    D = demand_matrix(inst.mu, inst.region, w.kind, w.scen_seeds[0], 3000, dtype=w.dtype)
    a = costs(inst.tour, inst.dist, D, inst.Q, inst.L, nthreads=1)
    b = costs(inst.tour, inst.dist, D, inst.Q, inst.L, nthreads=7)
    assert (a[0] == b[0]).all() and a[1:] == b[1:]


# ------------------------------------------------------------ mutation test

MUTANTS = {
    "dropped return leg": ("+ inner + dist[(int64_t)last * N1 + 0]", "+ inner"),
    "transposed first leg": ("dist[0 * N1 + first]", "dist[(int64_t)first * N1 + 0]"),
    "capacity off by one": ("if (load > Q) break;", "if (load >= Q) break;"),
    "route limit off by one": ("if (i - p > L) break;", "if (i - p >= L) break;"),
    "inner edge index": ("inner += dist[(int64_t)tour[p] * N1 + tour[p + 1]]",
                         "inner += dist[(int64_t)tour[p + 1] * N1 + tour[p]]"),
    "inner edge skipped": ("if (p < i - 1) inner", "if (p < i - 2) inner"),
    "missing predecessor cost": ("int64_t cost = f[p] +", "int64_t cost = 0 +"),
}

# Slips in route recovery; caught by the predecessor / route pins. (Each
# keeps every predecessor below its position, so the walk-back ends.)
ROUTE_MUTANTS = {
    "largest p on ties": ("if (cost < best || (cost == best && p < best_p))", "if (cost < best)"),
    "predecessor shifted": ("best_p = p;", "best_p = p > 0 ? p - 1 : p;"),
    "route end off by one": ("route_end[k++] = stack_i;", "route_end[k++] = stack_i - 1;"),
    "walk-back skips a route": ("stack_i = pred[stack_i];",
                                "stack_i = pred[stack_i] > 0 ? pred[pred[stack_i]] : 0;"),
}


@pytest.mark.parametrize("label", list(MUTANTS))
def test_pins_catch_mutants(oracle_lib, tmp_path, label):
    src = open(oracle._SRC).read()
    old, new = MUTANTS[label]
    assert src.count(old) == 1, label
    mpath = tmp_path / "mutant.c"
    mpath.write_text(src.replace(old, new))
    so = tmp_path / "mutant.so"
    subprocess.check_call(["gcc", "-O1", "-std=c11", "-fPIC", "-shared", "-pthread",
                           str(mpath), "-o", str(so)])
    lib = oracle.bind(str(so))
    caught = False
    for tour, dist, D, Q, L in brute_cases(seed=2, count=30, nmax=7):
        c, _, _, _ = oracle.split_costs(tour, dist, D, Q, L, lib=lib)
        for s in range(D.shape[1]):
            if as_opt(c[s]) != brute_force(tour, dist, D[:, s], Q, L):
                caught = True
                break
        if caught:
            break
    assert caught, f"no pin caught the mutant: {label}"


def build_mutant(tmp_path, old, new):
    src = open(oracle._SRC).read()
    assert src.count(old) == 1, old
    mpath = tmp_path / "mutant.c"
    mpath.write_text(src.replace(old, new))
    so = tmp_path / "mutant.so"
    subprocess.check_call(["gcc", "-O1", "-std=c11", "-fPIC", "-shared", "-pthread",
                           str(mpath), "-o", str(so)])
    return oracle.bind(str(so))


@pytest.mark.parametrize("label", list(ROUTE_MUTANTS))
def test_route_pins_catch_mutants(oracle_lib, tmp_path, label):
    lib = build_mutant(tmp_path, *ROUTE_MUTANTS[label])
    assert any(check_routes(*case, lib=lib) is not None for case in route_pin_cases()), \
        f"no route pin caught the mutant: {label}"
