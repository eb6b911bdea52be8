"""Invariants the deque kernels rely on, checked on the CPU (Section 3, Eq. 1-3).

The scenario-parallel walks keep, per scenario, a monotone deque of
candidate predecessors p with values g(p) = f(p) + A[p] (the separable
segment cost); position i reads the window minimum and adds C_i. The GPU
kernels skip or batch work on the strength of four facts about that walk,
which this file checks on a plain Python deque walk over random tours
(including tours with C_i <= 0, from duplicate points and points on a line
through the depot), random and all-zero demands and route-length caps:

1. No back pops at i when C_{i-1} > 0 and C_i > C_{i-1} (the skip bits).
2. With C_i > 0 the back walk never empties the deque (only positions with
   C_i <= 0 need the emptying walk).
3. Span rule, route length: if every front at the start of a span of 8
   positions satisfies p + L >= i0 + 7, no front leaves by the route-length
   limit inside the span.
4. Span rule, ring: if the deque holds at most R - 8 entries at the start of
   a span, it never holds more than R - 1 before a push inside the span (a
   ring of R slots cannot overflow).

The walk's result is also compared with the oracle, so the walk checked here
is the recursion the kernels compute.
"""
import numpy as np
import pytest

import oracle
from synth import instance_from_coords, make_instance

SPAN = 8
R = 16


def tour_costs(inst):
    """C_i (i = 1..n, index i - 1) and g0 as the kernels' tables define them."""
    t = [0] + [int(c) for c in inst.tour]
    d = inst.dist
    n = inst.n
    C = []
    for i in range(1, n):
        C.append(int(d[t[i], 0] + d[0, t[i + 1]] - d[t[i], t[i + 1]]))
    Dn = sum(int(d[t[k], t[k + 1]]) for k in range(1, n))
    C.append(Dn + int(d[t[n], 0]))
    return C, int(d[0, t[1]])


def walk(inst, q, L, events):
    """f(n) of one scenario by the monotone deque, recording what the
    invariants need; None if infeasible (some demand above Q)."""
    n, Q = inst.n, inst.Q
    if max(q) > Q:
        return None
    C, g0 = tour_costs(inst)
    P = [0]
    for i in range(1, n + 1):
        P.append(P[-1] + int(q[inst.tour[i - 1] - 1]))
    dq = [(0, g0)]                      # (p, g), front first, g increasing
    for i in range(1, n + 1):
        if (i - 1) % SPAN == 0:          # span start i0 = i
            events["span"].append((i, min(p for p, _ in dq), len(dq)))
        length_pops = 0
        while dq and (P[i] - P[dq[0][0]] > Q or i - dq[0][0] > L):
            if i - dq[0][0] > L and P[i] - P[dq[0][0]] <= Q:
                length_pops += 1
            dq.pop(0)
        assert dq, "a demand above Q would empty the deque"
        events["length_pop"].append((i, length_pops))
        gi = C[i - 1] + dq[0][1]
        if i == n:
            return gi
        back = 0
        while dq and dq[-1][1] >= gi:
            dq.pop()
            back += 1
        events["back"].append((i, back, not dq))
        events["size_before_push"].append((i, len(dq)))
        dq.append((i, gi))
    raise AssertionError("unreachable")


def line_instance(n, seed):
    """Customers on a line through the depot, on both sides, some repeated:
    many C_i = 0."""
    rng = np.random.default_rng(seed)
    xs = rng.integers(-40, 41, size=n) * 5
    coords = [[0, 0]] + [[int(x), 0] for x in xs]
    order = list(rng.permutation(np.arange(1, n + 1)))
    return instance_from_coords(coords, order, Q=int(rng.integers(20, 60)))


def cases():
    out = []
    for seed in range(12):
        inst = make_instance(int(40 + 7 * seed), 1, 10, seed=100 + seed, Q=35)
        out.append((f"random{seed}", inst))
    for seed in range(6):
        out.append((f"line{seed}", line_instance(45 + 5 * seed, 200 + seed)))
    dup = make_instance(50, 1, 10, seed=9, Q=30)
    coords = np.array(dup.coords)
    coords[10:20] = coords[10]              # duplicate points: zero legs
    out.append(("dup", instance_from_coords(coords.tolist(), list(dup.tour), Q=30)))
    return out


@pytest.mark.parametrize("name,inst", cases(), ids=[c[0] for c in cases()])
def test_walk_invariants(name, inst):
    rng = np.random.default_rng(len(name) * 7919 + inst.n)
    n = inst.n
    C, _ = tour_costs(inst)
    S = 40
    D = rng.integers(0, max(2, inst.Q // 4), size=(n, S)).astype(np.int32)
    D[:, 0] = 0                                     # whole-tour windows
    D[:, 1] = (np.arange(n) % 3 == 0)               # long windows
    saw = {"noback": 0, "general": 0, "span_l": 0, "span_r": 0}
    for L in (n, 9, 3):
        want, _, _, _ = oracle.split_costs(inst.tour, inst.dist, D, inst.Q, L)
        for s in range(S):
            q = D[:, s]
            ev = {"span": [], "length_pop": [], "back": [], "size_before_push": []}
            f = walk(inst, q, L, ev)
            assert f == want[s], (name, L, s)
            pops = dict((i, b) for i, b, _ in ev["back"])
            emptied = dict((i, e) for i, _, e in ev["back"])
            for i in range(2, n):                   # 1. the skip bits
                if C[i - 2] > 0 and C[i - 1] > C[i - 2]:
                    saw["noback"] += 1
                    assert pops[i] == 0, (name, L, s, i)
            for i in range(1, n):                   # 2. C_i > 0: the deque never empties
                if C[i - 1] > 0:
                    assert not emptied[i], (name, L, s, i)
                else:
                    saw["general"] += 1
            lp = dict(ev["length_pop"])
            size = dict(ev["size_before_push"])
            for i0, oldest, held in ev["span"]:
                span = range(i0, min(i0 + SPAN, n + 1))
                if oldest + L >= i0 + SPAN - 1:     # 3. no route-length pops in the span
                    saw["span_l"] += 1
                    assert all(lp[i] == 0 for i in span), (name, L, s, i0)
                if held <= R - SPAN:                # 4. the ring cannot fill in the span
                    saw["span_r"] += 1
                    assert all(size[i] <= R - 1 for i in span if i in size), (name, L, s, i0)
    assert saw["noback"] > 0 and saw["span_l"] > 0 and saw["span_r"] > 0
    if name.startswith("line"):
        assert saw["general"] > 0


def test_invariants_catch_a_violation():
    """The checks above are not vacuous: a walk that ignores the route-length
    limit breaks the comparison with the oracle on a capped case."""
    inst = make_instance(30, 1, 10, seed=4, Q=200)
    q = np.ones(inst.n, dtype=np.int32)
    want, _, _, _ = oracle.split_costs(inst.tour, inst.dist, q[:, None], inst.Q, 3)
    ev = {"span": [], "length_pop": [], "back": [], "size_before_push": []}
    assert walk(inst, q, 3, ev) == want[0]
    assert walk(inst, q, inst.n, dict((k, []) for k in ev)) != want[0]
