"""CPU oracle for the scenario-batched CVRPSD Split (Section 3, Eq. 1).

TEST INFRASTRUCTURE ONLY: the tests, the smoke check and the benchmark's CPU
baseline may use it; the product library never imports it and shares no code
with it. The arithmetic lives in split_oracle.c (plain C, int64, POSIX
threads over scenarios); this file compiles it with gcc and calls it through
ctypes.
"""
from __future__ import annotations

import ctypes
import os
import platform
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "split_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
INT32_MAX = 2**31 - 1

_lib = None


def lib_path() -> str:
    return os.path.join(_BUILD, f"liboracle_{platform.machine()}.so")


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (-O2, no architecture-specific flags)."""
    out = lib_path()
    if force or not os.path.exists(out) or os.path.getmtime(out) < os.path.getmtime(_SRC):
        os.makedirs(_BUILD, exist_ok=True)
        tmp = out + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-std=c11", "-fPIC", "-shared",
                               "-pthread", _SRC, "-o", tmp])
        os.replace(tmp, out)
    return out


def bind(path: str):
    """Load an oracle shared library (the built one, or a test's variant)."""
    lib = ctypes.CDLL(path)
    P = ctypes.c_void_p
    lib.oracle_split_many.restype = ctypes.c_int
    lib.oracle_split_many.argtypes = [
        ctypes.c_int32, P, P, P, ctypes.c_int, ctypes.c_int64, ctypes.c_int64,
        ctypes.c_int64, ctypes.c_int64, ctypes.c_int32, P, P, ctypes.c_int]
    lib.oracle_split_routes.restype = ctypes.c_int32
    lib.oracle_split_routes.argtypes = [
        ctypes.c_int32, P, P, P, ctypes.c_int, ctypes.c_int64, ctypes.c_int64,
        ctypes.c_int64, ctypes.c_int32, P, P, P]
    return lib


def _load():
    global _lib
    if _lib is None:
        _lib = bind(build())
    return _lib


def _ptr(a: np.ndarray):
    return ctypes.c_void_p(a.ctypes.data)


def split_costs(tour, dist, demand, Q: int, L: int | None = None,
                nthreads: int = 1, lib=None):
    """Per-scenario Split costs for every column of `demand` ([n][S], int16 or
    int32, row = customer id - 1). Returns (costs int32[S] with INT32_MAX for
    infeasible scenarios, sum of feasible costs, infeasible count,
    number of feasible (p, i) pairs examined)."""
    tour = np.ascontiguousarray(tour, dtype=np.int32)
    dist = np.ascontiguousarray(dist, dtype=np.int32)
    demand = np.asarray(demand)
    if demand.dtype not in (np.int16, np.int32):
        demand = demand.astype(np.int32)
    demand = np.ascontiguousarray(demand)
    n = tour.shape[0]
    if demand.ndim == 1:
        demand = demand.reshape(n, 1)
    S = demand.shape[1]
    L = n if L is None else int(L)
    out = np.empty(S, dtype=np.int32)
    out3 = np.zeros(3, dtype=np.int64)
    rc = (lib or _load()).oracle_split_many(n, _ptr(tour), _ptr(dist), _ptr(demand),
                                   demand.dtype.itemsize, S, 0, S, int(Q), L,
                                   _ptr(out), _ptr(out3), int(nthreads))
    if rc != 0:
        raise RuntimeError(f"oracle_split_many failed ({rc})")
    return out, int(out3[0]), int(out3[1]), int(out3[2])


def split_routes(tour, dist, demand_col, Q: int, L: int | None = None, lib=None):
    """Optimal split of one scenario: (cost or None, list of routes as lists of
    customer ids, predecessor array of length n+1: pred[i] is the smallest p
    attaining f(i), -1 where no feasible split of the first i customers
    exists)."""
    tour = np.ascontiguousarray(tour, dtype=np.int32)
    dist = np.ascontiguousarray(dist, dtype=np.int32)
    col = np.ascontiguousarray(np.asarray(demand_col).reshape(-1), dtype=np.int32)
    n = tour.shape[0]
    L = n if L is None else int(L)
    pred = np.full(n + 1, -1, dtype=np.int32)
    ends = np.zeros(max(n, 1), dtype=np.int32)
    cost = np.zeros(1, dtype=np.int64)
    k = (lib or _load()).oracle_split_routes(n, _ptr(tour), _ptr(dist), _ptr(col), 4, 1, 0,
                                    int(Q), L, _ptr(pred), _ptr(ends), _ptr(cost))
    if k == -2:
        raise MemoryError("oracle_split_routes")
    if k < 0:
        return None, [], pred
    routes, start = [], 0
    for e in ends[:k]:
        routes.append([int(c) for c in tour[start:e]])
        start = int(e)
    return int(cost[0]), routes, pred


def saa(costs) -> tuple[int, int, float]:
    """Sample-average over feasible scenarios (Appendix A estimator):
    (exact integer sum, infeasible count, mean)."""
    c = np.asarray(costs, dtype=np.int64)
    feas = c != INT32_MAX
    total = int(c[feas].sum())
    k = int(feas.sum())
    return total, int((~feas).sum()), (total / k if k else float("nan"))
