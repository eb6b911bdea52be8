"""The host scenario recipe (scenarios.demand_columns) over many columns at
once, spread over worker processes.

A full-size matrix (n = 1000 customers x 2^20 scenarios, 2.1 GB of int16)
takes minutes on one core; the workers fill disjoint column chunks of one
shared-memory buffer, so nothing is pickled. The pool is started with
`spawn`, which is safe after CUDA has been initialised in the parent. The
values are exactly those of demand_matrix (same recipe, same counters).
"""
from __future__ import annotations

import multiprocessing as mp
import os
from concurrent.futures import ProcessPoolExecutor
from multiprocessing import shared_memory

import numpy as np

from . import _cphilox
from .scenarios import demand_columns


def _fill(args):
    name, shape, dtype, mu, region, kind, seed, s0, a, b = args
    shm = shared_memory.SharedMemory(name=name)
    try:
        out = np.ndarray(shape, dtype=dtype, buffer=shm.buf)
        out[:, a:b] = demand_columns(mu, region, kind, seed, np.arange(s0 + a, s0 + b, dtype=np.int64), dtype)
        del out
    finally:
        shm.close()
    return b - a


def demand_matrix_parallel(mu, region, kind: int, seed: int, S: int, s0: int = 0, dtype=np.int16,
                           workers: int | None = None, chunk: int = 1 << 14, out: np.ndarray | None = None):
    """Scenarios s0 .. s0+S-1 as a [n][S] matrix, written into `out` if
    given (any C-contiguous [n][S] array of `dtype`, e.g. a pinned tensor's
    numpy view), generated by `workers` processes in chunks of `chunk`
    columns."""
    dtype = np.dtype(dtype)
    mu = np.asarray(mu, dtype=np.int64)
    region = np.asarray(region, dtype=np.int64)
    n = mu.shape[0]
    if out is None:
        out = np.empty((n, S), dtype=dtype)
    if out.shape != (n, S) or out.dtype != dtype or not out.flags.c_contiguous:
        raise ValueError("out must be a C-contiguous [n][S] array of the requested dtype")
    if S == 0:
        return out
    workers = max(1, min(workers or (os.cpu_count() or 1), (S + chunk - 1) // chunk))
    if workers == 1:
        for a in range(0, S, chunk):
            b = min(S, a + chunk)
            out[:, a:b] = demand_columns(mu, region, kind, seed, np.arange(s0 + a, s0 + b, dtype=np.int64), dtype)
        return out
    _cphilox.build()     # once, before the workers load it
    shm = shared_memory.SharedMemory(create=True, size=out.nbytes)
    try:
        jobs = [(shm.name, (n, S), dtype, mu, region, kind, seed, s0, a, min(S, a + chunk))
                for a in range(0, S, chunk)]
        with ProcessPoolExecutor(max_workers=workers, mp_context=mp.get_context("spawn")) as ex:
            done = sum(ex.map(_fill, jobs))
        assert done == S
        out[...] = np.ndarray((n, S), dtype=dtype, buffer=shm.buf)
    finally:
        shm.close()
        shm.unlink()
    return out
