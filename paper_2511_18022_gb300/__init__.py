"""GB300 scenario-batched Split for the CVRP with stochastic demands.

Python face of the C ABI in include/cvrpsd.h: the functions below carry the
same names as the C entry points and only marshal arguments (numpy arrays for
the host inputs, CUDA torch tensors or raw device pointers for device
buffers, the current torch stream by default). Every step of the Split runs
in the library's CUDA kernels; there is no CPU path.
"""
from __future__ import annotations

import ctypes
from dataclasses import dataclass

import numpy as np

from . import _lib
from ._lib import (CvrpsdError, Config, Stats, OK, WARN_INFEASIBLE, I16, I32, MAX_N,
                   KERNEL_AUTO, KERNEL_DEQUE, KERNEL_WARP, KERNEL_SEQPAR, GEN_NORMAL, GEN_CORRELATED,
                   WALK_AUTO, WALK_GLOBAL_TABLE, WALK_PARAM_TABLE)

__all__ = [
    "cvrpsd_create", "cvrpsd_destroy", "cvrpsd_set_config", "cvrpsd_get_config",
    "cvrpsd_last_stats", "cvrpsd_set_profiling", "cvrpsd_debug_fail_alloc", "cvrpsd_check_inputs", "cvrpsd_int_rate", "cvrpsd_set_log", "cvrpsd_split_eval", "cvrpsd_split_eval_host", "cvrpsd_split_eval_noalloc",
    "cvrpsd_batch_create", "cvrpsd_batch_autotune", "cvrpsd_batch_run", "cvrpsd_batch_results", "cvrpsd_batch_destroy",
    "cvrpsd_split_eval_batch", "Batch", "cvrpsd_autotune", "cvrpsd_split_routes", "routes_from_pred",
    "cvrpsd_split_eval_tours", "cvrpsd_neighbors", "cvrpsd_topk", "cvrpsd_gather_tours", "cvrpsd_accept_best", "Surrogate", "cvrpsd_gen_demand", "cvrpsd_version",
    "Splitter", "SplitResult", "CvrpsdError", "I16", "I32", "MAX_N", "KERNEL_AUTO",
    "KERNEL_DEQUE", "KERNEL_WARP", "KERNEL_SEQPAR", "GEN_NORMAL", "GEN_CORRELATED",
    "WALK_AUTO", "WALK_GLOBAL_TABLE", "WALK_PARAM_TABLE",
]

INT32_MAX = 2**31 - 1


def _i32(a) -> np.ndarray:
    return np.ascontiguousarray(np.asarray(a), dtype=np.int32)


def _stream_ptr(stream):
    if stream is None:
        import torch
        return torch.cuda.current_stream().cuda_stream
    if isinstance(stream, int):
        return stream
    return stream.cuda_stream


def _dev(buf):
    """(pointer, dtype code, shape) of a CUDA tensor, or a raw pointer."""
    if buf is None:
        return None, None, None
    if isinstance(buf, int):
        return buf, None, None
    if not buf.is_cuda:
        raise CvrpsdError(_lib.ERR_ARG, "device buffer expected, got a host tensor")
    import torch
    code = {torch.int16: I16, torch.int32: I32}.get(buf.dtype)
    return buf.data_ptr(), code, tuple(buf.shape)


def cvrpsd_version() -> str:
    return _lib.load().cvrpsd_version().decode()


def cvrpsd_create(device: int = 0) -> ctypes.c_void_p:
    lib = _lib.load()
    h = ctypes.c_void_p()
    rc = lib.cvrpsd_create(ctypes.byref(h), int(device))
    if rc != OK:
        raise CvrpsdError(rc, f"cvrpsd_create(device={device}) failed")
    return h


def cvrpsd_destroy(ctx) -> None:
    _lib.check(None, _lib.load().cvrpsd_destroy(ctx))


def cvrpsd_set_config(ctx, kernel=KERNEL_AUTO, threads=0, spt=0, ring=0, variant=0, rounds=0) -> None:
    cfg = Config(kernel, threads, spt, ring, variant, rounds)
    _lib.check(ctx, _lib.load().cvrpsd_set_config(ctx, ctypes.byref(cfg)))


def cvrpsd_get_config(ctx) -> dict:
    cfg = Config()
    _lib.check(ctx, _lib.load().cvrpsd_get_config(ctx, ctypes.byref(cfg)))
    return {f: getattr(cfg, f) for f, _ in Config._fields_}


def cvrpsd_set_profiling(ctx, on: bool) -> None:
    _lib.check(ctx, _lib.load().cvrpsd_set_profiling(ctx, int(bool(on))))


def cvrpsd_debug_fail_alloc(ctx, after: int) -> None:
    """Test hook: make the (after+1)-th next allocation of the context fail."""
    _lib.check(ctx, _lib.load().cvrpsd_debug_fail_alloc(ctx, int(after)))


_log_keep = {}


def cvrpsd_set_log(ctx, fn, max_level: int = 1) -> None:
    """Send the context's messages of level <= max_level to fn(level, text)
    (fn=None: off). The binding keeps the C callback alive with the context."""
    key = ctx.value if isinstance(ctx, ctypes.c_void_p) else int(ctx)
    if fn is None:
        _lib.check(ctx, _lib.load().cvrpsd_set_log(ctx, _lib.LOG_FN(), None, -1))
        _log_keep.pop(key, None)
        return
    cb = _lib.LOG_FN(lambda level, msg, user: fn(int(level), msg.decode(errors="replace")))
    _log_keep[key] = cb
    _lib.check(ctx, _lib.load().cvrpsd_set_log(ctx, cb, None, int(max_level)))


def cvrpsd_check_inputs(ctx, stream=None) -> None:
    """Wait for `stream`; raise CvrpsdError(ERR_DEVICE_STATUS) if a Split on
    the context since the last check found a negative demand (the record is
    cleared either way)."""
    _lib.check(ctx, _lib.load().cvrpsd_check_inputs(ctx, _stream_ptr(stream)))


def cvrpsd_int_rate(device: int = 0, iters: int = 20000, stream=None) -> tuple[float, float]:
    """(32-bit integer min/max operations per second, kernel ms) measured on
    `device`: the integer-ALU peak of the Split's window minimum."""
    ops, ms = ctypes.c_double(0.0), ctypes.c_double(0.0)
    _lib.check(None, _lib.load().cvrpsd_int_rate(int(device), int(iters), ctypes.byref(ops), ctypes.byref(ms),
                                                 _stream_ptr(stream)))
    return ops.value, ms.value


def cvrpsd_last_stats(ctx) -> dict:
    st = Stats()
    _lib.check(ctx, _lib.load().cvrpsd_last_stats(ctx, ctypes.byref(st)))
    return {f: getattr(st, f) for f, _ in Stats._fields_}


@dataclass
class SplitResult:
    status: int
    sum: int | None
    infeasible: int | None
    mean: float | None


def cvrpsd_split_eval(ctx, tour, dist, demand, Q: int, L: int | None = None, *,
                      S: int | None = None, ld: int | None = None, dtype: int | None = None,
                      out_cost=None, host_outputs: bool = True, stream=None) -> SplitResult:
    """Split one tour under every scenario column of `demand` (device [n][ld]).

    `tour` (customer ids 1..n) and `dist` ((n+1)^2, node 0 = depot) are host
    arrays. `out_cost` is an optional device int32 tensor of S entries. With
    host_outputs the call waits for the stream and returns the exact sum,
    the infeasible count and the mean; otherwise it only enqueues the work."""
    tour = _i32(tour)
    dist = _i32(dist)
    n = int(tour.shape[0])
    dptr, dcode, dshape = _dev(demand)
    if dshape is not None:
        if len(dshape) != 2 or dshape[0] != n:
            raise CvrpsdError(_lib.ERR_ARG, f"demand must be [n][ld] with n={n}, got {dshape}")
        if not demand.is_contiguous():
            raise CvrpsdError(_lib.ERR_ARG, "demand must be contiguous")
        ld = dshape[1] if ld is None else ld
        S = ld if S is None else S
        dtype = dcode if dtype is None else dtype
        if dtype is None:
            raise CvrpsdError(_lib.ERR_DTYPE, f"demand must be int16 or int32, got {demand.dtype}")
    if S is None or ld is None or dtype is None:
        raise CvrpsdError(_lib.ERR_ARG, "S, ld and dtype are required with a raw demand pointer")
    optr, _, oshape = _dev(out_cost)
    L = n if L is None else int(L)
    s_sum = ctypes.c_int64(0)
    s_inf = ctypes.c_int64(0)
    s_mean = ctypes.c_double(0.0)
    hs = (ctypes.byref(s_sum), ctypes.byref(s_inf), ctypes.byref(s_mean)) if host_outputs else (None,) * 3
    lib = _lib.load()
    rc = lib.cvrpsd_split_eval(ctx, tour.ctypes.data, n, dist.ctypes.data, dptr, int(dtype),
                               int(S), int(ld), int(Q), L, optr, *hs, _stream_ptr(stream))
    _lib.check(ctx, rc)
    if not host_outputs:
        return SplitResult(rc, None, None, None)
    return SplitResult(rc, s_sum.value, s_inf.value, s_mean.value)


def cvrpsd_split_eval_host(ctx, tour, dist, demand, Q: int, L: int | None = None, *, S: int | None = None,
                           out_cost=None, stream=None) -> SplitResult:
    """Split one tour under the scenario columns of a page-locked HOST tensor
    `demand` [n][ld] (torch pin_memory=True). The kernels read it in place
    across the host link; `out_cost` (optional) is a page-locked host int32
    tensor of S entries. Waits for the stream; returns the exact sum, the
    infeasible count and the mean."""
    import torch
    tour = _i32(tour)
    dist = _i32(dist)
    n = int(tour.shape[0])
    for t, what in ((demand, "demand"), (out_cost, "out_cost")):
        if t is None:
            continue
        if not isinstance(t, torch.Tensor) or t.is_cuda or not t.is_contiguous() or not t.is_pinned():
            raise CvrpsdError(_lib.ERR_ARG, f"{what} must be a contiguous page-locked host tensor")
    if demand.dim() != 2 or demand.shape[0] != n:
        raise CvrpsdError(_lib.ERR_ARG, f"demand must be [n][ld] with n={n}, got {tuple(demand.shape)}")
    dtype = {torch.int16: I16, torch.int32: I32}.get(demand.dtype)
    if dtype is None:
        raise CvrpsdError(_lib.ERR_DTYPE, f"demand must be int16 or int32, got {demand.dtype}")
    ld = int(demand.shape[1])
    S = ld if S is None else int(S)
    if out_cost is not None and (out_cost.dtype != torch.int32 or out_cost.numel() < S):
        raise CvrpsdError(_lib.ERR_ARG, f"out_cost must be int32 with at least {S} entries")
    L = n if L is None else int(L)
    s_sum, s_inf, s_mean = ctypes.c_int64(0), ctypes.c_int64(0), ctypes.c_double(0.0)
    rc = _lib.load().cvrpsd_split_eval_host(ctx, tour.ctypes.data, n, dist.ctypes.data, demand.data_ptr(), dtype,
                                            S, ld, int(Q), L, None if out_cost is None else out_cost.data_ptr(),
                                            ctypes.byref(s_sum), ctypes.byref(s_inf), ctypes.byref(s_mean),
                                            _stream_ptr(stream))
    _lib.check(ctx, rc)
    return SplitResult(rc, s_sum.value, s_inf.value, s_mean.value)


def cvrpsd_split_eval_noalloc(tour, dist, demand, Q: int, L: int | None = None, *,
                              S: int | None = None, ld: int | None = None, dtype: int | None = None,
                              out_cost=None, host_outputs: bool = True, stream=None) -> SplitResult:
    """Same Split as cvrpsd_split_eval on the current device, for callers that
    cannot allocate device memory at call time (their memory is all in their
    own pool, or a cudaMalloc could block or fail mid-loop). Uses the library's
    fixed device scratch: at most 2^20 scenarios, and calls that overlap on the
    GPU must be serialised by the caller."""
    tour = _i32(tour)
    dist = _i32(dist)
    n = int(tour.shape[0])
    dptr, dcode, dshape = _dev(demand)
    if dshape is not None:
        if len(dshape) != 2 or dshape[0] != n:
            raise CvrpsdError(_lib.ERR_ARG, f"demand must be [n][ld] with n={n}, got {dshape}")
        ld = dshape[1] if ld is None else ld
        S = ld if S is None else S
        dtype = dcode if dtype is None else dtype
        if dtype is None:
            raise CvrpsdError(_lib.ERR_DTYPE, f"demand must be int16 or int32, got {demand.dtype}")
    if S is None or ld is None or dtype is None:
        raise CvrpsdError(_lib.ERR_ARG, "S, ld and dtype are required with a raw demand pointer")
    optr, _, _ = _dev(out_cost)
    L = n if L is None else int(L)
    s_sum, s_inf, s_mean = ctypes.c_int64(0), ctypes.c_int64(0), ctypes.c_double(0.0)
    hs = (ctypes.byref(s_sum), ctypes.byref(s_inf), ctypes.byref(s_mean)) if host_outputs else (None,) * 3
    lib = _lib.load()
    rc = lib.cvrpsd_split_eval_noalloc(tour.ctypes.data, n, dist.ctypes.data, dptr, int(dtype), int(S),
                                       int(ld), int(Q), L, optr, *hs, _stream_ptr(stream))
    if rc < 0:
        raise CvrpsdError(rc, f"cvrpsd_split_eval_noalloc: {lib.cvrpsd_strerror(rc).decode()}")
    if not host_outputs:
        return SplitResult(rc, None, None, None)
    return SplitResult(rc, s_sum.value, s_inf.value, s_mean.value)


def cvrpsd_gen_demand(ctx, seed: int, kind: int, mu, region, out, *, S: int | None = None,
                      ld: int | None = None, dtype: int | None = None, stream=None) -> None:
    """Fill the device [n][ld] matrix `out` with seeded scenarios 0..S-1."""
    mu = _i32(mu)
    region = _i32(region) if region is not None else None
    n = int(mu.shape[0])
    optr, ocode, oshape = _dev(out)
    if oshape is not None:
        if len(oshape) != 2 or oshape[0] != n:
            raise CvrpsdError(_lib.ERR_ARG, f"out must be [n][ld] with n={n}, got {oshape}")
        ld = oshape[1] if ld is None else ld
        S = ld if S is None else S
        dtype = ocode if dtype is None else dtype
    rc = _lib.load().cvrpsd_gen_demand(ctx, int(seed) & (2**64 - 1), int(kind), mu.ctypes.data,
                                       None if region is None else region.ctypes.data, n, int(S),
                                       int(ld), int(dtype), optr, _stream_ptr(stream))
    _lib.check(ctx, rc)


def cvrpsd_split_routes(ctx, tour, dist, demand, Q: int, L: int | None = None, *, pred, out_cost=None,
                        S: int | None = None, stream=None) -> SplitResult:
    """cvrpsd_split_eval plus the optimal predecessor of every (position,
    scenario) in `pred`, a CUDA int16 tensor [n][ldp] (smallest p on ties)."""
    tour = _i32(tour)
    dist = _i32(dist)
    n = int(tour.shape[0])
    dptr, dcode, dshape = _dev(demand)
    if dshape is None or len(dshape) != 2 or dshape[0] != n or dcode is None:
        raise CvrpsdError(_lib.ERR_ARG, "demand must be a CUDA int16/int32 tensor [n][ld]")
    import torch
    if pred.dtype != torch.int16 or pred.dim() != 2 or pred.shape[0] != n or not pred.is_contiguous():
        raise CvrpsdError(_lib.ERR_ARG, "pred must be a contiguous CUDA int16 tensor [n][ldp]")
    pptr, _, _ = _dev(pred)
    optr, _, _ = _dev(out_cost)
    ld = dshape[1]
    S = ld if S is None else S
    s_sum, s_inf, s_mean = ctypes.c_int64(0), ctypes.c_int64(0), ctypes.c_double(0.0)
    rc = _lib.load().cvrpsd_split_routes(ctx, tour.ctypes.data, n, dist.ctypes.data, dptr, int(dcode), int(S),
                                         int(ld), int(Q), int(L or n), optr, pptr, int(pred.shape[1]),
                                         ctypes.byref(s_sum), ctypes.byref(s_inf), ctypes.byref(s_mean),
                                         _stream_ptr(stream))
    _lib.check(ctx, rc)
    return SplitResult(rc, s_sum.value, s_inf.value, s_mean.value)


def routes_from_pred(tour, pred_column) -> list[list[int]]:
    """Routes (lists of customer ids) of one scenario from its predecessor
    column pred[:, s] (host array of n entries)."""
    tour = np.asarray(tour)
    ends, i = [], len(tour)
    while i > 0:
        ends.append(i)
        i = int(pred_column[i - 1])
    routes, start = [], 0
    for e in reversed(ends):
        routes.append([int(c) for c in tour[start:e]])
        start = e
    return routes


def cvrpsd_autotune(ctx, tour, dist, demand, Q: int, L: int | None = None, *, S: int | None = None,
                    cache_path: str | None = None, stream=None) -> dict:
    """Time every launch shape on this workload, keep the fastest on the
    context (see include/cvrpsd.h); returns the chosen shape and timings."""
    tour = _i32(tour)
    dist = _i32(dist)
    n = int(tour.shape[0])
    dptr, dcode, dshape = _dev(demand)
    if dshape is None or len(dshape) != 2 or dshape[0] != n or dcode is None:
        raise CvrpsdError(_lib.ERR_ARG, "demand must be a CUDA int16/int32 tensor [n][ld]")
    ld = dshape[1]
    S = ld if S is None else S
    res = _lib.TuneResult()
    rc = _lib.load().cvrpsd_autotune(ctx, tour.ctypes.data, n, dist.ctypes.data, dptr, int(dcode), int(S),
                                     int(ld), int(Q), int(L or n),
                                     None if cache_path is None else str(cache_path).encode(),
                                     ctypes.byref(res), _stream_ptr(stream))
    _lib.check(ctx, rc)
    return {"threads": res.best.threads, "spt": res.best.spt, "ring": res.best.ring,
            "variant": res.best.variant, "rounds": res.best.rounds,
            "ms": res.best_ms, "dtype": res.best_dtype, "shapes_timed": res.shapes_timed}


def _dptr(t, dtype=None, what="buffer"):
    import torch
    if not isinstance(t, torch.Tensor) or not t.is_cuda or not t.is_contiguous():
        raise CvrpsdError(_lib.ERR_ARG, f"{what} must be a contiguous CUDA tensor")
    if dtype is not None and t.dtype != dtype:
        raise CvrpsdError(_lib.ERR_ARG, f"{what} must be {dtype}, got {t.dtype}")
    return t.data_ptr()


def cvrpsd_split_eval_tours(ctx, tours, dist, demand, Q: int, L: int | None = None, *, S: int | None = None,
                            mean=None, sums=None, infeasible=None, stream=None):
    """SAA evaluation of many device tours [T][n] of one instance (async)."""
    import torch
    T, n = int(tours.shape[0]), int(tours.shape[1])
    dptr, dcode, dshape = _dev(demand)
    if dshape is None or dshape[0] != n or dcode is None:
        raise CvrpsdError(_lib.ERR_ARG, "demand must be a CUDA int16/int32 tensor [n][ld]")
    ld = dshape[1]
    S = ld if S is None else S
    dist = _i32(dist)
    rc = _lib.load().cvrpsd_split_eval_tours(
        ctx, _dptr(tours, torch.int32, "tours"), T, n, dist.ctypes.data, dptr, int(dcode), int(S), int(ld),
        int(Q), int(L or n), None if mean is None else _dptr(mean, torch.float64, "mean"),
        None if sums is None else _dptr(sums, torch.int64, "sums"),
        None if infeasible is None else _dptr(infeasible, torch.int64, "infeasible"), _stream_ptr(stream))
    _lib.check(ctx, rc)


def cvrpsd_neighbors(ctx, base, moves, out, stream=None):
    import torch
    _lib.check(ctx, _lib.load().cvrpsd_neighbors(ctx, _dptr(base, torch.int32, "base"), int(base.shape[0]),
                                                 _dptr(moves, torch.int32, "moves"), int(moves.shape[0]),
                                                 _dptr(out, torch.int32, "out"), _stream_ptr(stream)))


def cvrpsd_topk(ctx, scores, k: int, out, stream=None):
    import torch
    _lib.check(ctx, _lib.load().cvrpsd_topk(ctx, _dptr(scores, torch.float32, "scores"), int(scores.shape[0]),
                                            int(k), _dptr(out, torch.int32, "idx"), _stream_ptr(stream)))


def cvrpsd_gather_tours(ctx, tours, idx, out, stream=None):
    import torch
    _lib.check(ctx, _lib.load().cvrpsd_gather_tours(ctx, _dptr(tours, torch.int32, "tours"), int(tours.shape[0]),
                                                    int(tours.shape[1]),
                                                    _dptr(idx, torch.int32, "idx"), int(idx.shape[0]),
                                                    _dptr(out, torch.int32, "out"), _stream_ptr(stream)))


def cvrpsd_accept_best(ctx, tours, cost, cur, cur_cost, trace=None, stream=None):
    """The search's improvement step on the device: the cheapest of the tours
    [T][n] (costs float64 [T]) replaces `cur` [n] if strictly cheaper than
    `cur_cost` (float64, one element); `trace` (optional float64, one element)
    gets the current cost after the step. Asynchronous."""
    import torch
    T, n = int(tours.shape[0]), int(tours.shape[1])
    if cost.numel() < T or cur.numel() != n or cur_cost.numel() < 1 or (trace is not None and trace.numel() < 1):
        raise CvrpsdError(_lib.ERR_ARG, f"cost needs {T} entries, cur {n}, cur_cost and trace one")
    _lib.check(ctx, _lib.load().cvrpsd_accept_best(ctx, _dptr(tours, torch.int32, "tours"), T, n,
                                                   _dptr(cost, torch.float64, "cost"), _dptr(cur, torch.int32, "cur"),
                                                   _dptr(cur_cost, torch.float64, "cur_cost"),
                                                   None if trace is None else _dptr(trace, torch.float64, "trace"),
                                                   _stream_ptr(stream)))


class Surrogate:
    """The tour-cost surrogate (cvrpsd_surrogate_*): hand-written BF16
    training and inference kernels with FP32 accumulation."""

    def __init__(self, ctx, cust, dist, Q: float, seed: int = 0):
        cust = np.ascontiguousarray(cust, dtype=np.float32)
        dist = _i32(dist)
        h = ctypes.c_void_p()
        _lib.check(ctx, _lib.load().cvrpsd_surrogate_create(ctx, int(cust.shape[0]), cust.ctypes.data,
                                                            dist.ctypes.data, float(Q), int(seed) & (2**64 - 1),
                                                            ctypes.byref(h)))
        self.ctx, self.handle, self.n = ctx, h, int(cust.shape[0])

    def set_scale(self, len_mean: float, len_sd: float):
        _lib.check(self.ctx, _lib.load().cvrpsd_surrogate_set_scale(self.handle, float(len_mean), float(len_sd)))

    def predict(self, tours, out, stream=None):
        import torch
        _lib.check(self.ctx, _lib.load().cvrpsd_surrogate_predict(
            self.handle, _dptr(tours, torch.int32, "tours"), int(tours.shape[0]),
            _dptr(out, torch.float32, "pred"), _stream_ptr(stream)))

    def train_step(self, tours, target, lr: float, loss=None, stream=None):
        import torch
        _lib.check(self.ctx, _lib.load().cvrpsd_surrogate_train_step(
            self.handle, _dptr(tours, torch.int32, "tours"), int(tours.shape[0]),
            _dptr(target, torch.float32, "target"), float(lr),
            None if loss is None else _dptr(loss, torch.float32, "loss"), _stream_ptr(stream)))

    def gradients(self, tours, target):
        import torch
        g = np.zeros(_lib.SURROGATE_PARAMS, np.float32)
        loss = ctypes.c_float(0.0)
        _lib.check(self.ctx, _lib.load().cvrpsd_surrogate_gradients(
            self.handle, _dptr(tours, torch.int32, "tours"), int(tours.shape[0]),
            _dptr(target, torch.float32, "target"), g.ctypes.data, ctypes.byref(loss)))
        return g, loss.value

    def params(self, new=None) -> np.ndarray:
        p = np.zeros(_lib.SURROGATE_PARAMS, np.float32)
        cnt = ctypes.c_int64(0)
        src = None if new is None else np.ascontiguousarray(new, dtype=np.float32)
        _lib.check(self.ctx, _lib.load().cvrpsd_surrogate_params(
            self.handle, p.ctypes.data, None if src is None else src.ctypes.data, ctypes.byref(cnt)))
        return p

    def state(self) -> bytes:
        """Checkpoint of the trainer (parameters, Adam moments and step, input
        scale) as bytes; see cvrpsd_surrogate_state."""
        lib = _lib.load()
        size = ctypes.c_int64(0)
        _lib.check(self.ctx, lib.cvrpsd_surrogate_state(self.handle, None, None, ctypes.byref(size)))
        buf = ctypes.create_string_buffer(size.value)
        _lib.check(self.ctx, lib.cvrpsd_surrogate_state(self.handle, buf, None, ctypes.byref(size)))
        return buf.raw

    def load_state(self, blob: bytes) -> None:
        """Resume from a checkpoint taken by state() on a network of the same n."""
        buf = ctypes.create_string_buffer(bytes(blob), len(blob))
        size = ctypes.c_int64(0)
        lib = _lib.load()
        _lib.check(self.ctx, lib.cvrpsd_surrogate_state(self.handle, None, None, ctypes.byref(size)))
        if len(blob) != size.value:
            raise CvrpsdError(_lib.ERR_ARG, f"checkpoint has {len(blob)} bytes, expected {size.value}")
        _lib.check(self.ctx, lib.cvrpsd_surrogate_state(self.handle, None, buf, ctypes.byref(size)))

    def save(self, path) -> None:
        with open(path, "wb") as f:
            f.write(self.state())

    def load(self, path) -> None:
        with open(path, "rb") as f:
            self.load_state(f.read())

    def close(self):
        if self.handle is not None:
            _lib.load().cvrpsd_surrogate_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def _tour_descs(tours, S):
    """ctypes descriptors for a list of dicts with keys tour, dist, demand
    (CUDA tensor [n][ld]), Q, L (optional), out_cost (optional CUDA int32
    tensor); also returns the host arrays and device tensors to keep alive."""
    arr = (_lib.TourDesc * len(tours))()
    keep, dtype = [], None
    for k, t in enumerate(tours):
        tour = _i32(t["tour"])
        dist = _i32(t["dist"])
        n = int(tour.shape[0])
        dptr, dcode, dshape = _dev(t["demand"])
        if dshape is None or len(dshape) != 2 or dshape[0] != n:
            raise CvrpsdError(_lib.ERR_ARG, f"tour {k}: demand must be a CUDA tensor [n][ld] with n={n}")
        if dtype is None:
            dtype = dcode
        elif dcode != dtype:
            raise CvrpsdError(_lib.ERR_DTYPE, f"tour {k}: all demand matrices must share one type")
        optr, _, _ = _dev(t.get("out_cost"))
        L = int(t.get("L") or n)
        arr[k] = _lib.TourDesc(tour.ctypes.data, n, dist.ctypes.data, dptr, int(dshape[1]), int(t["Q"]),
                               L, optr)
        keep += [tour, dist, t["demand"], t.get("out_cost")]
    if dtype is None:
        raise CvrpsdError(_lib.ERR_DTYPE, "demand must be int16 or int32")
    return arr, keep, dtype


class Batch:
    """A captured batch of tours (see cvrpsd_batch_create). Keeps the device
    tensors of its tours alive while it exists."""

    def __init__(self, ctx, tours, S: int):
        arr, keep, dtype = _tour_descs(tours, S)
        h = ctypes.c_void_p()
        lib = _lib.load()
        _lib.check(ctx, lib.cvrpsd_batch_create(ctx, len(tours), arr, int(S), int(dtype), ctypes.byref(h)))
        self.ctx, self.handle, self.T, self.S = ctx, h, len(tours), int(S)
        self._keep = [t for t in keep if t is not None and not isinstance(t, np.ndarray)]

    def run(self, stream=None):
        _lib.check(self.ctx, _lib.load().cvrpsd_batch_run(self.handle, _stream_ptr(stream)))

    def results(self) -> dict:
        T = self.T
        s = np.zeros(T, np.int64)
        inf = np.zeros(T, np.int64)
        mean = np.zeros(T, np.float64)
        st = np.zeros(T, np.int32)
        rc = _lib.load().cvrpsd_batch_results(self.handle, s.ctypes.data, inf.ctypes.data, mean.ctypes.data,
                                              st.ctypes.data)
        _lib.check(self.ctx, rc)
        return {"status": rc, "sum": s, "infeasible": inf, "mean": mean, "tour_status": st}

    def close(self):
        if self.handle is not None:
            _lib.load().cvrpsd_batch_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def cvrpsd_batch_create(ctx, tours, S: int) -> Batch:
    return Batch(ctx, tours, S)


def cvrpsd_batch_autotune(ctx, tours, S: int, stream=None) -> dict:
    """Time every launch shape of the batch kernel on these tours and keep the
    fastest on the context (see include/cvrpsd.h); returns the chosen shape."""
    arr, keep, dtype = _tour_descs(tours, S)
    res = _lib.TuneResult()
    _lib.check(ctx, _lib.load().cvrpsd_batch_autotune(ctx, len(tours), arr, int(S), int(dtype), ctypes.byref(res),
                                                      _stream_ptr(stream)))
    del keep
    return {"threads": res.best.threads, "spt": res.best.spt, "ring": res.best.ring,
            "variant": res.best.variant, "rounds": res.best.rounds,
            "ms": res.best_ms, "dtype": res.best_dtype, "shapes_timed": res.shapes_timed}


def cvrpsd_batch_run(batch: Batch, stream=None) -> None:
    batch.run(stream)


def cvrpsd_batch_results(batch: Batch) -> dict:
    return batch.results()


def cvrpsd_batch_destroy(batch: Batch) -> None:
    batch.close()


def cvrpsd_split_eval_batch(ctx, tours, S: int, stream=None) -> dict:
    """One-shot batch: per-tour exact sums, infeasible counts, means, status."""
    arr, keep, dtype = _tour_descs(tours, S)
    T = len(tours)
    s = np.zeros(T, np.int64)
    inf = np.zeros(T, np.int64)
    mean = np.zeros(T, np.float64)
    st = np.zeros(T, np.int32)
    rc = _lib.load().cvrpsd_split_eval_batch(ctx, T, arr, int(S), int(dtype), s.ctypes.data, inf.ctypes.data,
                                             mean.ctypes.data, st.ctypes.data, _stream_ptr(stream))
    _lib.check(ctx, rc)
    return {"status": rc, "sum": s, "infeasible": inf, "mean": mean, "tour_status": st}


class Splitter:
    """Owns one library context on one device."""

    def __init__(self, device: int = 0):
        self.device = device
        self.ctx = cvrpsd_create(device)

    def close(self):
        if self.ctx is not None:
            cvrpsd_destroy(self.ctx)
            _log_keep.pop(self.ctx.value, None)
            self.ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def configure(self, **kw):
        cvrpsd_set_config(self.ctx, **kw)

    def stats(self) -> dict:
        return cvrpsd_last_stats(self.ctx)

    def profiling(self, on: bool = True):
        cvrpsd_set_profiling(self.ctx, on)

    def check_inputs(self, stream=None):
        cvrpsd_check_inputs(self.ctx, stream)

    def set_log(self, fn, max_level: int = 1):
        cvrpsd_set_log(self.ctx, fn, max_level)

    def split(self, tour, dist, demand, Q, L=None, **kw) -> SplitResult:
        return cvrpsd_split_eval(self.ctx, tour, dist, demand, Q, L, **kw)

    def split_host(self, tour, dist, demand, Q, L=None, **kw) -> SplitResult:
        return cvrpsd_split_eval_host(self.ctx, tour, dist, demand, Q, L, **kw)

    def gen_demand(self, seed, kind, mu, region, out, **kw):
        cvrpsd_gen_demand(self.ctx, seed, kind, mu, region, out, **kw)

    def split_routes(self, tour, dist, demand, Q, L=None, **kw) -> SplitResult:
        return cvrpsd_split_routes(self.ctx, tour, dist, demand, Q, L, **kw)

    def autotune(self, tour, dist, demand, Q, L=None, **kw) -> dict:
        return cvrpsd_autotune(self.ctx, tour, dist, demand, Q, L, **kw)

    def batch(self, tours, S) -> Batch:
        return Batch(self.ctx, tours, S)

    def batch_autotune(self, tours, S, stream=None) -> dict:
        return cvrpsd_batch_autotune(self.ctx, tours, S, stream)

    def split_batch(self, tours, S, stream=None) -> dict:
        return cvrpsd_split_eval_batch(self.ctx, tours, S, stream)
