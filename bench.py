#!/usr/bin/env python
"""Benchmark of the scenario-batched Split (one JSON line on stdout).

Workload: million-n1000 -- one giant tour of n = 1000 customers, S = 2^20
correlated demand scenarios (int16, [n][S]), Q = 200, at most 60 customers per
route. A step is one cvrpsd_split_eval call through the C ABI: tour table,
Split kernel(s), exact int64 sums, read-back of sum / infeasible count / mean.
The scenario matrix is generated once on the device before timing (the
paper's fixed scenario set); at 2.1 GB it exceeds the 129 MB L2, so no flush
is needed between steps.

value    = scenario x customer cells per second over all ranks (each rank
           splits its own 2^20 scenarios: weak scaling, no collective on the
           data path).
e2e      = the same metric through the same call with the scenario matrix in
           pinned HOST memory: each step copies it to the device, splits, and
           reads back the per-scenario costs and the sums.
roofline = the Split kernel's algorithmic HBM bytes (2 B per demand read +
           4 B per cost written + the 8 B/position tour table) / its mean
           CUDA-event duration, against the measured copy bandwidth.
--impl reference times the CPU oracle (test infrastructure) on host cores.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "Split scenario·customer relaxations/s at n=1000,S=2^20 (bit-exact); % roofline"
UNIT = "cells/s"
KERNEL_FILES = ["paper_2511_18022_gb300/csrc/split_deque.cuh",
                "paper_2511_18022_gb300/csrc/split_deque.cu",
                "paper_2511_18022_gb300/csrc/split_deque2.cuh",
                "paper_2511_18022_gb300/csrc/split_deque2.cu",
                "paper_2511_18022_gb300/csrc/deque2.h",
                "paper_2511_18022_gb300/csrc/kernels.h"]
TRAFFIC_FILE = os.path.join(ROOT, "profiles", "split_deque_million-n1000.traffic.json")
BATCH_KERNEL_FILES = ["paper_2511_18022_gb300/csrc/split_batch.cu",
                      "paper_2511_18022_gb300/csrc/split_batch2.cu",
                      "paper_2511_18022_gb300/csrc/split_deque.cuh",
                      "paper_2511_18022_gb300/csrc/split_deque2.cuh",
                      "paper_2511_18022_gb300/csrc/deque2.h",
                      "paper_2511_18022_gb300/csrc/kernels.h"]
BATCH_TRAFFIC_FILE = os.path.join(ROOT, "profiles", "split_batch_batched-512.traffic.json")


def kernel_hash(files=None) -> str:
    """Hash of a kernel's sources with // comments and blank lines removed: a
    comment edit does not invalidate the recorded counters."""
    h = hashlib.sha256()
    for f in files or KERNEL_FILES:
        for line in open(os.path.join(ROOT, f), encoding="utf-8"):
            code = line.split("//", 1)[0].rstrip()
            if code:
                h.update(code.encode() + b"\n")
    return h.hexdigest()[:16]


def peaks() -> tuple[float, str]:
    try:
        p = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
        return float(p["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


def host_cores() -> int:
    try:
        return len(os.sched_getaffinity(0))
    except Exception:
        return os.cpu_count() or 1


class ClockSampler:
    """nvidia-smi clocks / throttle reasons sampled in the background."""
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.f = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)
        self.proc = None
        self.t0 = self.t1 = None

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), f"--query-gpu=timestamp,{self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "100"],
                stdout=self.f, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None
        time.sleep(0.3)

    def mark(self, begin: bool):
        if begin:
            self.t0 = time.time()
        else:
            self.t1 = time.time()

    def stop(self) -> dict:
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        time.sleep(0.25)
        self.proc.terminate()
        self.proc.wait()
        self.f.seek(0)
        rows = []
        for line in self.f.read().splitlines():
            parts = [x.strip() for x in line.split(",")]
            if len(parts) < 10:
                continue
            try:
                ts = time.mktime(time.strptime(parts[0].split(".")[0], "%Y/%m/%d %H:%M:%S"))
                rows.append((ts, parts))
            except Exception:
                continue
        os.unlink(self.f.name)
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        inside = [r for ts, r in rows if self.t0 - 1 <= ts <= self.t1 + 1] or [r for _, r in rows]
        sm = [float(r[2]) for r in inside if r[2].replace(".", "").isdigit()]
        smax = [float(r[3]) for r in inside if r[3].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[k] for r in inside for k in range(4) if r[6 + k] == "Active"})
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(smax) if smax else None, "reasons": reasons,
                "samples": len(inside)}


def dist_setup():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        import torch.distributed as dist
        import torch
        # CPU tensors (timing barrier, max over ranks, parity counts) over
        # gloo; the per-step SAA all-reduce of CUDA tensors over NCCL
        backend = "cpu:gloo,cuda:nccl" if torch.cuda.is_available() else "gloo"
        dist.init_process_group(backend)
    return world, rank, local


def barrier(world):
    if world > 1:
        import torch.distributed as dist
        dist.barrier()


def sum_over_ranks(world, xs):
    if world == 1:
        return list(xs)
    import torch
    import torch.distributed as dist
    t = torch.tensor([int(x) for x in xs], dtype=torch.int64)
    dist.all_reduce(t, op=dist.ReduceOp.SUM)
    return [int(v) for v in t.tolist()]


def max_over_ranks(world, x: float) -> float:
    if world == 1:
        return x
    import torch
    import torch.distributed as dist
    t = torch.tensor([x], dtype=torch.float64)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def oracle_sample(w, inst, cols: int, seed_offset: int = 0):
    from synth import demand_columns
    import numpy as np
    return demand_columns(inst.mu, inst.region, w.kind, w.scen_seeds[0] + seed_offset,
                          np.arange(cols), w.dtype)


def time_oracle(inst, D, seconds: float, threads: int):
    """Repeat the oracle over the sample until `seconds` have passed."""
    import oracle
    cells = 0
    t0 = time.perf_counter()
    reps = 0
    while True:
        oracle.split_costs(inst.tour, inst.dist, D, inst.Q, inst.L, nthreads=threads)
        reps += 1
        cells += inst.n * D.shape[1]
        el = time.perf_counter() - t0
        if el >= seconds:
            return cells / el, reps, el


def run_reference(args):
    world, rank, _ = dist_setup()
    if rank != 0:
        return 0
    from synth import workload
    w = workload(args.workload, S=args.S or None)
    inst = w.instances[0]
    cores = host_cores()
    cols = args.ref_cols
    D = oracle_sample(w, inst, cols)
    import oracle
    for _ in range(args.warmup):
        oracle.split_costs(inst.tour, inst.dist, D, inst.Q, inst.L, nthreads=cores)
    times = []
    for _ in range(args.steps):
        t0 = time.perf_counter()
        oracle.split_costs(inst.tour, inst.dist, D, inst.Q, inst.L, nthreads=cores)
        times.append(time.perf_counter() - t0)
    total = sum(times)
    value = inst.n * cols * args.steps / total
    sample = (f"{cols} host-generated scenarios of the {args.workload} instance "
              f"(n={inst.n}) per step, {cores} threads")
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": total / args.steps * 1e3,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "i64",
        "data": "synthetic", "config": workload_config(w, inst),
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle",
                         "sample": sample},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
        "gpu_launches": 0,
    }
    print(json.dumps(line))
    return 0


def workload_config(w, inst) -> dict:
    gb = inst.n * w.S * 2 / 1e9
    return {"workload": w.name, "n": inst.n, "S": w.S, "Q": inst.Q, "L": inst.L,
            "demand": "correlated lognormal, int16 [n][S]",
            "l2": f"inputs larger than L2 ({gb:.2f} GB scenario matrix per step), no flush"}


def run_ours(args):
    import numpy as np
    import torch

    world, rank, local = dist_setup()
    torch.cuda.set_device(local)
    import paper_2511_18022_gb300 as cv
    from paper_2511_18022_gb300 import build, hostmem, shard
    from synth import demand_matrix_parallel, workload

    build.build()
    w = workload(args.workload, S=args.S or None)
    inst = w.instances[0]
    n, S = inst.n, w.S
    cores = host_cores()
    # Weak scaling over one scenario set of world * S columns: rank r splits
    # its contiguous shard, generated on the host from the workload's seed.
    S_total = world * S
    lo, hi = shard.scenario_range(S_total, rank, world)
    assert hi - lo == S
    # The page-locked matrix is allocated by a thread running on the CPUs
    # next to this GPU, so that its pages sit on the GPU's NUMA node (the
    # e2e step streams it across the host link).
    H, placement = hostmem.pinned_near_gpu((n, S), torch.int16, local)
    t0 = time.perf_counter()
    demand_matrix_parallel(inst.mu, inst.region, w.kind, w.scen_seeds[0], S, s0=lo, dtype=np.int16,
                           workers=max(1, cores // world), out=H.numpy())
    gen_s = time.perf_counter() - t0
    D = H.cuda()
    sp = cv.Splitter(local)
    out = torch.empty(S, dtype=torch.int32, device="cuda")
    stream = torch.cuda.current_stream()
    tuned = None
    if args.shape:
        t, s, r, *v = (int(x) for x in args.shape.split(","))
        sp.configure(kernel=cv.KERNEL_DEQUE, threads=t, spt=s, ring=r, variant=v[0] if v else 0)
    elif not args.no_tune:
        tuned = sp.autotune(inst.tour, inst.dist, D, inst.Q, inst.L)

    def split_shard():
        return sp.split(inst.tour, inst.dist, D, inst.Q, inst.L, out_cost=out)

    def step():
        # this rank's shard, then the exact SAA over all ranks (one int64
        # all-reduce of the sum and the infeasible count; none on one GPU)
        return shard.split_and_reduce(split_shard, S_total, world, device="cuda")

    for _ in range(args.warmup):
        g = step()
    # integer min/max rate of this GPU (the ALU roof), measured before the timed region
    int_ops, int_ms = cv.cvrpsd_int_rate(local)
    sp.profiling(True)
    clocks = ClockSampler(local)
    clocks.start()
    barrier(world)
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    kms, launches, overflow = [], 0, 0
    clocks.mark(True)
    e0.record(stream)
    for _ in range(args.steps):
        g = step()
        st = sp.stats()
        kms.append(st["kernel_ms"])
        launches += st["launches"]
        overflow += max(st["overflow"], 0)
    e1.record(stream)
    torch.cuda.synchronize()
    clocks.mark(False)
    barrier(world)
    clk = clocks.stop()
    sp.profiling(False)
    elapsed_ms = max_over_ranks(world, e0.elapsed_time(e1))
    ms_per_step = elapsed_ms / args.steps
    value = world * n * S * args.steps / (elapsed_ms / 1e3)
    kernel_ms = statistics.mean(kms)

    # Parity of the timed run: every scenario's cost against the oracle on
    # the same host matrix (outside the timed region).
    parity = None
    relax_per_cell = None
    if not args.no_parity:
        import oracle
        got = out.cpu().numpy()
        t0 = time.perf_counter()
        want, osum, oinf, orelax = oracle.split_costs(inst.tour, inst.dist, H.numpy(), inst.Q, inst.L,
                                                      nthreads=max(1, cores // world))
        osec = time.perf_counter() - t0
        local_r = split_shard()
        mism = int((got != want).sum())
        tot = sum_over_ranks(world, [mism, S, orelax, int(local_r.sum != osum or local_r.infeasible != oinf)])
        relax_per_cell = tot[2] / (n * tot[1])
        parity = {"scenarios_checked": tot[1], "mismatches": tot[0], "sum_mismatches": tot[3],
                  "global_sum": g[0], "global_infeasible": g[1], "oracle_seconds": round(osec, 2),
                  "oracle_threads": max(1, cores // world),
                  "inputs": "host-generated scenario matrix (synth), the one the timed steps split"}

    roofline = roofline_lines(args, S, n, kernel_ms, st, clk, int_ops, int_ms, relax_per_cell, local)

    # end to end from pinned host memory
    def e2e_step():
        # the C-ABI call on host buffers: the kernels read the page-locked
        # scenario matrix in place across the host link and write the costs
        # back to page-locked host memory; the call returns after the stream
        return sp.split_host(inst.tour, inst.dist, H, inst.Q, inst.L, out_cost=Hout)

    e2e = None
    if args.e2e_steps > 0:
        Hout = torch.empty(S, dtype=torch.int32, pin_memory=True)
        e2e_step()
        barrier(world)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for _ in range(args.e2e_steps):
            e2e_step()
        torch.cuda.synchronize()
        e2e_s = max_over_ranks(world, time.perf_counter() - t0)
        e2e = {"value": world * n * S * args.e2e_steps / e2e_s, "unit": UNIT,
               "h2d_bytes_per_step": n * S * 2 + n * 8, "d2h_bytes_per_step": S * 4 + 32,
               "steps": args.e2e_steps,
               "host_memory": placement | {"pages_by_node": hostmem.pages_by_node(H.data_ptr())}}

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu:
        Dc = oracle_sample(w, inst, args.cpu_cols)
        v, reps, el = time_oracle(inst, Dc, args.cpu_seconds, cores)
        cpu = {"value": v, "unit": UNIT, "cores": cores, "kind": "oracle",
               "sample": f"{args.cpu_cols} host-generated scenarios of this instance, "
                         f"split {reps} times in {el:.1f} s on {cores} threads"}

    if rank == 0:
        metric = METRIC if parity and parity["mismatches"] == 0 and parity["sum_mismatches"] == 0 else \
            METRIC.replace(" (bit-exact)", "")
        line = {
            "metric": metric, "value": value, "unit": UNIT, "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms_per_step,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "i32",
            "data": "synthetic", "config": workload_config(w, inst) | {
                "kernel": (f"deque walk={'parameter-table' if st['variant'] == 2 else 'global-table'} "
                           f"threads={st['threads']} spt={st['spt']} ring={st['ring']}"),
                "shape_source": "fixed" if args.shape else ("autotuned" if tuned else "library default"),
                "parallelism": (f"scenario shards x{world} of one {S_total}-scenario set, one int64 "
                                f"all-reduce (NCCL) of the SAA per step") if world > 1 else "one GPU"},
            "roofline": roofline, "parity": parity, "cpu_baseline": cpu, "e2e": e2e,
            "gpu_launches": launches, "clocks": clk,
            "result": {"sum": g[0], "infeasible": g[1], "mean": g[2],
                       "overflow_scenarios": overflow // max(args.steps, 1)},
            "setup": {"host_generation_s": round(gen_s, 2)},
        }
        print(json.dumps(line))
    sp.close()
    return 0


def roofline_lines(args, S, n, kernel_ms, st, clk, int_ops, int_ms, relax_per_cell, local) -> dict:
    """Both roofs of the Split kernel. HBM: its algorithmic bytes (2 B per
    demand read + 4 B per cost written + 8 B per position of table) over its
    mean CUDA-event time, against the measured copy bandwidth. Integer ALU:
    the literal Eq. 3 work, one min per feasible (p, i) candidate (the
    oracle's exact relaxation count) plus 6 operations per cell (load prefix,
    window start, the two cost terms, the demand unpack), against the
    measured min/max rate. The headline fraction is the binding roof's floor
    time over the kernel time."""
    import torch
    algo_bytes = n * S * 2 + S * 4 + n * 8
    peak, peak_kind = peaks()
    achieved = algo_bytes / (kernel_ms / 1e3) / 1e9
    traffic, winst = None, None
    shape = f"{st['threads']},{st['spt']},{st['ring']},walk{st['variant']}"
    try:
        t = json.load(open(TRAFFIC_FILE))
        if t.get("kernel_hash") == kernel_hash() and S == (1 << 20):
            walk = f"walk{st['variant']}"
            traffic = t["shapes"].get(shape) or t.get("walks", {}).get(walk)
            winst = t.get("inst_executed", {}).get(shape) or t.get("walks_inst_executed", {}).get(walk)
    except Exception:
        pass
    hbm = {"achieved": round(achieved, 1), "peak": peak, "unit": "GB/s", "frac": round(achieved / peak, 4),
           "traffic": traffic, "peak_kind": peak_kind, "algorithmic_bytes": algo_bytes,
           "floor_ms": round(algo_bytes / (peak * 1e9) * 1e3, 4)}
    roof = {"bound": "hbm", "achieved": hbm["achieved"], "peak": peak, "unit": "GB/s", "frac": hbm["frac"],
            "traffic": traffic, "peak_kind": peak_kind,
            "kernel": "split_deque2_kernel" if st["variant"] == 2 else "split_deque_kernel",
            "kernel_ms": round(kernel_ms, 4), "algorithmic_bytes": algo_bytes, "hbm": hbm}
    if relax_per_cell is not None and int_ops:
        ops_per_cell = relax_per_cell + 6.0
        ops = ops_per_cell * n * S
        alu = {"achieved": round(ops / (kernel_ms / 1e3) / 1e12, 3), "peak": round(int_ops / 1e12, 3),
               "unit": "T int32 ops/s", "frac": round(ops / (kernel_ms / 1e3) / int_ops, 4),
               "relaxations_per_cell": round(relax_per_cell, 4), "ops_per_cell": round(ops_per_cell, 4),
               "peak_kind": "measured (cvrpsd_int_rate: 32-bit min/max chains, full grid, "
                            f"{int_ms:.2f} ms)", "floor_ms": round(ops / int_ops * 1e3, 4)}
        roof["alu"] = alu
        if alu["floor_ms"] > hbm["floor_ms"]:
            roof.update({"bound": "alu", "achieved": alu["achieved"], "peak": alu["peak"], "unit": alu["unit"],
                         "frac": alu["frac"], "peak_kind": alu["peak_kind"]})
    # Instruction issue: warp instructions per launch (ncu, same kernel source
    # and shape) against one instruction per clock per scheduler, 4 schedulers
    # per SM, at the SM clock sampled in the timed region.
    if winst and clk.get("sm_mhz"):
        sms = torch.cuda.get_device_properties(local).multi_processor_count
        ipeak = sms * 4 * clk["sm_mhz"] * 1e6
        iach = winst / (kernel_ms / 1e3)
        roof["issue"] = {"achieved": round(iach / 1e9, 1), "peak": round(ipeak / 1e9, 1),
                         "unit": "G warp-instructions/s", "frac": round(iach / ipeak, 4),
                         "warp_instructions_per_launch": winst,
                         "counts_shape": shape if shape in t.get("inst_executed", {})
                         else next(iter(t.get("inst_executed", {})), None),
                         "per_warp_position": round(winst / (S / 32 * n), 2)}
    return roof


def run_batched(args):
    """batched-512: one graph launch evaluates every tour of the workload."""
    import numpy as np
    import torch

    world, rank, local = dist_setup()
    torch.cuda.set_device(local)
    import paper_2511_18022_gb300 as cv
    from paper_2511_18022_gb300 import build
    from synth import workload

    build.build()
    w = workload("batched-512", S=args.S or None, T=args.T or None)
    S = w.S
    sp = cv.Splitter(local)
    tours, mats = [], []
    for t, (inst, sd) in enumerate(zip(w.instances, w.scen_seeds)):
        D = torch.empty((inst.n, S), dtype=torch.int16, device="cuda")
        sp.gen_demand(sd + 7919 * rank, cv.GEN_CORRELATED, inst.mu, inst.region, D)
        mats.append(D)
        tours.append(dict(tour=inst.tour, dist=inst.dist, demand=D, Q=inst.Q, L=inst.L))
    tuned = None
    if args.shape:
        t_, s_, r_ = (int(x) for x in args.shape.split(","))
        sp.configure(kernel=cv.KERNEL_DEQUE, threads=t_, spt=s_, ring=r_)
    elif not args.no_tune:
        tuned = sp.batch_autotune(tours, S)
    b = sp.batch(tours, S)
    stream = torch.cuda.current_stream()
    for _ in range(args.warmup):
        b.run()
        res = b.results()
    clocks = ClockSampler(local)
    clocks.start()
    barrier(world)
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    clocks.mark(True)
    e0.record(stream)
    for _ in range(args.steps):
        b.run()
        res = b.results()
    e1.record(stream)
    torch.cuda.synchronize()
    clocks.mark(False)
    barrier(world)
    clk = clocks.stop()
    ms = max_over_ranks(world, e0.elapsed_time(e1))
    cells = sum(inst.n for inst in w.instances) * S
    value = world * cells * args.steps / (ms / 1e3)
    algo_bytes = cells * 2 + len(w.instances) * S * 4
    peak, peak_kind = peaks()
    step_ms = ms / args.steps
    st = sp.stats()
    traffic = None
    try:   # DRAM bytes of one launch from an ncu record of the same kernel source and shape
        t = json.load(open(BATCH_TRAFFIC_FILE))
        key = f"{st['threads']},{st['spt']},{st['ring']}"
        if t.get("kernel_hash") == kernel_hash(BATCH_KERNEL_FILES) and S == 65536 and len(w.instances) == 512:
            traffic = t["shapes"].get(key)
    except Exception:
        pass
    if rank == 0:
        print(json.dumps({
            "metric": "batched Split scenario·customer cells/s, 512 tours x 65,536 scenarios", "value": value,
            "unit": UNIT, "n_gpus": world, "steps": args.steps, "warmup": args.warmup, "ms_per_step": step_ms,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "i32",
            "data": "synthetic",
            "config": {"workload": w.name, "tours": len(w.instances), "S": S, "cells": cells,
                       "demand": "correlated lognormal, int16, one [n_t][S] matrix per tour",
                       "l2": f"inputs larger than L2 ({cells * 2 / 1e9:.1f} GB per step), no flush",
                       "kernel": f"persistent deque threads={st['threads']} spt={st['spt']} ring={st['ring']}",
                       "shape_source": "fixed" if args.shape else ("autotuned" if tuned else "library default"),
                       "graph": "clear + persistent kernel + set-aside pass + result copy"},
            "roofline": {"bound": "hbm", "achieved": round(algo_bytes / (step_ms / 1e3) / 1e9, 1), "peak": peak,
                         "unit": "GB/s", "frac": round(algo_bytes / (step_ms / 1e3) / 1e9 / peak, 4),
                         "traffic": traffic, "algorithmic_bytes": algo_bytes, "peak_kind": peak_kind,
                         "kernel": "split_batch_kernel (whole graph)"},
            "gpu_launches": 2 * args.steps, "clocks": clk,
            "result": {"set_aside": st["overflow"], "infeasible": int(res["infeasible"].sum()),
                       "mean_of_means": float(np.nanmean(res["mean"]))},
        }))
    b.close()
    sp.close()
    return 0


def run_surrogate(args):
    """surrogate-n200: label tours with the exact GPU Split, train the
    surrogate on them, then compare surrogate-screened local search with
    plain GPU-Split local search from the same start."""
    import numpy as np
    import torch

    world, rank, local = dist_setup()
    torch.cuda.set_device(local)
    import paper_2511_18022_gb300 as cv
    from paper_2511_18022_gb300 import build, search
    from synth import workload

    build.build()
    w = workload("surrogate-n200", S=args.S or None)
    inst, S = w.instances[0], w.S
    sp = cv.Splitter(local)
    D = torch.empty((inst.n, S), dtype=torch.int16, device="cuda")
    sp.gen_demand(w.scen_seeds[0] + rank, cv.GEN_CORRELATED, inst.mu, inst.region, D)
    cust = search.customer_features(inst, D[:, :8192].cpu().numpy())
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    tours, costs = search.training_set(sp.ctx, inst, D, args.train_pairs, seed=11)
    torch.cuda.synchronize()
    t_label = time.perf_counter() - t0
    sur = cv.Surrogate(sp.ctx, cust, inst.dist, Q=float(inst.Q), seed=5)
    t0 = time.perf_counter()
    scale, mae = search.train_surrogate(sur, tours, costs, dist=inst.dist, epochs=args.epochs)
    torch.cuda.synchronize()
    t_train = time.perf_counter() - t0
    M, k = 4096, 64
    trained = sur.state()
    starts = [np.random.default_rng(1234 + r).permutation(np.arange(1, inst.n + 1)).astype(np.int32)
              for r in range(max(1, args.repeats))]
    # warm-up on a copy (first launches, allocations)
    search.LocalSearch(sp.ctx, inst, D, starts[0], M=M, seed=1, exact_all=True).run(max(args.warmup, 1))
    search.LocalSearch(sp.ctx, inst, D, starts[0], surrogate=sur, M=M, k=k, seed=1, scale=scale).run(
        max(args.warmup, 1))
    # Per start: the plain-Split search (every one of the M neighbours split
    # exactly), then the screened search with the same moves, at equal
    # iterations and at equal wall time, each from the trained surrogate.
    # One search is one sample of a noisy trajectory: several starts.
    runs = []
    for r, start in enumerate(starts):
        plain = search.LocalSearch(sp.ctx, inst, D, start, M=M, seed=99 + r, exact_all=True)
        plog = plain.run(args.steps)
        sur.load_state(trained)
        screened = search.LocalSearch(sp.ctx, inst, D, start, surrogate=sur, M=M, k=k, seed=99 + r,
                                      retrain_every=25, scale=scale)
        slog = screened.run(args.steps)
        sur.load_state(trained)
        timed = search.LocalSearch(sp.ctx, inst, D, start, surrogate=sur, M=M, k=k, seed=99 + r,
                                   retrain_every=25, scale=scale)
        tlog = timed.run(1_000_000, seconds=plog.seconds)
        runs.append({"start": r, "plain_cost": plain.cur_cost, "plain_seconds": plog.seconds,
                     "plain_candidates_per_s": plog.candidates_per_s,
                     "screened_cost": screened.cur_cost, "screened_seconds": slog.seconds,
                     "screened_candidates_per_s": slog.candidates_per_s,
                     "gap_equal_iterations": (screened.cur_cost - plain.cur_cost) / plain.cur_cost,
                     "timed_cost": timed.cur_cost, "timed_iterations": timed.iterations,
                     "gap_equal_time": (timed.cur_cost - plain.cur_cost) / plain.cur_cost,
                     "plain_tour": plain.cur.cpu().numpy(), "screened_tour": screened.cur.cpu().numpy()})
    sur.load_state(trained)
    # the old baseline: k random neighbours split exactly
    rand = search.LocalSearch(sp.ctx, inst, D, starts[0], k=k, seed=99)
    rlog = rand.run(args.steps)
    quality = [search.neighbourhood_quality(sp.ctx, inst, D, sur, scale, t, M=M, k=k, seed=17 + j)
               for j, t in enumerate([starts[0], runs[0]["plain_tour"], runs[0]["screened_tour"]])]
    if rank == 0:
        cand_s = float(np.mean([x["screened_candidates_per_s"] for x in runs]))
        plain_cand_s = float(np.mean([x["plain_candidates_per_s"] for x in runs]))
        s_ms = float(np.mean([x["screened_seconds"] for x in runs])) / args.steps * 1e3
        p_ms = float(np.mean([x["plain_seconds"] for x in runs])) / args.steps * 1e3
        print(json.dumps({
            "metric": "surrogate-screened local search: candidate tours/s (exact Split on the top 64 of 4096)",
            "value": cand_s, "unit": "tours/s", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": s_ms, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "bf16 weights, fp32 accumulation; i32 Split",
            "data": "synthetic",
            "config": {"workload": w.name, "n": inst.n, "S": S, "Q": inst.Q, "L": inst.L,
                       "train_pairs": args.train_pairs, "epochs": args.epochs, "screen": M, "exact": k},
            "plain_split_search": {"what": f"all {M} neighbours split exactly per iteration, same moves",
                                   "candidate_tours_per_s": plain_cand_s, "iterations": args.steps,
                                   "ms_per_iteration": p_ms,
                                   "final_saa_cost": [x["plain_cost"] for x in runs]},
            "screened_equal_iterations": {"final_saa_cost": [x["screened_cost"] for x in runs],
                                          "iterations": args.steps, "ms_per_iteration": s_ms,
                                          "gap_vs_plain": [x["gap_equal_iterations"] for x in runs],
                                          "mean_gap_vs_plain": float(np.mean([x["gap_equal_iterations"]
                                                                              for x in runs]))},
            "screened_equal_time": {"final_saa_cost": [x["timed_cost"] for x in runs],
                                    "iterations": [x["timed_iterations"] for x in runs],
                                    "gap_vs_plain": [x["gap_equal_time"] for x in runs],
                                    "mean_gap_vs_plain": float(np.mean([x["gap_equal_time"] for x in runs]))},
            "starts": len(runs),
            "random_k_search": {"what": f"{k} random neighbours split exactly per iteration (first start)",
                                "final_saa_cost": rand.cur_cost,
                                "ms_per_iteration": rlog.seconds / args.steps * 1e3},
            "speedup_candidates": cand_s / plain_cand_s,
            "surrogate": {"holdout_mae": mae, "training_cost_sd": float(costs.std().item()),
                          "label_seconds": t_label, "train_seconds": t_train,
                          "neighbourhoods": quality,
                          "mean_spearman": float(np.mean([q["spearman"] for q in quality])),
                          "mean_recall_at_k": float(np.mean([q["recall_at_k"] for q in quality])),
                          "mean_mae": float(np.mean([q["mae"] for q in quality]))},
            "gpu_launches": None,
        }))
    sur.close()
    sp.close()
    return 0


def run_oos(args):
    """oos-n200: optimise with 1, 100, 1,000 and 10,000 training scenarios and
    evaluate every result on 10^6 held-out scenarios (Section 4.2's study on a
    synthetic instance)."""
    import torch

    world, rank, local = dist_setup()
    torch.cuda.set_device(local)
    import paper_2511_18022_gb300 as cv
    from paper_2511_18022_gb300 import build, search
    from synth import workload

    build.build()
    w = workload("surrogate-n200", S=10_000)
    inst = w.instances[0]
    sp = cv.Splitter(local)
    D_train = torch.empty((inst.n, 10_000), dtype=torch.int16, device="cuda")
    sp.gen_demand(w.scen_seeds[0], cv.GEN_CORRELATED, inst.mu, inst.region, D_train)
    S_test = args.S or 1_000_000
    D_test = torch.empty((inst.n, S_test), dtype=torch.int16, device="cuda")
    sp.gen_demand(w.scen_seeds[0] + 77_777, cv.GEN_CORRELATED, inst.mu, inst.region, D_test)
    t0 = time.perf_counter()
    rows = search.oos_study(sp.ctx, inst, D_train, D_test, [1, 100, 1000, 10_000], iterations=args.steps, seed=3,
                            repeats=args.repeats)
    el = time.perf_counter() - t0
    if rank == 0:
        print(json.dumps({
            "metric": "out-of-sample SAA cost of the searched tour vs training scenario count",
            "value": rows[-1][2], "unit": "cost", "n_gpus": world, "steps": args.steps, "warmup": 0,
            "ms_per_step": el / (4 * args.steps * args.repeats) * 1e3, "higher_is_better": False, "scaling": "weak",
            "vs_baseline": None, "dtype": "i32", "data": "synthetic",
            "config": {"workload": w.name, "n": inst.n, "Q": inst.Q, "L": inst.L, "S_test": S_test,
                       "repeats": args.repeats,
                       "search": "best of 64 random 2-opt/relocate neighbours per iteration, exact GPU Split"},
            "rows": [{"S_train": r[0], "in_sample": r[1], "out_of_sample": r[2]} for r in rows],
            "gpu_launches": None,
        }))
    sp.close()
    return 0


def run_latency(args):
    """latency-n1000: device time of one Split call of the n = 1000 tour for
    few scenarios, per kernel (deque, warp, sequence-parallel): the regime
    where scenario parallelism cannot fill the GPU."""
    import numpy as np
    import torch

    world, rank, local = dist_setup()
    torch.cuda.set_device(local)
    import paper_2511_18022_gb300 as cv
    from paper_2511_18022_gb300 import build
    from synth import workload

    build.build()
    w = workload("million-n1000", S=4096)
    inst = w.instances[0]
    sp = cv.Splitter(local)
    D = torch.empty((inst.n, 4096), dtype=torch.int16, device="cuda")
    sp.gen_demand(w.scen_seeds[0], cv.GEN_CORRELATED, inst.mu, inst.region, D)
    sp.profiling(True)
    kernels = (("deque", cv.KERNEL_DEQUE), ("warp", cv.KERNEL_WARP), ("seqpar", cv.KERNEL_SEQPAR))
    rows, launches = [], 0
    for S in (1, 8, 64, 512, 4096):
        row = {"S": S}
        sums = set()
        for name, k in kernels:
            sp.configure(kernel=k)
            for _ in range(max(args.warmup, 1)):
                sp.split(inst.tour, inst.dist, D, inst.Q, inst.L, S=S)
            ms = []
            for _ in range(args.steps):
                r = sp.split(inst.tour, inst.dist, D, inst.Q, inst.L, S=S)
                st = sp.stats()
                ms.append(st["kernel_ms"] + max(st["fallback_ms"], 0.0))
                launches += st["launches"]
                sums.add(r.sum)
            row[name + "_ms"] = float(np.median(ms))
        assert len(sums) == 1, "kernels disagree"
        rows.append(row)
    sp.configure(kernel=cv.KERNEL_AUTO)
    if rank == 0:
        best = rows[0]["seqpar_ms"]
        print(json.dumps({
            "metric": "device time of one Split call, n=1000, S=1 (sequence-parallel kernel)", "value": best,
            "unit": "ms", "n_gpus": world, "steps": args.steps, "warmup": args.warmup, "ms_per_step": best,
            "higher_is_better": False, "scaling": "weak", "vs_baseline": None, "dtype": "i32",
            "data": "synthetic",
            "config": {"workload": "latency-n1000", "n": inst.n, "Q": inst.Q, "L": inst.L,
                       "timing": "CUDA events of the library around its kernels, median per call"},
            "rows": rows, "gpu_launches": launches,
        }))
    sp.close()
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=1000)
    ap.add_argument("--warmup", type=int, default=10)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="million-n1000")
    ap.add_argument("--T", type=int, default=0, help="tours of the batched workload (default 512)")
    ap.add_argument("--S", type=int, default=0,
                    help="scenarios per rank (default: the workload's own); a smaller S gives a "
                         "scaled-down case of the same generator, e.g. for ncu captures")
    ap.add_argument("--shape", default="", help="threads,spt,ring[,walk] of the deque kernel (walk 1: global "
                                                "table, 2: parameter table, default: automatic)")
    ap.add_argument("--e2e-steps", type=int, default=5)
    ap.add_argument("--cpu-seconds", type=float, default=12.0)
    ap.add_argument("--cpu-cols", type=int, default=8192)
    ap.add_argument("--ref-cols", type=int, default=8192)
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--no-parity", action="store_true", help="skip the full oracle comparison of the timed run")
    ap.add_argument("--no-tune", action="store_true", help="skip the autotuner (library default shape)")
    ap.add_argument("--train-pairs", type=int, default=200_000, help="surrogate-n200: labelled tours")
    ap.add_argument("--epochs", type=int, default=8, help="surrogate-n200: training epochs")
    ap.add_argument("--repeats", type=int, default=3, help="oos-n200: searches per training-set size; "
                    "surrogate-n200: search starts")
    args = ap.parse_args()
    if args.steps < 1 or args.warmup < 0:
        raise SystemExit("steps >= 1, warmup >= 0")
    if args.impl == "reference":
        return run_reference(args)
    if args.workload == "batched-512":
        return run_batched(args)
    if args.workload == "surrogate-n200":
        return run_surrogate(args)
    if args.workload == "latency-n1000":
        return run_latency(args)
    if args.workload == "oos-n200":
        return run_oos(args)
    return run_ours(args)


if __name__ == "__main__":
    sys.exit(main())
