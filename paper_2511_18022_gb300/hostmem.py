"""Page-locked host buffers placed next to the GPU.

The host-buffer Split (cvrpsd_split_eval_host) streams the scenario matrix
from page-locked host memory across the CPU-GPU link. Pages are placed on
the NUMA node of the thread that allocates them, so the allocation is made
by the calling thread while it is bound to the CPUs next to the GPU (sysfs
local_cpulist of the GPU's PCI function), and the placement can be read back
from /proc/self/numa_maps. Host-side plumbing only: no Split arithmetic.
"""
from __future__ import annotations

import os
import subprocess


def _cpulist(text: str) -> set:
    cpus = set()
    for part in text.strip().split(","):
        if "-" in part:
            a, b = part.split("-")
            cpus |= set(range(int(a), int(b) + 1))
        elif part:
            cpus.add(int(part))
    return cpus


def gpu_numa(device: int = 0):
    """(NUMA node, set of nearby CPU ids) of CUDA device `device`, read from
    sysfs through its PCI bus id; (None, None) where unknown."""
    try:
        bus = subprocess.run(["nvidia-smi", "-i", str(device), "--query-gpu=pci.bus_id",
                              "--format=csv,noheader"], capture_output=True, text=True,
                             timeout=30).stdout.strip().lower()
        dom, rest = bus.split(":", 1)
        path = f"/sys/bus/pci/devices/{int(dom, 16):04x}:{rest}"
        node = int(open(path + "/numa_node").read().strip())
        cpus = _cpulist(open(path + "/local_cpulist").read())
        return node, cpus
    except Exception:
        return None, None


def pages_by_node(addr: int) -> dict:
    """Resident pages per NUMA node ({"N0": count, ...}) of the mapping that
    holds host address `addr`, from /proc/self/numa_maps; {} if not found."""
    try:
        ranges = {}
        with open("/proc/self/maps") as m:
            for ml in m:
                a, b = (int(x, 16) for x in ml.split()[0].split("-"))
                ranges[a] = b
        for line in open("/proc/self/numa_maps"):
            parts = line.split()
            start = int(parts[0], 16)
            if start <= addr < ranges.get(start, start):
                return {kv.split("=")[0]: int(kv.split("=")[1]) for kv in parts[2:]
                        if kv.startswith("N") and "=" in kv}
    except Exception:
        pass
    return {}


def pinned_near_gpu(shape, dtype, device: int = 0):
    """A page-locked torch tensor whose pages were allocated (and touched)
    while this thread ran on the CPUs next to CUDA device `device`. Returns
    (tensor, placement) with placement = {"gpu_numa_node", "pages_by_node",
    "bound"}."""
    import torch
    node, cpus = gpu_numa(device)
    keep = os.sched_getaffinity(0)
    usable = (cpus or set()) & keep
    if usable:
        os.sched_setaffinity(0, usable)
    try:
        t = torch.empty(shape, dtype=dtype, pin_memory=True)
        t.numpy().fill(0)
    finally:
        os.sched_setaffinity(0, keep)
    return t, {"gpu_numa_node": node, "pages_by_node": pages_by_node(t.data_ptr()), "bound": bool(usable)}
