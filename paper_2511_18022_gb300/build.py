"""Builds libcvrpsd.so (the C ABI of include/cvrpsd.h) in-tree with nvcc for
sm_103a. Translation units compile in parallel; nothing is installed."""
from __future__ import annotations

import concurrent.futures as cf
import fcntl
import os
import platform
import shutil
import subprocess

PKG = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(PKG)
CSRC = os.path.join(PKG, "csrc")
INCLUDE = os.path.join(ROOT, "include")
BUILD = os.path.join(PKG, "_build", platform.machine())
LIB = os.path.join(BUILD, "libcvrpsd.so")

ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
CFLAGS = ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", "-Xptxas", "-v",
          "-I" + INCLUDE, "-I" + CSRC]

# (source, extra defines, object name)
UNITS = [("split_deque.cu", [f"-DCVRPSD_DEQUE_PART={k}"], f"split_deque_{k}.o") for k in range(4)] + [
    ("split_deque2.cu", [f"-DCVRPSD_DEQUE2_PART={k}"], f"split_deque2_{k}.o") for k in range(4)] + [
    ("split_batch.cu", ["-DCVRPSD_BATCH_PART=0"], "split_batch_0.o"),
    ("split_batch.cu", ["-DCVRPSD_BATCH_PART=1"], "split_batch_1.o"),
    ("split_batch.cu", ["-DCVRPSD_BATCH_PART=2"], "split_batch_2.o"),
    ("split_batch.cu", ["-DCVRPSD_BATCH_PART=3"], "split_batch_3.o"),
    ("split_batch2.cu", ["-DCVRPSD_BATCH2_PART=0"], "split_batch2_0.o"),
    ("split_batch2.cu", ["-DCVRPSD_BATCH2_PART=1"], "split_batch2_1.o"),
    ("split_warp.cu", [], "split_warp.o"),
    ("gen_demand.cu", [], "gen_demand.o"),
    ("api.cu", [], "api.o"),
    ("search.cu", [], "search.o"),
    ("seqpar.cu", [], "seqpar.o"),
    ("mlp.cu", [], "mlp.o"),
    ("mlp_tc.cu", [], "mlp_tc.o"),
    ("search_api.cu", [], "search_api.o"),
    ("noalloc.cu", [], "noalloc.o"),
    ("probe.cu", [], "probe.o"),
]


def nvcc() -> str:
    exe = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    if not os.path.exists(exe):
        raise RuntimeError("nvcc not found: the CUDA toolkit is required to build libcvrpsd")
    return exe


def _deps_mtime() -> float:
    files = [os.path.join(CSRC, f) for f in os.listdir(CSRC)] + [os.path.join(INCLUDE, "cvrpsd.h"),
                                                                  os.path.abspath(__file__)]
    return max(os.path.getmtime(f) for f in files if os.path.isfile(f))


def _compile(unit, build_dir=None, extra=()):
    src, defs, obj = unit
    out = os.path.join(build_dir or BUILD, obj)
    cmd = [nvcc()] + ARCH + CFLAGS + list(extra) + defs + ["-c", os.path.join(CSRC, src), "-o", out]
    r = subprocess.run(cmd, capture_output=True, text=True)
    with open(out + ".log", "w") as f:
        f.write(" ".join(cmd) + "\n" + r.stdout + r.stderr)
    if r.returncode != 0:
        raise RuntimeError(f"nvcc failed on {src}:\n{r.stderr[-4000:]}")
    return out


def build(force: bool = False, jobs: int | None = None, build_dir: str | None = None,
          extra_flags=()) -> str:
    """Compile every CUDA unit and link the shared library; returns its path.
    `build_dir` / `extra_flags` build a variant elsewhere (tuning experiments)."""
    lib = os.path.join(build_dir, "libcvrpsd.so") if build_dir else LIB
    if not force and os.path.exists(lib) and os.path.getmtime(lib) >= _deps_mtime():
        return lib
    bdir = build_dir or BUILD
    os.makedirs(bdir, exist_ok=True)
    # One build at a time per directory (several ranks may start at once);
    # whoever waited finds the library current and returns.
    with open(os.path.join(bdir, ".lock"), "w") as lock:
        fcntl.flock(lock, fcntl.LOCK_EX)
        try:
            if not force and os.path.exists(lib) and os.path.getmtime(lib) >= _deps_mtime():
                return lib
            return _build_locked(lib, bdir, jobs, extra_flags)
        finally:
            fcntl.flock(lock, fcntl.LOCK_UN)


def _build_locked(lib, bdir, jobs, extra_flags) -> str:
    jobs = jobs or min(len(UNITS), os.cpu_count() or 4)
    with cf.ThreadPoolExecutor(jobs) as ex:
        objs = list(ex.map(lambda u: _compile(u, bdir, extra_flags), UNITS))
    tmp = lib + f".tmp{os.getpid()}"
    cmd = [nvcc()] + ARCH + ["-shared", "-cudart", "shared", "-Xlinker", "-rpath=/usr/local/cuda/lib64",
                             "-o", tmp] + objs
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"link failed:\n{r.stderr[-4000:]}")
    os.replace(tmp, lib)
    return lib


def build_checked(force: bool = False) -> str:
    """The checked variant of the library (-DCVRPSD_CHECKED=1: every index a
    Split kernel forms from data is compared with its buffer, and a bad one
    is reported as CVRPSD_ERR_DEVICE_STATUS instead of being used) in its own
    build folder; returns its path. A debugging aid, slower than the regular
    build."""
    return build(force=force, build_dir=BUILD + "-checked", extra_flags=["-DCVRPSD_CHECKED=1"])


def resource_usage() -> str:
    """ptxas register / spill / shared-memory report of the last build."""
    out = []
    for _, _, obj in UNITS:
        log = os.path.join(BUILD, obj + ".log")
        if os.path.exists(log):
            out += [ln for ln in open(log) if "registers" in ln or "spill" in ln or "Compiling entry" in ln]
    return "".join(out)


if __name__ == "__main__":
    import sys
    print(build_checked(force=True) if "--checked" in sys.argv else build(force=True))
