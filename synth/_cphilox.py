"""Loader of synth/philox.c (compiled with gcc on first use, like the oracle):
Philox4x32-10 words for a grid of counters, bit-identical to
rng.philox4x32_10 and much faster on large grids. None if it cannot be built;
callers then use the numpy version."""
from __future__ import annotations

import ctypes
import os
import platform
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "philox.c")
_lib = None
_tried = False


def lib_path() -> str:
    return os.path.join(_HERE, "_build", f"libsynth_{platform.machine()}.so")


def build() -> str:
    out = lib_path()
    if not os.path.exists(out) or os.path.getmtime(out) < os.path.getmtime(_SRC):
        os.makedirs(os.path.dirname(out), exist_ok=True)
        tmp = out + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-std=c11", "-fPIC", "-shared", _SRC, "-o", tmp])
        os.replace(tmp, out)
    return out


def load():
    global _lib, _tried
    if _tried:
        return _lib
    _tried = True
    try:
        lib = ctypes.CDLL(build())
        P = ctypes.c_void_p
        lib.synth_philox_words.restype = None
        lib.synth_philox_words.argtypes = [P, ctypes.c_int64, P, ctypes.c_int64, ctypes.c_uint32,
                                           ctypes.c_uint32, ctypes.c_uint32, P, P]
        _lib = lib
    except Exception:
        _lib = None
    return _lib


def words(s: np.ndarray, index: np.ndarray, domain: int, k0: int, k1: int):
    """Words 0 and 1 of Philox4x32-10 at counters (s[j], index[r], domain, 0)
    as [len(index)][len(s)] uint32 arrays, or None without the C library."""
    lib = load()
    if lib is None:
        return None
    s = np.ascontiguousarray(s, dtype=np.int64).reshape(-1)
    index = np.ascontiguousarray(index, dtype=np.int64).reshape(-1)
    w0 = np.empty((index.size, s.size), dtype=np.uint32)
    w1 = np.empty_like(w0)
    lib.synth_philox_words(s.ctypes.data, s.size, index.ctypes.data, index.size, domain & 0xFFFFFFFF,
                           k0 & 0xFFFFFFFF, k1 & 0xFFFFFFFF, w0.ctypes.data, w1.ctypes.data)
    return w0, w1
