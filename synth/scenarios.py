"""Counter-based demand scenarios.

Demand of customer id k (row k-1) in scenario s, for the two workload kinds:

* NORMAL: d = max(0, round(mu_k + 0.3 * mu_k * Z_sk)), Z ~ N(0, 1) i.i.d.
* CORRELATED: d = max(0, round(mu_k * exp(0.3 * (0.6 * F_{s,r(k)}
                                              + 0.8 * E_sk) - 0.045))),
  F and E i.i.d. N(0, 1); F is shared by the customers of one quadrant r in
  one scenario, so log-demands correlate at 0.6^2 = 0.36 within a quadrant
  and not at all across quadrants. 0.6^2 + 0.8^2 = 1 and the -0.045 =
  -0.3^2 / 2 shift make the multiplier mean-preserving: E[exp(0.3 Y - 0.045)]
  = 1 for Y ~ N(0, 1).

round() is half-away-from-zero; values are clamped to the storage type's
maximum. Each standard normal is one Box-Muller draw from the first two words
of a Philox4x32-10 block whose counter is (s, index, domain, 0) and whose key
is the 64-bit scenario seed split into two 32-bit halves:
    u1 = (w0 + 0.5) / 2^32,   u2 = w1 / 2^32,
    z  = sqrt(-2 log u1) * cos(TWO_PI * u2),
with domain 0 for E (index = customer row), 1 for F (index = quadrant) and
2 for Z (index = customer row). All arithmetic is float64, each operation
rounded on its own (no fused multiply-add), in the order written here.

The CUDA scenario generator computes the same recipe; its math library may
differ from numpy's by an ulp in log/cos/exp, which can move a demand across a
rounding boundary, so the two agree except on rare entries (by at most 1).
This module holds no Split arithmetic.
"""
from __future__ import annotations

import numpy as np

from . import _cphilox
from .rng import philox4x32_10

KIND_NORMAL = 0
KIND_CORRELATED = 1

DOM_E = 0
DOM_F = 1
DOM_Z = 2

TWO_PI = 6.283185307179586
INV_2_32 = 1.0 / 4294967296.0

DTYPE_MAX = {np.dtype(np.int16): 32767, np.dtype(np.int32): 2147483647}


def key_halves(seed: int) -> tuple[int, int]:
    return seed & 0xFFFFFFFF, (seed >> 32) & 0xFFFFFFFF


def box_muller(w0: np.ndarray, w1: np.ndarray) -> np.ndarray:
    u1 = (w0.astype(np.float64) + 0.5) * INV_2_32
    u2 = w1.astype(np.float64) * INV_2_32
    return np.sqrt(-2.0 * np.log(u1)) * np.cos(TWO_PI * u2)


def std_normal(seed: int, s: np.ndarray, index: np.ndarray, domain: int) -> np.ndarray:
    k0, k1 = key_halves(seed)
    s, index = np.asarray(s), np.asarray(index)
    if s.ndim == 2 and s.shape[0] == 1 and index.ndim == 2 and index.shape[1] == 1:
        # a [rows][columns] grid: the C words (same function, faster)
        w = _cphilox.words(s[0], index[:, 0], domain, k0, k1)
        if w is not None:
            return box_muller(w[0], w[1])
    w = philox4x32_10(s, index, domain, 0, k0, k1)
    return box_muller(w[0], w[1])


def round_half_away(x: np.ndarray) -> np.ndarray:
    r = np.floor(x)
    return r + ((x - r) >= 0.5)


def demand_columns(mu, region, kind: int, seed: int, scen, dtype=np.int16) -> np.ndarray:
    """Demands for the scenarios listed in `scen`: array [n][len(scen)]
    (row = customer id - 1, scenario fastest), the layout the Split reads."""
    mu = np.asarray(mu, dtype=np.int64)
    region = np.asarray(region, dtype=np.int64)
    scen = np.asarray(scen, dtype=np.int64)
    n = mu.shape[0]
    s2 = scen[None, :]
    rows = np.arange(n, dtype=np.int64)[:, None]
    muf = mu.astype(np.float64)[:, None]
    if kind == KIND_NORMAL:
        z = std_normal(seed, s2, rows, DOM_Z)
        x = muf + (0.3 * muf) * z
    elif kind == KIND_CORRELATED:
        e = std_normal(seed, s2, rows, DOM_E)
        f4 = std_normal(seed, s2, np.arange(4, dtype=np.int64)[:, None], DOM_F)
        f = f4[region, :]
        y = 0.6 * f + 0.8 * e
        x = muf * np.exp(0.3 * y - 0.045)
    else:
        raise ValueError(f"unknown demand kind {kind}")
    d = np.maximum(round_half_away(x), 0.0)
    d = np.minimum(d, float(DTYPE_MAX[np.dtype(dtype)]))
    return d.astype(dtype)


def demand_matrix(mu, region, kind: int, seed: int, S: int, s0: int = 0,
                  dtype=np.int16, chunk: int = 1 << 15) -> np.ndarray:
    """All scenarios s0 .. s0+S-1, generated in column chunks."""
    n = len(mu)
    out = np.empty((n, S), dtype=dtype)
    for a in range(0, S, chunk):
        b = min(S, a + chunk)
        out[:, a:b] = demand_columns(mu, region, kind, seed,
                                     np.arange(s0 + a, s0 + b), dtype)
    return out
