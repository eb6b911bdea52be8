"""Synthetic CVRPSD instances: customers, distances, mean demands, tours.

Recipe (seeded, host side; every draw comes from one SplitMix64 stream):
  1. customer coordinates x_1, y_1, ..., x_n, y_n: uniform integers in
     [0, 1000] (both ends included), drawn in that order; the depot is node 0
     at (500, 500);
  2. mean demands mu_1..mu_n: uniform integers in [mu_lo, mu_hi];
  3. the giant tour: a Fisher-Yates permutation of customer ids 1..n.
Distances are rounded Euclidean integers, floor(sqrt(dx^2 + dy^2) + 0.5),
computed in float64 (sqrt is correctly rounded and sqrt of a non-square
integer is irrational, so no half-way tie exists). The correlation region of a
customer is its quadrant around the depot, r = (dx < 0) + 2 * (dy < 0).

This module holds no Split arithmetic.
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np

from .rng import SplitMix64, derive_seed

DEPOT_XY = (500, 500)
COORD_MAX = 1000


@dataclass
class Instance:
    n: int
    coords: np.ndarray        # (n+1, 2) int64, row 0 = depot
    dist: np.ndarray          # (n+1, n+1) int32, row = from, column = to
    mu: np.ndarray            # (n,) int64, mean demand of customer id k at [k-1]
    region: np.ndarray        # (n,) int64 in 0..3, quadrant of customer id k at [k-1]
    tour: np.ndarray          # (n,) int32, customer ids 1..n in visiting order
    Q: int
    L: int
    seed: int
    meta: dict = field(default_factory=dict)


def rounded_euclidean(coords: np.ndarray) -> np.ndarray:
    c = np.asarray(coords, dtype=np.float64)
    d = np.sqrt(((c[:, None, :] - c[None, :, :]) ** 2).sum(-1))
    return np.floor(d + 0.5).astype(np.int32)


def quadrant_regions(coords: np.ndarray) -> np.ndarray:
    dx = coords[1:, 0] - coords[0, 0]
    dy = coords[1:, 1] - coords[0, 1]
    return (dx < 0).astype(np.int64) + 2 * (dy < 0).astype(np.int64)


def make_instance(n: int, mu_lo: int, mu_hi: int, seed: int,
                  Q: int | None = None, L: int | None = None,
                  q_from_mean: int | None = None) -> Instance:
    """Draw one instance. `q_from_mean=k` sets Q to k * mean(mu) rounded to
    the nearest integer, computed exactly as floor((k*sum(mu) + n//2) / n)."""
    rng = SplitMix64(seed)
    xy = rng.integers(0, COORD_MAX, 2 * n).reshape(n, 2)
    coords = np.vstack([np.array([DEPOT_XY], dtype=np.int64), xy])
    mu = rng.integers(mu_lo, mu_hi, n)
    tour = rng.permutation(range(1, n + 1)).astype(np.int32)
    if q_from_mean is not None:
        Q = (q_from_mean * int(mu.sum()) + n // 2) // n
    if Q is None:
        raise ValueError("Q is required")
    return Instance(n=n, coords=coords, dist=rounded_euclidean(coords), mu=mu,
                    region=quadrant_regions(coords), tour=tour, Q=int(Q),
                    L=int(n if L is None else L), seed=seed)


def instance_from_coords(coords, tour, Q: int, L: int | None = None,
                         mu=None) -> Instance:
    """Instance with given coordinates (row 0 = depot) and tour."""
    coords = np.asarray(coords, dtype=np.int64)
    n = coords.shape[0] - 1
    mu = np.ones(n, dtype=np.int64) if mu is None else np.asarray(mu, dtype=np.int64)
    return Instance(n=n, coords=coords, dist=rounded_euclidean(coords), mu=mu,
                    region=quadrant_regions(coords),
                    tour=np.asarray(tour, dtype=np.int32), Q=int(Q),
                    L=int(n if L is None else L), seed=-1)


def batched_tour_sizes(T: int, n_lo: int, n_hi: int, seed: int) -> np.ndarray:
    return SplitMix64(seed).integers(n_lo, n_hi, T)


def batched_instances(T: int, n_lo: int, n_hi: int, mu_lo: int, mu_hi: int,
                      seed: int, q_mult: int) -> list[Instance]:
    """Multi-tour workload: tour t has n_t ~ U{n_lo..n_hi} customers, its own
    coordinates and mean demands (seed derived from (seed, t)),
    Q_t = q_mult * mean(mu_t) rounded, and no route-length cap (L = n_t)."""
    sizes = batched_tour_sizes(T, n_lo, n_hi, seed)
    return [make_instance(int(sizes[t]), mu_lo, mu_hi, derive_seed(seed, t),
                          q_from_mean=q_mult) for t in range(T)]
