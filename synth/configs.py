"""Named synthetic workloads for the scenario-batched Split.

plain-n50      : n=50, S=1,000, NORMAL demands, mu ~ U{1..10}, Q=40, no
                 route-length cap, int32 demands, instance seed 0.
corr-n200      : n=200, S=100,000, CORRELATED demands, mu ~ U{5..20},
                 Q=150, at most 40 customers per route, int16 demands.
million-n1000  : n=1,000, S=2^20, CORRELATED demands, mu ~ U{1..30},
                 Q=200, at most 60 customers per route, int16 demands.
batched-512    : 512 tours, n_t ~ U{100..1000}, each with its own
                 coordinates and mu ~ U{1..10}, CORRELATED demands,
                 Q_t = 10 * mean(mu_t) rounded, no cap, S=65,536 each.
surrogate-n200 : the corr-n200 instance generator, for local search.

Scenario seeds are derived from (instance seed, 1000 + tour index) so every
workload is reproducible from its name alone.
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np

from .instances import Instance, make_instance, batched_instances
from .rng import derive_seed
from .scenarios import KIND_NORMAL, KIND_CORRELATED


@dataclass
class Workload:
    name: str
    instances: list
    S: int
    kind: int
    dtype: type
    scen_seeds: list

    @property
    def cells(self) -> int:
        return int(sum(inst.n for inst in self.instances)) * self.S


def _single(name, n, mu, seed, Q, L, S, kind, dtype):
    inst = make_instance(n, mu[0], mu[1], seed, Q=Q, L=L)
    return Workload(name, [inst], S, kind, dtype, [derive_seed(seed, 1000)])


def workload(name: str, S: int | None = None, T: int | None = None) -> Workload:
    """Build a named workload. `S` (and `T` for the batched one) may be
    overridden to make a scaled-down case of the same generator."""
    if name == "plain-n50":
        return _single(name, 50, (1, 10), 0, 40, None, S or 1000,
                       KIND_NORMAL, np.int32)
    if name == "corr-n200":
        return _single(name, 200, (5, 20), 1, 150, 40, S or 100_000,
                       KIND_CORRELATED, np.int16)
    if name == "million-n1000":
        return _single(name, 1000, (1, 30), 2, 200, 60, S or (1 << 20),
                       KIND_CORRELATED, np.int16)
    if name == "batched-512":
        T = T or 512
        insts = batched_instances(T, 100, 1000, 1, 10, seed=3, q_mult=10)
        seeds = [derive_seed(3, 1000 + t) for t in range(T)]
        return Workload(name, insts, S or 65_536, KIND_CORRELATED, np.int16, seeds)
    if name == "surrogate-n200":
        return _single(name, 200, (5, 20), 4, 150, 40, S or 65_536,
                       KIND_CORRELATED, np.int16)
    raise KeyError(name)


WORKLOADS = ["plain-n50", "corr-n200", "million-n1000", "batched-512",
             "surrogate-n200"]
