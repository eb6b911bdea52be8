"""Seeded synthetic inputs shared by the oracle tests, the CUDA parity tests and
the benchmark. Nothing here computes any part of the Split itself."""
from .rng import SplitMix64, derive_seed, philox4x32_10
from .instances import (Instance, make_instance, instance_from_coords,
                        batched_instances, batched_tour_sizes, rounded_euclidean)
from .scenarios import (KIND_NORMAL, KIND_CORRELATED, demand_columns,
                        demand_matrix)
from .configs import WORKLOADS, workload
from .parallel import demand_matrix_parallel

__all__ = [
    "SplitMix64", "derive_seed", "philox4x32_10", "Instance", "make_instance",
    "instance_from_coords", "batched_instances", "batched_tour_sizes",
    "rounded_euclidean", "KIND_NORMAL", "KIND_CORRELATED", "demand_columns",
    "demand_matrix", "demand_matrix_parallel", "WORKLOADS", "workload",
]
