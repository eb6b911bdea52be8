"""Scenario sharding across ranks (one process per GPU).

Scenarios are independent, so the Split shards by scenario with no exchange
on the data path: rank r of W splits the contiguous columns
[r * S // W, (r + 1) * S // W) of the scenario matrix. The sample average
over all S scenarios (Appendix A) is the only cross-rank step: one int64
all-reduce of (sum of feasible costs, infeasible count).
"""
from __future__ import annotations


def scenario_range(S: int, rank: int, world: int) -> tuple[int, int]:
    """Contiguous scenario columns [lo, hi) of `rank`; the ranges of ranks
    0..world-1 partition 0..S-1."""
    if world < 1 or not 0 <= rank < world:
        raise ValueError("need 0 <= rank < world")
    return S * rank // world, S * (rank + 1) // world


def allreduce_saa(local_sum: int, local_infeasible: int, S_total: int, device: str = "cpu"):
    """Exact global (sum, infeasible, mean) from every rank's partial sums,
    with torch.distributed's current process group: one all-reduce of two
    int64 on `device` ("cuda" goes over NCCL, "cpu" over gloo)."""
    import torch
    import torch.distributed as dist
    t = torch.tensor([int(local_sum), int(local_infeasible)], dtype=torch.int64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.SUM)
    total, inf = int(t[0].item()), int(t[1].item())
    feas = S_total - inf
    return total, inf, (total / feas if feas > 0 else float("nan"))


def split_and_reduce(split_shard, S_total: int, world: int, device: str = "cpu"):
    """One sharded step: `split_shard()` splits this rank's scenarios and
    returns an object with .sum and .infeasible; the global SAA follows from
    one all-reduce (none with a single rank). Returns (sum, infeasible, mean)
    over all S_total scenarios."""
    r = split_shard()
    if world == 1:
        feas = S_total - r.infeasible
        return r.sum, r.infeasible, (r.sum / feas if feas > 0 else float("nan"))
    return allreduce_saa(r.sum, r.infeasible, S_total, device)
