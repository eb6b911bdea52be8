"""The multi-rank path on CPU: two gloo ranks split one scenario set, each
evaluates its columns, and the benchmark's step function (shard.split_and_reduce:
one int64 all-reduce) gives the exact global SAA sum; the benchmark's barrier,
max-over-ranks timing and sum-over-ranks parity helpers work across ranks. (The kernels run one process per GPU; here the CPU oracle stands in
for each rank's kernel, since only the host logic is under test.)"""
import os
import socket

import numpy as np
import pytest
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def worker(rank, world, port, S, out):
    import sys
    sys.path.insert(0, ROOT)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), WORLD_SIZE=str(world), RANK=str(rank),
                      LOCAL_RANK=str(rank))
    import bench
    import oracle
    from paper_2511_18022_gb300.shard import scenario_range, split_and_reduce
    from synth import demand_columns, workload
    w_, r_, _ = bench.dist_setup()
    assert (w_, r_) == (world, rank)
    w = workload("corr-n200", S=S)
    inst = w.instances[0]
    lo, hi = scenario_range(S, rank, world)
    D = demand_columns(inst.mu, inst.region, w.kind, w.scen_seeds[0], np.arange(lo, hi), np.int16)
    D[0, 0] = inst.Q + 1                                  # one infeasible scenario per rank

    class R:                                               # what a Split call returns
        pass

    def split_shard():                                     # the oracle stands in for the kernel
        r = R()
        _, r.sum, r.infeasible, _ = oracle.split_costs(inst.tour, inst.dist, D, inst.Q, inst.L)
        return r

    # the benchmark's step: this rank's shard, then one all-reduce of the SAA
    total, tinf, mean = split_and_reduce(split_shard, S, world, device="cpu")
    bench.barrier(world)
    mx = bench.max_over_ranks(world, float(rank) + 1.5)
    counts = bench.sum_over_ranks(world, [rank + 1, 10 * rank])
    out.put((rank, lo, hi, total, tinf, mean, mx, counts))
    import torch.distributed as dist
    dist.destroy_process_group()


def test_two_gloo_ranks_shard_scenarios_exactly():
    S, world = 301, 2
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = free_port()
    procs = [ctx.Process(target=worker, args=(r, world, port, S, q)) for r in range(world)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=300) for _ in range(world))
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    import oracle
    from synth import demand_matrix, workload
    w = workload("corr-n200", S=S)
    inst = w.instances[0]
    D = demand_matrix(inst.mu, inst.region, w.kind, w.scen_seeds[0], S, dtype=np.int16)
    for (_, lo, _, _, _, _, _, _) in res:
        D[0, lo] = inst.Q + 1
    _, s, inf, _ = oracle.split_costs(inst.tour, inst.dist, D, inst.Q, inst.L)
    assert [r[1:3] for r in res] == [(0, 150), (150, 301)]
    for r in res:
        assert (r[3], r[4]) == (s, inf) and r[5] == s / (S - inf)
        assert r[6] == 2.5                                # max over ranks of rank + 1.5
        assert r[7] == [3, 10]                            # sums over ranks (parity counts)


def test_scenario_range_partitions():
    from paper_2511_18022_gb300.shard import scenario_range
    for S in (0, 1, 7, 1000, 2**20 + 3):
        for world in (1, 2, 3, 8):
            ranges = [scenario_range(S, r, world) for r in range(world)]
            assert ranges[0][0] == 0 and ranges[-1][1] == S
            assert all(a[1] == b[0] for a, b in zip(ranges, ranges[1:]))
    with pytest.raises(ValueError):
        scenario_range(10, 2, 2)


def test_cpulist_parsing():
    from paper_2511_18022_gb300.hostmem import _cpulist
    assert _cpulist("0-3,8,10-11\n") == {0, 1, 2, 3, 8, 10, 11}
    assert _cpulist("") == set()
