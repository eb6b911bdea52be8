"""Bit-exact parity of the full headline workload, every scenario.

million-n1000 (n = 1000, S = 2^20, Q = 200, L = 60, correlated int16
demands): the whole 2.1 GB scenario matrix is generated on the host by the
seeded recipe (synth, worker processes), copied to the device, split there
in the launch configuration the benchmark times (autotuned shape), and all
1,048,576 per-scenario costs, the exact sum and the infeasible count are
compared with the oracle run over every column on the host cores. The
host-buffer entry point (the benchmark's end-to-end call) is checked on the
same matrix, also in full."""
import os

import numpy as np
import pytest

import oracle
from synth import demand_matrix_parallel, workload

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu
INT32_MAX = 2**31 - 1


@pytest.fixture(scope="module")
def cv():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2511_18022_gb300 import build
    build.build()
    import paper_2511_18022_gb300 as m
    return m


@pytest.fixture(scope="module")
def million():
    w = workload("million-n1000")
    inst = w.instances[0]
    H = torch.empty((inst.n, w.S), dtype=torch.int16, pin_memory=True)
    demand_matrix_parallel(inst.mu, inst.region, w.kind, w.scen_seeds[0], w.S, dtype=np.int16,
                           workers=os.cpu_count(), out=H.numpy())
    want, wsum, winf, relax = oracle.split_costs(inst.tour, inst.dist, H.numpy(), inst.Q, inst.L,
                                                 nthreads=os.cpu_count())
    return w, inst, H, want, wsum, winf, relax


def test_every_scenario_of_the_headline_workload(cv, million):
    w, inst, H, want, wsum, winf, relax = million
    sp = cv.Splitter(0)
    try:
        D = H.cuda()
        sp.autotune(inst.tour, inst.dist, D, inst.Q, inst.L)   # the benchmark's launch shape
        out = torch.full((w.S,), -1, dtype=torch.int32, device="cuda")
        r = sp.split(inst.tour, inst.dist, D, inst.Q, inst.L, out_cost=out)
        got = out.cpu().numpy()
        assert int((got != want).sum()) == 0
        assert (r.sum, r.infeasible) == (wsum, winf)
        assert r.mean == wsum / (w.S - winf)
        # the exact relaxation count the ALU roofline uses: one per feasible (p, i)
        assert 12.0 < relax / (inst.n * w.S) < 14.0
    finally:
        sp.close()


def test_every_scenario_through_host_buffers(cv, million):
    w, inst, H, want, wsum, winf, _ = million
    sp = cv.Splitter(0)
    try:
        Hout = torch.full((w.S,), -1, dtype=torch.int32, pin_memory=True)
        r = sp.split_host(inst.tour, inst.dist, H, inst.Q, inst.L, out_cost=Hout)
        assert int((Hout.numpy() != want).sum()) == 0
        assert (r.sum, r.infeasible) == (wsum, winf)
    finally:
        sp.close()
