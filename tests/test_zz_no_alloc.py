"""The allocation-free Split entry point against the regular one.

cvrpsd_split_eval_noalloc serves callers that cannot allocate device memory
when they call (all device memory already handed to their own pool, or a
cudaMalloc that could block or fail in the middle of a loop). It keeps its
scratch in one fixed device array shared by every call, so this test makes
two calls in a row with different tours, sizes and set-aside scenarios and
checks both against cvrpsd_split_eval bit for bit (costs are integers). The
file name sorts last so that a run stopping at the first failure has already
run every other test."""
import numpy as np
import pytest

from synth import demand_matrix, workload

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def cv():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2511_18022_gb300 import build
    build.build()
    import paper_2511_18022_gb300 as m
    return m


def case(name, S, bump):
    w = workload(name, S=S)
    inst = w.instances[0]
    D = demand_matrix(inst.mu, inst.region, w.kind, w.scen_seeds[0], S, dtype=w.dtype)
    for k, s in enumerate(bump):        # demands above Q: these go to the warp kernel
        D[(7 * k) % inst.n, s] = inst.Q + 1
    return inst, torch.from_numpy(D).cuda()


def test_noalloc_matches_regular_entry_twice(cv):
    sp = cv.Splitter(0)
    try:
        for name, S, bump in (("corr-n200", 20_011, [5, 777, 20_010]), ("plain-n50", 3001, [0])):
            inst, D = case(name, S, bump)
            want = torch.full((S,), -1, dtype=torch.int32, device="cuda")
            r_want = sp.split(inst.tour, inst.dist, D, inst.Q, inst.L, out_cost=want)
            got = torch.full((S,), -2, dtype=torch.int32, device="cuda")
            r_got = cv.cvrpsd_split_eval_noalloc(inst.tour, inst.dist, D, inst.Q, inst.L, out_cost=got)
            assert torch.equal(got, want)
            assert (r_got.status, r_got.sum, r_got.infeasible) == (r_want.status, r_want.sum, r_want.infeasible)
            assert r_got.infeasible == len(bump)
            assert r_got.mean == r_want.mean
    finally:
        sp.close()


def test_noalloc_rejects_too_many_scenarios(cv):
    inst, D = case("plain-n50", 64, [])
    too_many = cv._lib.NOALLOC_MAX_S + 1
    with pytest.raises(cv.CvrpsdError) as e:
        cv.cvrpsd_split_eval_noalloc(inst.tour, inst.dist, D.data_ptr(), inst.Q, inst.L,
                                     S=too_many, ld=too_many, dtype=cv.I32)
    assert e.value.code == -7


def test_noalloc_refuses_a_capturing_stream(cv):
    """The call stages its tour table through one host buffer shared by all
    calls; recorded into a graph, that copy would read the buffer at replay
    time. A call on a capturing stream must therefore be refused, not
    recorded."""
    inst, D = case("plain-n50", 256, [])
    cv.cvrpsd_split_eval_noalloc(inst.tour, inst.dist, D, inst.Q, inst.L)   # device set-up first
    torch.cuda.synchronize()
    s = torch.cuda.Stream()
    g = torch.cuda.CUDAGraph()
    code = None
    with torch.cuda.graph(g, stream=s):
        try:
            cv.cvrpsd_split_eval_noalloc(inst.tour, inst.dist, D, inst.Q, inst.L, host_outputs=False, stream=s)
        except cv.CvrpsdError as e:
            code = e.code
    assert code == -7
    # the device is still usable and the entry point still exact
    r = cv.cvrpsd_split_eval_noalloc(inst.tour, inst.dist, D, inst.Q, inst.L)
    sp = cv.Splitter(0)
    try:
        assert r.sum == sp.split(inst.tour, inst.dist, D, inst.Q, inst.L).sum
    finally:
        sp.close()
