"""Error paths under memory exhaustion, without exhausting memory: the
library's test hook makes one allocation of a context fail as if the device
were out of memory. Every call must then fail cleanly with CVRPSD_ERR_NOMEM
(no launch on a half-allocated context), and the same context must give exact
results once memory is available again."""
import numpy as np
import pytest

import oracle
from synth import KIND_NORMAL, demand_matrix, make_instance

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


def case():
    inst = make_instance(120, 5, 20, seed=21, Q=70, L=25)
    S = 640
    D = demand_matrix(inst.mu, inst.region, KIND_NORMAL, 8, S)
    want, wsum, winf, _ = oracle.split_costs(inst.tour, inst.dist, D, inst.Q, inst.L, nthreads=8)
    return inst, S, D, want, wsum, winf


def run_all(cv, sp, inst, S, Dd):
    """Every allocating path of a context once; returns the results."""
    out = torch.empty(S, dtype=torch.int32, device="cuda")
    r = sp.split(inst.tour, inst.dist, Dd, inst.Q, inst.L, out_cost=out)
    G = torch.empty((inst.n, 64), dtype=torch.int16, device="cuda")
    sp.gen_demand(5, cv.GEN_NORMAL, inst.mu, inst.region, G)
    b = sp.batch([dict(tour=inst.tour, dist=inst.dist, demand=Dd, Q=inst.Q, L=inst.L)], S)
    b.run()
    bres = b.results()
    b.close()
    cust = np.column_stack([inst.coords[1:, 0], inst.coords[1:, 1], inst.mu,
                            np.ones(inst.n)]).astype(np.float32)
    sur = cv.Surrogate(sp.ctx, cust, inst.dist, Q=float(inst.Q), seed=1)
    tours = torch.from_numpy(np.stack([inst.tour, inst.tour[::-1].copy()]).astype(np.int32)).cuda()
    pred = torch.empty(2, dtype=torch.float32, device="cuda")
    sur.predict(tours, pred)
    sur.close()
    mean = torch.empty(2, dtype=torch.float64, device="cuda")
    cv.cvrpsd_split_eval_tours(sp.ctx, tours, inst.dist, Dd, inst.Q, inst.L, mean=mean)
    torch.cuda.synchronize()
    return r, out.cpu().numpy(), bres, mean.cpu().numpy()


def test_every_allocation_failure_is_clean(cv):
    inst, S, D, want, wsum, winf = case()
    Dd = torch.from_numpy(D).cuda()
    rev = inst.tour[::-1].copy()
    rsum = oracle.split_costs(rev, inst.dist, D, inst.Q, inst.L, nthreads=8)[1]
    failures = 0
    for k in range(40):
        sp = cv.Splitter(0)
        cv.cvrpsd_debug_fail_alloc(sp.ctx, k)
        try:
            run_all(cv, sp, inst, S, Dd)
        except cv.CvrpsdError as e:
            assert e.code == cv._lib.ERR_NOMEM, str(e)
            failures += 1
        cv.cvrpsd_debug_fail_alloc(sp.ctx, -1)
        # the context recovers: everything runs and is exact
        r, got, bres, mean = run_all(cv, sp, inst, S, Dd)
        assert np.array_equal(got, want)
        assert (r.sum, r.infeasible) == (wsum, winf)
        assert (int(bres["sum"][0]), int(bres["infeasible"][0])) == (wsum, winf)
        assert mean[0] == pytest.approx(wsum / (S - winf), rel=1e-15)
        assert mean[1] == pytest.approx(rsum / (S - winf), rel=1e-15)
        sp.close()
    # the hook reached allocations on every path before the count ran out
    assert failures >= 30
