"""Route recovery on the GPU (cvrpsd_split_routes) against the CPU oracle's
predecessors (Eq. 1, smallest optimal p on ties), element by element."""
import numpy as np
import pytest

import oracle
from synth import demand_matrix, instance_from_coords, make_instance, workload

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


@pytest.fixture()
def sp(cv):
    s = cv.Splitter(0)
    yield s
    s.close()


def check_routes(sp, cv, inst, D, Q, L, sample=None):
    n, S = D.shape
    dD = torch.from_numpy(np.ascontiguousarray(D)).cuda()
    pred = torch.full((n, S), -9, dtype=torch.int16, device="cuda")
    out = torch.empty(S, dtype=torch.int32, device="cuda")
    r = sp.split_routes(inst.tour, inst.dist, dD, Q, L, pred=pred, out_cost=out)
    P = pred.cpu().numpy()
    costs = out.cpu().numpy()
    want, wsum, winf, _ = oracle.split_costs(inst.tour, inst.dist, D, Q, L)
    assert np.array_equal(costs, want) and (r.sum, r.infeasible) == (wsum, winf)
    cols = range(S) if sample is None else sample
    for s in cols:
        cost, routes, opred = oracle.split_routes(inst.tour, inst.dist, D[:, s], Q, L)
        if cost is None:
            continue
        assert np.array_equal(P[:, s], opred[1:]), f"scenario {s}"
        assert cv.routes_from_pred(inst.tour, P[:, s]) == routes
    return P


def test_routes_plain_n50(sp, cv):
    w = workload("plain-n50")
    inst = w.instances[0]
    D = demand_matrix(inst.mu, inst.region, w.kind, w.scen_seeds[0], w.S, dtype=w.dtype)
    check_routes(sp, cv, inst, D, inst.Q, inst.L)


def test_routes_corr_n200_capped(sp, cv):
    w = workload("corr-n200", S=3001)
    inst = w.instances[0]
    D = demand_matrix(inst.mu, inst.region, w.kind, w.scen_seeds[0], 3001, dtype=w.dtype)
    D[3, 17] = inst.Q + 5                          # an infeasible scenario
    check_routes(sp, cv, inst, D, inst.Q, inst.L, sample=range(0, 3001, 7))


def test_routes_ties_and_general_blocks(sp, cv):
    """Equal-cost splits everywhere (unit depot legs, free travel) and C_i = 0
    at every position: the smallest optimal predecessor must win."""
    n = 40
    dist = np.zeros((n + 1, n + 1), np.int32)
    dist[0, 1:] = 1
    dist[1:, 0] = 1
    inst = make_instance(n, 1, 10, seed=3, Q=12)
    inst.dist = dist
    rng = np.random.default_rng(5)
    D = rng.integers(0, 6, size=(n, 999)).astype(np.int16)
    check_routes(sp, cv, inst, D, 12, n)


def test_routes_set_aside_scenarios(sp, cv):
    n = 100
    coords = [[0, 0]] + [[3 * k, 4 * k] for k in range(1, n + 1)]
    inst = instance_from_coords(coords, list(range(1, n + 1)), Q=70)
    rng = np.random.default_rng(8)
    D = rng.integers(0, 2, size=(n, 600)).astype(np.int16)
    sp.configure(kernel=cv.KERNEL_DEQUE, threads=128, spt=1, ring=16)
    check_routes(sp, cv, inst, D, 70, n)
    assert sp.stats()["overflow"] > 0
