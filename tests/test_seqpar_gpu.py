"""GPU parity of the sequence-parallel Split (min-plus transfer matrices over
blocks of tour positions) against the CPU oracle, bit for bit."""
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
    s.configure(kernel=cv.KERNEL_SEQPAR)
    yield s
    s.close()


def parity(sp, inst, D, Q=None, L=None):
    Q = inst.Q if Q is None else Q
    L = inst.L if L is None else L
    want, ws, wi, _ = oracle.split_costs(inst.tour, inst.dist, D, Q, L, nthreads=8)
    out = torch.full((D.shape[1],), -5, dtype=torch.int32, device="cuda")
    r = sp.split(inst.tour, inst.dist, torch.from_numpy(np.ascontiguousarray(D)).cuda(), Q, L, out_cost=out)
    assert np.array_equal(out.cpu().numpy(), want)
    assert (r.sum, r.infeasible) == (ws, wi)
    return r


@pytest.mark.parametrize("name,S", [("plain-n50", 1000), ("corr-n200", 2000), ("million-n1000", 64)])
def test_seqpar_named(sp, cv, name, S):
    w = workload(name, S=S)
    inst = w.instances[0]
    D = demand_matrix(inst.mu, inst.region, w.kind, w.scen_seeds[0], S, dtype=w.dtype)
    parity(sp, inst, D)
    assert sp.stats()["kernel"] == cv.KERNEL_SEQPAR


def test_seqpar_single_scenario_and_n1(sp):
    w = workload("million-n1000", S=1)
    inst = w.instances[0]
    D = demand_matrix(inst.mu, inst.region, w.kind, w.scen_seeds[0], 1, dtype=w.dtype)
    parity(sp, inst, D)
    one = instance_from_coords([[0, 0], [3, 4]], [1], Q=5)
    parity(sp, one, np.array([[0, 5, 6, 2]], np.int16))


def test_seqpar_long_windows_infeasible_negative(sp, cv):
    n = 120                                   # windows up to 120 > 64: warp kernel
    coords = [[0, 0]] + [[3 * k, 4 * k] for k in range(1, n + 1)]
    ray = instance_from_coords(coords, list(range(1, n + 1)), Q=80)
    rng = np.random.default_rng(4)
    D = rng.integers(0, 2, size=(n, 333)).astype(np.int16)
    D[5, 9] = 81                              # infeasible
    r = parity(sp, ray, D, Q=80, L=n)
    assert sp.stats()["overflow"] > 0 and r.infeasible == 1
    inst = make_instance(30, 1, 10, seed=2, Q=20, L=7)
    D = np.ones((30, 50), np.int16)
    D[3, 4] = -1
    with pytest.raises(cv.CvrpsdError):
        sp.split(inst.tour, inst.dist, torch.from_numpy(D).cuda(), 20, 7)


def test_seqpar_rejects_large_S(sp, cv):
    inst = make_instance(10, 1, 10, seed=1, Q=20)
    D = torch.ones((10, 5000), dtype=torch.int16, device="cuda")
    with pytest.raises(cv.CvrpsdError) as e:
        sp.split(inst.tour, inst.dist, D, 20, 10)
    assert e.value.code == -7
