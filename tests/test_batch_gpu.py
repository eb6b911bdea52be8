"""GPU parity of the batched Split (one persistent launch in a CUDA graph)
against the CPU oracle, tour by tour, bit for bit."""
import numpy as np
import pytest

import oracle
from synth import (demand_matrix, demand_columns, instance_from_coords, make_instance,
                   workload)

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


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def mixed_tours(S, dtype=np.int16, capped=False):
    w = workload("batched-512", S=S, T=6)
    insts = list(w.instances) + [make_instance(1, 1, 10, seed=77, Q=12),
                                 make_instance(37, 5, 20, seed=78, Q=60, L=7 if capped else None)]
    seeds = list(w.scen_seeds) + [11, 12]
    mats = [demand_matrix(inst.mu, inst.region, w.kind, sd, S, dtype=dtype)
            for inst, sd in zip(insts, seeds)]
    return insts, mats


def run_batch(sp, insts, mats, S, reruns=1):
    outs = [torch.full((S,), -3, dtype=torch.int32, device="cuda") for _ in insts]
    tours = [dict(tour=i.tour, dist=i.dist, demand=dev(m), Q=i.Q, L=i.L, out_cost=o)
             for i, m, o in zip(insts, mats, outs)]
    b = sp.batch(tours, S)
    res = None
    for _ in range(reruns):
        b.run()
        res = b.results()
    return b, tours, outs, res


@pytest.mark.parametrize("capped", [False, True])
def test_batch_matches_oracle(sp, capped):
    S = 3001
    insts, mats = mixed_tours(S, capped=capped)
    mats[2][5, 100] = insts[2].Q + 1                     # one infeasible scenario
    b, tours, outs, res = run_batch(sp, insts, mats, S, reruns=2)
    for t, (inst, D) in enumerate(zip(insts, mats)):
        want, wsum, winf, _ = oracle.split_costs(inst.tour, inst.dist, D, inst.Q, inst.L, nthreads=8)
        assert np.array_equal(outs[t].cpu().numpy(), want), f"tour {t}"
        assert (res["sum"][t], res["infeasible"][t]) == (wsum, winf), f"tour {t}"
    assert res["tour_status"][2] == 1 and res["status"] == 1
    b.close()


def test_batch_graph_sees_new_demands(sp):
    S = 1000
    insts, mats = mixed_tours(S, dtype=np.int32)
    b, tours, outs, first = run_batch(sp, insts, mats, S)
    rng = np.random.default_rng(3)
    for t, inst in enumerate(insts):             # new scenarios, same tours
        new = rng.integers(0, max(1, inst.Q // 6), size=mats[t].shape).astype(np.int32)
        tours[t]["demand"].copy_(dev(new))
        mats[t] = new
    b.run()
    res = b.results()
    for t, inst in enumerate(insts):
        want, wsum, winf, _ = oracle.split_costs(inst.tour, inst.dist, mats[t], inst.Q, inst.L)
        assert np.array_equal(outs[t].cpu().numpy(), want)
        assert res["sum"][t] == wsum
    b.close()


def test_batch_set_aside_and_one_shot(sp, cv):
    """Ray instances make the deque hold the whole window, so many scenarios
    are set aside to the warp kernel; the one-shot entry agrees."""
    n, S = 90, 700
    coords = [[0, 0]] + [[3 * k, 4 * k] for k in range(1, n + 1)]
    ray = instance_from_coords(coords, list(range(1, n + 1)), Q=60)
    rng = np.random.default_rng(2)
    D = rng.integers(0, 2, size=(n, S)).astype(np.int16)
    other = make_instance(120, 1, 10, seed=5, Q=40)
    D2 = demand_matrix(other.mu, other.region, 1, 9, S, dtype=np.int16)
    want1, s1, i1, _ = oracle.split_costs(ray.tour, ray.dist, D, 60, n)
    want2, s2, i2, _ = oracle.split_costs(other.tour, other.dist, D2, other.Q, other.L)
    o1 = torch.empty(S, dtype=torch.int32, device="cuda")
    o2 = torch.empty(S, dtype=torch.int32, device="cuda")
    tours = [dict(tour=ray.tour, dist=ray.dist, demand=dev(D), Q=60, L=n, out_cost=o1),
             dict(tour=other.tour, dist=other.dist, demand=dev(D2), Q=other.Q, L=other.L, out_cost=o2)]
    res = sp.split_batch(tours, S)
    assert np.array_equal(o1.cpu().numpy(), want1) and np.array_equal(o2.cpu().numpy(), want2)
    assert list(res["sum"]) == [s1, s2] and list(res["infeasible"]) == [i1, i2]
    assert sp.stats()["overflow"] > 0


@pytest.mark.parametrize("capped", [False, True])
def test_batch_autotune(sp, cv, capped):
    """The batch autotuner times every batch shape, checks that each gives the
    same per-tour results, and leaves the fastest on the context; a batch
    created afterwards uses it and still matches the oracle."""
    S = 3000
    insts, mats = mixed_tours(S, capped=capped)
    tours = [dict(tour=i.tour, dist=i.dist, demand=dev(m), Q=i.Q, L=i.L) for i, m in zip(insts, mats)]
    r = sp.batch_autotune(tours, S)
    # scenarios per block 32..512 x rings 16 / 32 / 64: every compiled shape timed
    shapes = {(t, s, g) for t in (32, 64, 128, 256) for s in (1, 2) for g in (16, 32, 64)
              if not (t == 256 and g == 64) and not (t == 128 and s == 2 and g == 64)
              and not (t == 256 and s == 2 and g > 16)} | {(512, 1, 16)}
    assert len(shapes) == 21
    assert r["shapes_timed"] == 21 and r["ms"] > 0
    assert (r["threads"], r["spt"], r["ring"]) in shapes
    assert r["dtype"] in (cv.I16, cv.I32)
    b, tours, outs, res = run_batch(sp, insts, mats, S)
    st = sp.stats()
    assert (st["threads"], st["spt"], st["ring"]) == (r["threads"], r["spt"], r["ring"])
    for k, (inst, m) in enumerate(zip(insts, mats)):
        want, wsum, winf, _ = oracle.split_costs(inst.tour, inst.dist, m, inst.Q, inst.L, nthreads=8)
        assert (res["sum"][k], res["infeasible"][k]) == (wsum, winf)
        assert np.array_equal(outs[k].cpu().numpy(), want)
    b.close()


def test_batch_rejects_bad_tour(sp, cv):
    S = 64
    insts, mats = mixed_tours(S)
    tours = [dict(tour=i.tour, dist=i.dist, demand=dev(m), Q=i.Q, L=i.L) for i, m in zip(insts, mats)]
    tours[3]["tour"] = np.r_[insts[3].tour[:-1], insts[3].tour[0]]
    with pytest.raises(cv.CvrpsdError) as e:
        sp.batch(tours, S)
    assert "tour 3" in str(e.value)


def test_batched_512_sampled(sp, cv):
    """Full size: 512 tours, n ~ U{100..1000}, S = 65,536 each (about 37 GB of
    int16 demands), generated on the device; two 512-column blocks of five
    tours are overwritten with host-generated demands and compared with the
    oracle after one graph run."""
    w = workload("batched-512")
    S = w.S
    mats = []
    for inst, sd in zip(w.instances, w.scen_seeds):
        D = torch.empty((inst.n, S), dtype=torch.int16, device="cuda")
        sp.gen_demand(sd, cv.GEN_CORRELATED, inst.mu, inst.region, D)
        mats.append(D)
    outs = [torch.empty(S, dtype=torch.int32, device="cuda") for _ in w.instances]
    check = [0, 17, 255, 400, 511]
    blocks = [0, S - 512]
    host = {}
    for t in check:
        inst = w.instances[t]
        for a in blocks:
            cols = demand_columns(inst.mu, inst.region, w.kind, w.scen_seeds[t] + 7, np.arange(a, a + 512),
                                  np.int16)
            mats[t][:, a:a + 512] = dev(cols)
            host[t, a] = cols
    tours = [dict(tour=i.tour, dist=i.dist, demand=D, Q=i.Q, L=i.L, out_cost=o)
             for i, D, o in zip(w.instances, mats, outs)]
    b = sp.batch(tours, S)
    b.run()
    res = b.results()
    for t in check:
        inst = w.instances[t]
        got = outs[t].cpu().numpy()
        for a in blocks:
            want, _, _, _ = oracle.split_costs(inst.tour, inst.dist, host[t, a], inst.Q, inst.L, nthreads=8)
            assert np.array_equal(got[a:a + 512], want), f"tour {t} block {a}"
        feas = got != INT32_MAX
        assert res["sum"][t] == int(got[feas].astype(np.int64).sum())
        assert res["infeasible"][t] == int((~feas).sum())
    b.close()


def test_batch_autotune_dtype_arm_skips_int16_when_demands_do_not_fit(sp, cv):
    """The demand-storage arm times int16 and int32 copies of a sample; a
    demand beyond int16 (here in an int32 batch) leaves only int32."""
    S = 1000
    insts, mats = mixed_tours(S)
    mats32 = [m.astype(np.int32) for m in mats]
    mats32[2][5, 17] = 40_000                      # above int16; also above Q: infeasible there
    tours = [dict(tour=i.tour, dist=i.dist, demand=dev(m), Q=i.Q, L=i.L) for i, m in zip(insts, mats32)]
    r = sp.batch_autotune(tours, S)
    assert r["dtype"] == cv.I32 and r["shapes_timed"] == 21


@pytest.mark.parametrize("shape", [(64, 1, 16), (128, 1, 32), (256, 1, 16)])
def test_batch_second_walk_general_blocks_and_overflow(sp, cv, shape):
    """int16 demands with one scenario per thread run the batch on the second
    walk. Customers on a line through the depot, visited on alternating
    sides, make C_i = 0 at most positions (blocks of the emptying back walk);
    all-zero demand columns make the deque hold the whole window (ring
    overflow, set aside) unless the route-length cap L bounds it; a demand
    above Q makes a scenario infeasible. Every cost against the oracle."""
    n, S = 70, 2049
    coords = [[0, 0]] + [[(7 * ((k + 1) // 2)) * (1 if k % 2 else -1), 0] for k in range(1, n + 1)]
    line = instance_from_coords(coords, list(range(1, n + 1)), Q=50)
    sig = [0] + list(line.tour)
    C = [line.dist[sig[i], 0] + line.dist[0, sig[i + 1]] - line.dist[sig[i], sig[i + 1]] for i in range(1, n)]
    assert sum(c <= 0 for c in C) > n // 2
    rng = np.random.default_rng(8)
    D1 = rng.integers(0, 13, size=(n, S)).astype(np.int16)
    D1[:, :40] = 0                                  # whole-tour windows
    D1[9, 777] = 51                                 # above Q
    other = make_instance(150, 1, 10, seed=21, Q=45)
    D2 = demand_matrix(other.mu, other.region, 1, 4, S, dtype=np.int16)
    D2[:, 1000:1010] = 0
    cases = [(line, D1, n), (line, D1, 6), (other, D2, 9)]
    outs = [torch.empty(S, dtype=torch.int32, device="cuda") for _ in cases]
    tours = [dict(tour=i.tour, dist=i.dist, demand=dev(D), Q=i.Q, L=L, out_cost=o)
             for (i, D, L), o in zip(cases, outs)]
    sp.configure(kernel=cv.KERNEL_DEQUE, threads=shape[0], spt=shape[1], ring=shape[2])
    res = sp.split_batch(tours, S)
    for t, ((inst, D, L), o) in enumerate(zip(cases, outs)):
        want, wsum, winf, _ = oracle.split_costs(inst.tour, inst.dist, D, inst.Q, L, nthreads=8)
        assert np.array_equal(o.cpu().numpy(), want), f"tour {t}"
        assert (res["sum"][t], res["infeasible"][t]) == (wsum, winf), f"tour {t}"
    assert res["infeasible"][0] >= 1 and sp.stats()["overflow"] > 0
