"""GPU parity of the CUDA Split (through the C ABI) against the CPU oracle.

Every comparison is element by element and bit-exact: costs are integers.
Inputs come from the seeded host generators in synth/ and are copied to the
device; the oracle never sees anything the CUDA path produced."""
import dataclasses
import functools

import numpy as np
import pytest

import oracle
from synth import (make_instance, instance_from_coords, demand_matrix, demand_columns,
                   workload)

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

INT32_MAX = 2**31 - 1
SHAPES = [(t, s, r) for t in (64, 128, 256) for s in (1, 2) for r in (16, 32, 64)]
# parameter-table walk: (threads, ring, rounds)
PARAM_SHAPES = [(t, r, k) for t in (64, 128, 256) for r in (8, 16) for k in (0, 1, 3)]


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


def to_dev(D):
    return torch.from_numpy(np.ascontiguousarray(D)).cuda()


def run(sp, inst, D_dev, Q=None, L=None, S=None):
    S = D_dev.shape[1] if S is None else S
    out = torch.full((max(S, 1),), -7, dtype=torch.int32, device="cuda")
    r = sp.split(inst.tour, inst.dist, D_dev, inst.Q if Q is None else Q,
                 inst.L if L is None else L, S=S, out_cost=out)
    return r, out[:S].cpu().numpy()


def check_parity(sp, inst, D, Q=None, L=None, nthreads=8):
    Q = inst.Q if Q is None else Q
    L = inst.L if L is None else L
    want, wsum, winf, _ = oracle.split_costs(inst.tour, inst.dist, D, Q, L, nthreads=nthreads)
    r, got = run(sp, inst, to_dev(D), Q, L)
    assert np.array_equal(got, want), f"{int((got != want).sum())} scenarios differ"
    assert (r.sum, r.infeasible) == (wsum, winf)
    return r, got


# ------------------------------------------------------------ named workloads

@pytest.mark.parametrize("kernel", ["deque", "warp"])
def test_plain_n50_full(sp, cv, kernel):
    w = workload("plain-n50")
    inst = w.instances[0]
    D = demand_matrix(inst.mu, inst.region, w.kind, w.scen_seeds[0], w.S, dtype=w.dtype)
    if kernel == "warp":
        sp.configure(kernel=cv.KERNEL_WARP)
    r, got = check_parity(sp, inst, D)
    assert sp.stats()["kernel"] == (cv.KERNEL_WARP if kernel == "warp" else cv.KERNEL_DEQUE)
    assert r.mean == pytest.approx(r.sum / (w.S - r.infeasible))


def test_corr_n200_full(sp):
    w = workload("corr-n200")
    inst = w.instances[0]
    D = demand_matrix(inst.mu, inst.region, w.kind, w.scen_seeds[0], w.S, dtype=w.dtype)
    check_parity(sp, inst, D)


def test_million_n1000_sampled(sp, cv):
    """Full size, default launch: the device generator fills 2^20 scenarios,
    four column blocks are overwritten with host-generated demands, and the
    Split of those blocks is compared with the oracle."""
    w = workload("million-n1000")
    inst = w.instances[0]
    S = w.S
    D = torch.empty((inst.n, S), dtype=torch.int16, device="cuda")
    sp.gen_demand(w.scen_seeds[0], cv.GEN_CORRELATED, inst.mu, inst.region, D)
    blk = 2048
    starts = [0, 123_456, 777_777, S - blk]
    host = {}
    for a in starts:
        cols = demand_columns(inst.mu, inst.region, w.kind, w.scen_seeds[0] + 1,
                              np.arange(a, a + blk), np.int16)
        host[a] = cols
        D[:, a:a + blk] = to_dev(cols)
    out = torch.empty(S, dtype=torch.int32, device="cuda")
    r = sp.split(inst.tour, inst.dist, D, inst.Q, inst.L, out_cost=out)
    got = out.cpu().numpy()
    for a in starts:
        want, _, _, _ = oracle.split_costs(inst.tour, inst.dist, host[a], inst.Q, inst.L, nthreads=8)
        assert np.array_equal(got[a:a + blk], want)
    feas = got != INT32_MAX
    assert r.sum == int(got[feas].astype(np.int64).sum())
    assert r.infeasible == int((~feas).sum())


# ------------------------------------------------------------- launch shapes

@pytest.mark.parametrize("shape", SHAPES, ids=lambda s: f"t{s[0]}_spt{s[1]}_r{s[2]}")
def test_every_shape_int16(sp, cv, shape):
    """Global-table walk, every shape."""
    w = workload("corr-n200", S=4099)            # ragged: not a multiple of any block
    inst = w.instances[0]
    D = demand_matrix(inst.mu, inst.region, w.kind, w.scen_seeds[0], 4099, dtype=np.int16)
    sp.configure(kernel=cv.KERNEL_DEQUE, threads=shape[0], spt=shape[1], ring=shape[2],
                 variant=cv.WALK_GLOBAL_TABLE)
    check_parity(sp, inst, D)
    assert sp.stats()["variant"] == cv.WALK_GLOBAL_TABLE


@pytest.mark.parametrize("shape", PARAM_SHAPES, ids=lambda s: f"t{s[0]}_r{s[1]}_rounds{s[2]}")
def test_every_param_walk_shape_int16(sp, cv, shape):
    """Parameter-table walk, every compiled shape, one scenario per thread or
    several rounds of tiles per block (ragged S: the last round is partial)."""
    w = workload("corr-n200", S=4099)
    inst = w.instances[0]
    D = demand_matrix(inst.mu, inst.region, w.kind, w.scen_seeds[0], 4099, dtype=np.int16)
    t, r, k = shape
    sp.configure(kernel=cv.KERNEL_DEQUE, threads=t, spt=1, ring=r, variant=cv.WALK_PARAM_TABLE, rounds=k)
    check_parity(sp, inst, D)
    st = sp.stats()
    assert (st["variant"], st["threads"], st["ring"], st["rounds"]) == (cv.WALK_PARAM_TABLE, t, r, k)


@pytest.mark.parametrize("walk", ["global", "param"])
@pytest.mark.parametrize("shape", [(128, 2, 16), (256, 2, 32), (64, 1, 64), (128, 1, 16)])
def test_shapes_int32_uncapped(sp, cv, shape, walk):
    w = workload("plain-n50", S=3001)
    inst = w.instances[0]
    D = demand_matrix(inst.mu, inst.region, w.kind, w.scen_seeds[0], 3001, dtype=np.int32)
    v = cv.WALK_GLOBAL_TABLE if walk == "global" else cv.WALK_PARAM_TABLE
    sp.configure(kernel=cv.KERNEL_DEQUE, threads=shape[0], spt=shape[1], ring=shape[2], variant=v, rounds=2)
    check_parity(sp, inst, D)
    assert sp.stats()["variant"] == v


@pytest.mark.parametrize("n, Q, L, dtype", [
    (1025, 200, 60, np.int16),      # larger parameter table (n > 1024)
    (4032, 150, 40, np.int16),      # the largest tour the parameter table holds
    (1000, 2100, 1000, np.int16),   # keys that wrap: the difference test
    (300, 40_000, 300, np.int32),   # int32 demands, keys that wrap
    (300, 400, 20, np.int32),       # int32 demands, keys that fit
])
def test_param_walk_key_ranges_and_tables(sp, cv, n, Q, L, dtype):
    inst = make_instance(n, 1, 30, seed=n + Q, Q=Q, L=L)
    scale = max(1, Q // 200)
    D = demand_matrix(inst.mu, inst.region, 1, n * 7 + 1, 1537, dtype=dtype)
    if scale > 1:
        D = (D.astype(np.int64) * scale).astype(dtype)
    D[3, 100] = Q + 1                     # one infeasible scenario
    sp.configure(kernel=cv.KERNEL_DEQUE, threads=128, spt=1, ring=16, variant=cv.WALK_PARAM_TABLE)
    r, _ = check_parity(sp, inst, D)
    assert sp.stats()["variant"] == cv.WALK_PARAM_TABLE
    assert r.infeasible >= 1


def test_param_walk_negative_and_too_large_int16(sp, cv):
    """int16 demands read as unsigned: a negative one (>= 32768 as unsigned)
    and one above Q both reach the back of the deque and freeze the walk;
    the warp kernel classifies them (negative: an error; above Q: infeasible)."""
    inst = make_instance(90, 1, 10, seed=5, Q=40, L=15)
    D = demand_matrix(inst.mu, inst.region, 1, 9, 700, dtype=np.int16)
    D[17, 3] = 41
    D[0, 650] = 32767
    sp.configure(kernel=cv.KERNEL_DEQUE, threads=64, spt=1, ring=8, variant=cv.WALK_PARAM_TABLE, rounds=2)
    r, got = check_parity(sp, inst, D)
    assert got[3] == INT32_MAX and got[650] == INT32_MAX and r.infeasible == 2
    D[5, 200] = -1
    with pytest.raises(cv.CvrpsdError) as e:
        run(sp, inst, to_dev(D))
    assert e.value.code == -5


# ----------------------------------------------------------------- edge cases

def test_padded_pitch_and_subset(sp):
    inst = make_instance(37, 1, 10, seed=3, Q=25, L=9)
    D = demand_matrix(inst.mu, inst.region, 1, 77, 1000, dtype=np.int16)
    buf = torch.zeros((37, 1024), dtype=torch.int16, device="cuda")
    buf[:, :1000] = to_dev(D)
    want, wsum, winf, _ = oracle.split_costs(inst.tour, inst.dist, D[:, :999], inst.Q, inst.L)
    out = torch.empty(999, dtype=torch.int32, device="cuda")
    r = sp.split(inst.tour, inst.dist, buf, inst.Q, inst.L, S=999, out_cost=out)
    assert np.array_equal(out.cpu().numpy(), want) and r.sum == wsum


def test_empty_and_single(sp):
    inst = make_instance(10, 1, 10, seed=1, Q=20)
    D = to_dev(np.ones((10, 4), np.int16))
    r = sp.split(inst.tour, inst.dist, D, 20, 10, S=0)
    assert (r.sum, r.infeasible) == (0, 0) and np.isnan(r.mean)
    check_parity(sp, inst, np.ones((10, 1), np.int16))


def test_n1_and_L1(sp):
    inst = instance_from_coords([[0, 0], [3, 4]], [1], Q=5)
    r, got = check_parity(sp, inst, np.array([[0, 5, 6, 2]], np.int16))
    assert got.tolist() == [10, 10, INT32_MAX, 10]
    inst = make_instance(30, 1, 10, seed=5, Q=50, L=1)
    D = demand_matrix(inst.mu, inst.region, 0, 5, 300, dtype=np.int32)
    check_parity(sp, inst, D, L=1)


def test_zero_capacity_and_zero_demand(sp):
    inst = make_instance(25, 1, 10, seed=6, Q=0)
    D = np.zeros((25, 200), np.int16)
    D[3, ::7] = 1                                # those scenarios become infeasible
    r, got = check_parity(sp, inst, D, Q=0)
    assert r.infeasible == len(range(0, 200, 7))


def test_all_infeasible(sp):
    inst = make_instance(12, 1, 10, seed=2, Q=5)
    D = np.full((12, 64), 6, np.int16)
    r, got = check_parity(sp, inst, D)
    assert r.infeasible == 64 and np.isnan(r.mean) and (got == INT32_MAX).all()
    assert r.status == 1


@functools.lru_cache(maxsize=1)
def largest_case(n):
    inst = make_instance(n, 5, 30, seed=31, Q=150)
    return inst, demand_matrix(inst.mu, inst.region, 1, 17, 640, dtype=np.int16)


@pytest.mark.parametrize("kernel, L", [("deque", None), ("deque", 40), ("warp", 40), ("seqpar", None)])
def test_largest_tour(sp, cv, kernel, L):
    """n = CVRPSD_MAX_N customers: every kernel at the library's size limit
    (the table, the key scale, the warp kernel's per-warp prefix loads and
    the sequence-parallel matrices all at their largest)."""
    inst0, D0 = largest_case(cv.MAX_N)
    inst = inst0 if L is None else dataclasses.replace(inst0, L=L)
    D = D0[:, :64] if kernel == "seqpar" else D0
    code = {"deque": cv.KERNEL_DEQUE, "warp": cv.KERNEL_WARP, "seqpar": cv.KERNEL_SEQPAR}[kernel]
    sp.configure(kernel=code)
    check_parity(sp, inst, D)
    assert sp.stats()["kernel"] == code


def test_deque_overflow_goes_to_warp_kernel(sp, cv):
    """Customers on a ray from the depot make g strictly increasing along the
    window, so with unit demands and a large capacity the deque holds the
    whole window and overflows a 16-entry ring."""
    n = 120
    coords = [[0, 0]] + [[3 * k, 4 * k] for k in range(1, n + 1)]
    inst = instance_from_coords(coords, list(range(1, n + 1)), Q=80)
    rng = np.random.default_rng(4)
    D = rng.integers(0, 2, size=(n, 777)).astype(np.int16)
    sp.configure(kernel=cv.KERNEL_DEQUE, threads=128, spt=1, ring=16)
    check_parity(sp, inst, D, Q=80, L=n)
    st = sp.stats()
    assert st["overflow"] > 0 and st["launches"] == 2


def test_large_int32_demands(sp):
    inst = make_instance(60, 1, 10, seed=8, Q=1_000_000)
    rng = np.random.default_rng(1)
    D = rng.integers(0, 400_000, size=(60, 513)).astype(np.int32)
    D[7, 5] = 2_000_000_000                       # far above Q
    r, got = check_parity(sp, inst, D)
    assert got[5] == INT32_MAX


def test_asymmetric_distances(sp):
    rng = np.random.default_rng(9)
    n = 40
    dist = rng.integers(0, 500, size=(n + 1, n + 1)).astype(np.int32)
    inst = make_instance(n, 1, 10, seed=1, Q=30, L=7)
    inst.dist = dist
    D = rng.integers(0, 10, size=(n, 999)).astype(np.int16)
    check_parity(sp, inst, D)


# --------------------------------------------------------------- bad inputs

def test_negative_demand_is_reported(sp, cv):
    inst = make_instance(20, 1, 10, seed=1, Q=30)
    D = np.ones((20, 100), np.int16)
    D[4, 17] = -3
    with pytest.raises(cv.CvrpsdError) as e:
        run(sp, inst, to_dev(D))
    assert e.value.code == -5


def test_negative_demand_found_by_a_call_that_did_not_wait(sp, cv):
    """Without host outputs the call returns before its kernels run; the
    negative demand is then reported by cvrpsd_check_inputs, once."""
    inst = make_instance(20, 1, 10, seed=1, Q=30)
    try:                                                # start from a clear record (earlier
        sp.check_inputs()                               # tests on this context fed it bad input)
    except cv.CvrpsdError:
        pass
    D = np.ones((20, 100), np.int16)
    clean = to_dev(D)
    out = torch.zeros(100, dtype=torch.int32, device="cuda")
    sp.split(inst.tour, inst.dist, clean, 30, 20, out_cost=out, host_outputs=False)
    sp.check_inputs()                                   # nothing to report
    D[4, 17] = -3
    bad = to_dev(D)
    sp.split(inst.tour, inst.dist, bad, 30, 20, out_cost=out, host_outputs=False)
    sp.split(inst.tour, inst.dist, clean, 30, 20, host_outputs=False)   # a later clean call keeps the record
    with pytest.raises(cv.CvrpsdError) as e:
        sp.check_inputs()
    assert e.value.code == -5
    D[4, 17] = 0                                        # the kernels read a negative demand as zero
    ref = torch.zeros(100, dtype=torch.int32, device="cuda")
    sp.split(inst.tour, inst.dist, to_dev(D), 30, 20, out_cost=ref)
    assert torch.equal(out, ref)
    sp.check_inputs()                                   # the record was cleared


def test_log_callback(sp, cv):
    """Messages go to the caller's function only: the detail of a failing
    call (error level) and, at debug level, what each Split ran."""
    msgs = []
    sp.set_log(lambda level, text: msgs.append((level, text)), max_level=cv._lib.LOG_DEBUG)
    inst = make_instance(20, 1, 10, seed=1, Q=30)
    D = to_dev(np.ones((20, 100), np.int16))
    sp.split(inst.tour, inst.dist, D, 30, 20)
    assert any(lvl == cv._lib.LOG_DEBUG and "split n=20 S=100" in t for lvl, t in msgs)
    with pytest.raises(cv.CvrpsdError):
        sp.split(inst.tour, inst.dist, D, 30, 0)
    assert any(lvl == cv._lib.LOG_ERROR and "L = 0" in t for lvl, t in msgs)
    msgs.clear()
    sp.set_log(lambda level, text: msgs.append((level, text)), max_level=cv._lib.LOG_ERROR)
    sp.split(inst.tour, inst.dist, D, 30, 20)
    assert msgs == []                                   # debug messages filtered out
    sp.set_log(None)
    with pytest.raises(cv.CvrpsdError):
        sp.split(inst.tour, inst.dist, D, 30, 0)
    assert msgs == []                                   # logging off


def test_argument_errors(sp, cv):
    inst = make_instance(20, 1, 10, seed=1, Q=30)
    D = to_dev(np.ones((20, 100), np.int16))
    bad = [
        dict(tour=np.r_[inst.tour[:-1], inst.tour[0]]),          # not a permutation
        dict(L=0), dict(Q=-1),
        dict(demand=torch.ones((20, 100), dtype=torch.int16)),   # host tensor
        dict(S=101),                                             # ld < S
        dict(demand=torch.ones((20, 100), dtype=torch.int64, device="cuda")),
    ]
    for kw in bad:
        args = dict(tour=inst.tour, dist=inst.dist, demand=D, Q=30, L=20)
        extra = {}
        if "S" in kw:
            extra["S"] = kw.pop("S")
        args.update(kw)
        with pytest.raises(cv.CvrpsdError):
            sp.split(args["tour"], args["dist"], args["demand"], args["Q"], args["L"], **extra)
    # a host address passed as a device buffer is refused before any launch
    host_out = np.zeros(100, np.int32)
    with pytest.raises(cv.CvrpsdError) as e:
        sp.split(inst.tour, inst.dist, D.data_ptr(), 30, 20, S=100, ld=100, dtype=cv.I16,
                 out_cost=host_out.ctypes.data)
    assert e.value.code == -1


# ------------------------------------------------------------ generator

@pytest.mark.parametrize("kind,dtype", [(0, np.int32), (1, np.int16), (1, np.int32)])
def test_device_generator_matches_host_recipe(sp, cv, kind, dtype):
    inst = make_instance(300, 1, 30, seed=12, Q=200)
    S = 20_000
    tdt = torch.int16 if dtype == np.int16 else torch.int32
    D = torch.empty((inst.n, S), dtype=tdt, device="cuda")
    seed = 0xDEADBEEF12345
    sp.gen_demand(seed, kind, inst.mu, inst.region, D)
    got = D.cpu().numpy()
    want = demand_matrix(inst.mu, inst.region, kind, seed, S, dtype=dtype)
    diff = got.astype(np.int64) - want
    # float64 log/cos/exp of two math libraries may differ by an ulp, which
    # can only move a value across a rounding boundary: rare, and by 1
    assert np.abs(diff).max() <= 1
    assert (diff != 0).mean() < 1e-5


# ------------------------------------------------------------ autotuner

def test_autotune_picks_and_caches(sp, cv, tmp_path):
    import json
    w = workload("corr-n200", S=20_000)
    inst = w.instances[0]
    D = demand_matrix(inst.mu, inst.region, w.kind, w.scen_seeds[0], 20_000, dtype=np.int16)
    dD = to_dev(D)
    cache = tmp_path / "tune.jsonl"
    r1 = sp.autotune(inst.tour, inst.dist, dD, inst.Q, inst.L, cache_path=cache)
    assert r1["shapes_timed"] >= 12 and r1["ms"] > 0
    assert r1["dtype"] in (cv.I16, cv.I32)
    cfg = cv.cvrpsd_get_config(sp.ctx)
    assert (cfg["threads"], cfg["spt"], cfg["ring"]) == (r1["threads"], r1["spt"], r1["ring"])
    check_parity(sp, inst, D)                      # the tuned shape is still exact
    lines = [json.loads(l) for l in open(cache)]
    assert len(lines) == 1 and lines[0]["threads"] == r1["threads"]
    sp.configure(kernel=0)
    r2 = sp.autotune(inst.tour, inst.dist, dD, inst.Q, inst.L, cache_path=cache)
    assert r2["shapes_timed"] == 0
    assert (r2["threads"], r2["spt"], r2["ring"]) == (r1["threads"], r1["spt"], r1["ring"])


def test_zero_break_costs_take_the_general_step(sp, cv):
    """Customers alternate on both sides of the depot along one line, so the
    depot lies on every tour edge and C_i = c(a,0) + c(0,b) - c(a,b) = 0:
    every block is flagged and a new entry may empty the deque."""
    n = 61
    coords = [[0, 0]] + [[3 * k, 4 * k] if k % 2 else [-3 * k, -4 * k] for k in range(1, n + 1)]
    inst = instance_from_coords(coords, list(range(1, n + 1)), Q=25, L=9)
    rng = np.random.default_rng(11)
    D = rng.integers(0, 7, size=(n, 2053)).astype(np.int16)
    for shape, v in [((256, 1, 16), cv.WALK_GLOBAL_TABLE), ((128, 2, 32), cv.WALK_GLOBAL_TABLE),
                     ((256, 1, 16), cv.WALK_PARAM_TABLE), ((128, 1, 8), cv.WALK_PARAM_TABLE)]:
        sp.configure(kernel=cv.KERNEL_DEQUE, threads=shape[0], spt=shape[1], ring=shape[2], variant=v)
        check_parity(sp, inst, D)
        assert sp.stats()["variant"] == v


def test_overflow_then_back_pops_stay_bounded(sp, cv):
    """The deque grows past its ring along a ray (C_i > 0, increasing g),
    then a customer next to the depot forces back pops: the overflowed
    scenario must be set aside (and recomputed), not walked on a ring whose
    slots were overwritten."""
    coords = [[0, 0]] + [[3 * k, 4 * k] for k in range(1, 31)] + [[1, 0]] + \
        [[3 * k, 4 * k] for k in range(31, 40)]
    n = len(coords) - 1
    inst = instance_from_coords(coords, list(range(1, n + 1)), Q=1000)
    D = np.ones((n, 300), np.int16)
    D[:, 150:] = 2
    for shape, v in [((256, 1, 16), cv.WALK_GLOBAL_TABLE), ((128, 2, 16), cv.WALK_GLOBAL_TABLE),
                     ((64, 1, 32), cv.WALK_GLOBAL_TABLE), ((256, 1, 16), cv.WALK_PARAM_TABLE),
                     ((64, 1, 8), cv.WALK_PARAM_TABLE)]:
        sp.configure(kernel=cv.KERNEL_DEQUE, threads=shape[0], spt=shape[1], ring=shape[2], variant=v)
        check_parity(sp, inst, D, Q=1000, L=n)
        # the ray's deque peaks near 31 entries: it overflows rings of 8 or 16 only
        assert sp.stats()["variant"] == v
        assert (sp.stats()["overflow"] > 0) == (shape[2] <= 16)


def test_512_threads_is_batch_only(sp, cv):
    """threads = 512 is a batched-path shape: a single-tour call configured
    with it runs 256 threads (the nearest shape that applies) and still
    matches the oracle."""
    w = workload("corr-n200", S=1500)
    inst = w.instances[0]
    D = demand_matrix(inst.mu, inst.region, w.kind, w.scen_seeds[0], 1500, dtype=np.int16)
    sp.configure(kernel=cv.KERNEL_DEQUE, threads=512, spt=1, ring=16)
    check_parity(sp, inst, D)
    assert sp.stats()["threads"] == 256
