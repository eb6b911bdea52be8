"""The checked build of the library (-DCVRPSD_CHECKED=1): every index a Split
kernel forms from data is compared with its buffer before use, and a bad one
is reported as CVRPSD_ERR_DEVICE_STATUS instead of being used (nothing
traps). On valid inputs the checked build must give exactly the oracle's
results and report nothing: both walks, the warp kernel's set-aside pass,
ragged S, and the batched path."""
import ctypes

import numpy as np
import pytest

import oracle
from synth import demand_matrix, instance_from_coords, make_instance, workload

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def lib():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2511_18022_gb300 import _lib, build
    return _lib.load(build.build_checked())


@pytest.fixture()
def ctx(lib):
    h = ctypes.c_void_p()
    assert lib.cvrpsd_create(ctypes.byref(h), 0) == 0
    yield h
    lib.cvrpsd_destroy(h)


def split(lib, ctx, inst, D, Q, L, cfg):
    from paper_2511_18022_gb300 import _lib
    assert lib.cvrpsd_set_config(ctx, ctypes.byref(_lib.Config(*cfg))) == 0
    Dd = torch.from_numpy(np.ascontiguousarray(D)).cuda()
    S = D.shape[1]
    out = torch.full((S,), -9, dtype=torch.int32, device="cuda")
    tour = np.ascontiguousarray(inst.tour, np.int32)
    dist = np.ascontiguousarray(inst.dist, np.int32)
    s64, i64, mean = ctypes.c_int64(), ctypes.c_int64(), ctypes.c_double()
    code = 2 if D.dtype == np.int16 else 4
    rc = lib.cvrpsd_split_eval(ctx, tour.ctypes.data, len(tour), dist.ctypes.data, Dd.data_ptr(), code, S, S, Q, L,
                               out.data_ptr(), ctypes.byref(s64), ctypes.byref(i64), ctypes.byref(mean),
                               torch.cuda.current_stream().cuda_stream)
    return rc, out.cpu().numpy(), s64.value, i64.value


CFGS = [(1, 128, 1, 16, 1, 0), (1, 128, 2, 16, 1, 0), (1, 256, 1, 8, 2, 0), (1, 128, 1, 16, 2, 3)]


@pytest.mark.parametrize("cfg", CFGS, ids=["walk1", "walk1_spt2", "walk2_r8", "walk2_rounds"])
def test_checked_build_is_exact_and_silent(lib, ctx, cfg):
    w = workload("corr-n200", S=3001)
    inst = w.instances[0]
    D = demand_matrix(inst.mu, inst.region, w.kind, w.scen_seeds[0], 3001, dtype=np.int16)
    D[9, 100] = inst.Q + 1                          # infeasible: through the warp kernel
    want, wsum, winf, _ = oracle.split_costs(inst.tour, inst.dist, D, inst.Q, inst.L, nthreads=8)
    rc, got, s, i = split(lib, ctx, inst, D, inst.Q, inst.L, cfg)
    assert rc == 1 and (s, i) == (wsum, winf)       # CVRPSD_WARN_INFEASIBLE, no index error
    assert np.array_equal(got, want)


def test_checked_build_ring_overflow_and_int32(lib, ctx):
    n = 90
    coords = [[0, 0]] + [[3 * k, 4 * k] for k in range(1, n + 1)]
    inst = instance_from_coords(coords, list(range(1, n + 1)), Q=80)
    D = np.random.default_rng(4).integers(0, 2, size=(n, 513)).astype(np.int32)
    want, wsum, winf, _ = oracle.split_costs(inst.tour, inst.dist, D, 80, n)
    for cfg in [(1, 128, 1, 16, 1, 0), (1, 128, 1, 16, 2, 0)]:
        rc, got, s, i = split(lib, ctx, inst, D, 80, n, cfg)
        assert rc == 0 and np.array_equal(got, want) and (s, i) == (wsum, winf)


def test_checked_build_batch(lib, ctx):
    from paper_2511_18022_gb300 import _lib
    S = 777
    insts = [make_instance(n, 1, 10, seed=n, Q=30, L=12) for n in (1, 40, 130)]
    mats = [demand_matrix(i.mu, i.region, 0, 3 + k, S, dtype=np.int16) for k, i in enumerate(insts)]
    keep = []
    descs = (_lib.TourDesc * len(insts))()
    for k, (inst, D) in enumerate(zip(insts, mats)):
        tour = np.ascontiguousarray(inst.tour, np.int32)
        dist = np.ascontiguousarray(inst.dist, np.int32)
        Dd = torch.from_numpy(D).cuda()
        keep += [tour, dist, Dd]
        descs[k] = _lib.TourDesc(tour.ctypes.data, inst.n, dist.ctypes.data, Dd.data_ptr(), S, inst.Q, inst.L, None)
    sums = np.zeros(3, np.int64)
    infs = np.zeros(3, np.int64)
    rc = lib.cvrpsd_split_eval_batch(ctx, 3, descs, S, 2, sums.ctypes.data, infs.ctypes.data, None, None,
                                     torch.cuda.current_stream().cuda_stream)
    assert rc >= 0
    for k, (inst, D) in enumerate(zip(insts, mats)):
        _, ws, wi, _ = oracle.split_costs(inst.tour, inst.dist, D, inst.Q, inst.L)
        assert (sums[k], infs[k]) == (ws, wi)
