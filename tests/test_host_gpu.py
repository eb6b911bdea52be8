"""GPU parity of the host-buffer Split entry point (cvrpsd_split_eval_host):
the scenario matrix and the cost vector stay in page-locked host memory and
the kernels read and write them in place. Results must equal the oracle's
and the device entry point's bit for bit."""
import numpy as np
import pytest

import oracle
from synth import KIND_NORMAL, demand_matrix, make_instance, workload

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


@pytest.fixture()
def sp(cv):
    s = cv.Splitter(0)
    yield s
    s.close()


def mk(n, seed, Q):
    return make_instance(n, 5, 30, seed, Q=Q)


def dm(inst, S, seed, dtype=np.int16):
    return demand_matrix(inst.mu, inst.region, KIND_NORMAL, seed, S, dtype=dtype)


def pinned(a):
    return torch.from_numpy(np.ascontiguousarray(a)).pin_memory()


@pytest.mark.parametrize("name", ["plain-n50", "corr-n200"])
def test_host_matches_oracle(sp, name):
    w = workload(name, S=3000)
    inst = w.instances[0]
    D = demand_matrix(inst.mu, inst.region, w.kind, w.scen_seeds[0], w.S, dtype=w.dtype)
    want, wsum, winf, _ = oracle.split_costs(inst.tour, inst.dist, D, inst.Q, inst.L, nthreads=8)
    Dh = pinned(D)
    out = torch.full((D.shape[1],), -7, dtype=torch.int32).pin_memory()
    r = sp.split_host(inst.tour, inst.dist, Dh, inst.Q, inst.L, out_cost=out)
    assert np.array_equal(out.numpy(), want)
    assert (r.sum, r.infeasible) == (wsum, winf)


@pytest.mark.parametrize("kernel", ["deque", "warp", "seqpar"])
def test_host_equals_device_every_kernel(sp, cv, kernel):
    inst = mk(300, 11, 150)
    S = 64 if kernel == "seqpar" else 2500
    D = dm(inst, S, 5)
    code = {"deque": cv.KERNEL_DEQUE, "warp": cv.KERNEL_WARP, "seqpar": cv.KERNEL_SEQPAR}[kernel]
    sp.configure(kernel=code)
    dev_out = torch.empty(S, dtype=torch.int32, device="cuda")
    rd = sp.split(inst.tour, inst.dist, torch.from_numpy(D).cuda(), inst.Q, inst.L, out_cost=dev_out)
    host_out = torch.empty(S, dtype=torch.int32).pin_memory()
    rh = sp.split_host(inst.tour, inst.dist, pinned(D), inst.Q, inst.L, out_cost=host_out)
    assert np.array_equal(host_out.numpy(), dev_out.cpu().numpy())
    assert (rh.sum, rh.infeasible) == (rd.sum, rd.infeasible)


def test_host_ragged_subset_and_int32(sp):
    """S < ld (a column prefix of a wider matrix), int32 demands, no cost output."""
    inst = mk(120, 3, 90)
    D = dm(inst, 777, 9, np.int32)
    S = 501
    want, wsum, winf, _ = oracle.split_costs(inst.tour, inst.dist, D[:, :S], inst.Q, inst.L, nthreads=8)
    r = sp.split_host(inst.tour, inst.dist, pinned(D), inst.Q, inst.L, S=S)
    assert (r.sum, r.infeasible) == (wsum, winf)


def test_host_rejects_pageable_and_device_buffers(sp, cv):
    inst = mk(40, 1, 60)
    D = dm(inst, 64, 2)
    with pytest.raises(cv.CvrpsdError):
        sp.split_host(inst.tour, inst.dist, torch.from_numpy(D), inst.Q, inst.L)          # pageable
    with pytest.raises(cv.CvrpsdError):
        sp.split_host(inst.tour, inst.dist, torch.from_numpy(D).cuda(), inst.Q, inst.L)   # device
    # the C entry point itself refuses pageable memory (no kernel is launched)
    from paper_2511_18022_gb300 import _lib
    import ctypes
    lib = _lib.load()
    tour = np.ascontiguousarray(inst.tour, np.int32)
    dist = np.ascontiguousarray(inst.dist, np.int32)
    Dp = np.ascontiguousarray(D)
    rc = lib.cvrpsd_split_eval_host(sp.ctx, tour.ctypes.data, inst.n, dist.ctypes.data, Dp.ctypes.data, cv.I16,
                                    64, 64, inst.Q, inst.L, None, None, None, None,
                                    torch.cuda.current_stream().cuda_stream)
    assert rc == _lib.ERR_ARG
    assert b"page-locked" in lib.cvrpsd_last_error(sp.ctx)


def test_host_empty(sp):
    inst = mk(30, 4, 50)
    D = np.zeros((inst.n, 8), np.int16)
    r = sp.split_host(inst.tour, inst.dist, pinned(D), inst.Q, inst.L, S=0)
    assert (r.sum, r.infeasible) == (0, 0)


def _range_reported(ptr):
    """Whether the driver reports the allocation range of a host pointer."""
    import ctypes
    try:
        cu = ctypes.CDLL("libcuda.so.1")
    except OSError:
        return False
    base, size = ctypes.c_uint64(0), ctypes.c_size_t(0)
    return cu.cuMemGetAddressRange_v2(ctypes.byref(base), ctypes.byref(size), ctypes.c_uint64(ptr)) == 0


def test_host_rejects_short_buffer(sp, cv):
    """A pitch that runs past the page-locked allocation is refused before any
    launch (checked only where the driver reports the allocation's range)."""
    inst = mk(40, 1, 60)
    Dh = pinned(dm(inst, 64, 2))
    if not _range_reported(Dh.data_ptr()):
        pytest.skip("the driver does not report host allocation ranges")
    from paper_2511_18022_gb300 import _lib
    lib = _lib.load()
    tour = np.ascontiguousarray(inst.tour, np.int32)
    dist = np.ascontiguousarray(inst.dist, np.int32)
    rc = lib.cvrpsd_split_eval_host(sp.ctx, tour.ctypes.data, inst.n, dist.ctypes.data, Dh.data_ptr(), cv.I16,
                                    64, 1 << 22, inst.Q, inst.L, None, None, None, None,
                                    torch.cuda.current_stream().cuda_stream)
    assert rc == _lib.ERR_ARG
    assert b"allocation ends" in lib.cvrpsd_last_error(sp.ctx)


def test_host_million_n1000_sampled(sp, cv):
    """The bench's end-to-end call at full size: 2^20 scenarios in page-locked
    host memory (device-generated, then four column blocks replaced by
    host-generated ones), split in place; those blocks match the oracle and
    the sum matches the device entry point on the same matrix."""
    from synth import demand_columns
    w = workload("million-n1000")
    inst, S = w.instances[0], w.S
    D = torch.empty((inst.n, S), dtype=torch.int16, device="cuda")
    sp.gen_demand(w.scen_seeds[0], cv.GEN_CORRELATED, inst.mu, inst.region, D)
    blk, starts, host = 2048, [0, 300_001, 654_321, S - 2048], {}
    for a in starts:
        host[a] = demand_columns(inst.mu, inst.region, w.kind, w.scen_seeds[0] + 2, np.arange(a, a + blk), np.int16)
        D[:, a:a + blk] = torch.from_numpy(host[a]).cuda()
    H = torch.empty((inst.n, S), dtype=torch.int16).pin_memory()
    H.copy_(D)
    Hout = torch.empty(S, dtype=torch.int32).pin_memory()
    rh = sp.split_host(inst.tour, inst.dist, H, inst.Q, inst.L, out_cost=Hout)
    rd = sp.split(inst.tour, inst.dist, D, inst.Q, inst.L)
    assert (rh.sum, rh.infeasible) == (rd.sum, rd.infeasible)
    got = Hout.numpy()
    for a in starts:
        want, _, _, _ = oracle.split_costs(inst.tour, inst.dist, host[a], inst.Q, inst.L, nthreads=8)
        assert np.array_equal(got[a:a + blk], want)


def test_pinned_matrix_sits_on_the_gpus_numa_node():
    """The e2e matrix is allocated by a thread bound to the CPUs next to the
    GPU; every resident page of it must then be on the GPU's NUMA node."""
    from paper_2511_18022_gb300 import hostmem
    node, cpus = hostmem.gpu_numa(0)
    if node is None or node < 0:
        pytest.skip("the GPU reports no NUMA node")
    H, placement = hostmem.pinned_near_gpu((64, 1 << 16), torch.int16, 0)
    pages = hostmem.pages_by_node(H.data_ptr())
    assert placement["bound"] and pages, placement
    assert set(pages) == {f"N{node}"}, pages
