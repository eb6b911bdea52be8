"""Checks of the seeded input generators against their published definitions
and against the distributional facts the workload recipe fixes."""
import numpy as np
import pytest

from synth import (SplitMix64, philox4x32_10, make_instance, demand_columns,
                   demand_matrix, workload, KIND_NORMAL, KIND_CORRELATED)
from synth.scenarios import std_normal, round_half_away, DOM_E, DOM_F


def test_philox_known_answers():
    # Known-answer vectors published with Random123 for Philox4x32-10
    # (Salmon et al., SC 2011): (counter, key) -> output.
    kat = [((0, 0, 0, 0), (0, 0), (0x6627E8D5, 0xE169C58D, 0xBC57AC4C, 0x9B00DBD8)),
           ((0xFFFFFFFF,) * 4, (0xFFFFFFFF,) * 2, (0x408F276D, 0x41C83B0E, 0xA20BC7C6, 0x6D5451FD)),
           ((0x243F6A88, 0x85A308D3, 0x13198A2E, 0x03707344), (0xA4093822, 0x299F31D0),
            (0xD16CFE09, 0x94FDCCEB, 0x5001E420, 0x24126EA1))]
    for ctr, key, want in kat:
        got = philox4x32_10(*ctr, *key)
        assert tuple(int(x) for x in got) == want


def test_c_philox_words_match_numpy():
    """The C Philox used for large grids gives the numpy version's words."""
    from synth import _cphilox
    if _cphilox.load() is None:
        pytest.skip("no C compiler")
    s = np.array([0, 1, 2**32 - 1, 77, 123456789], dtype=np.int64)
    idx = np.array([0, 3, 999, 2**31], dtype=np.int64)
    w0, w1 = _cphilox.words(s, idx, 2, 0xA4093822, 0x299F31D0)
    ref = philox4x32_10(s[None, :], idx[:, None], 2, 0, 0xA4093822, 0x299F31D0)
    assert (w0 == ref[0]).all() and (w1 == ref[1]).all()
    # the first Random123 known answer has a zero counter and key
    kat = _cphilox.words(np.array([0]), np.array([0]), 0, 0, 0)
    assert (int(kat[0][0, 0]), int(kat[1][0, 0])) == (0x6627E8D5, 0xE169C58D)


def test_parallel_matrix_equals_serial():
    from synth import demand_matrix_parallel
    inst = make_instance(30, 1, 30, seed=3, Q=200)
    a = demand_matrix_parallel(inst.mu, inst.region, KIND_CORRELATED, 41, 5000, s0=17, workers=2, chunk=1024)
    b = demand_matrix(inst.mu, inst.region, KIND_CORRELATED, 41, 5000, s0=17)
    assert (a == b).all()


def test_splitmix64_reference_outputs():
    # First outputs of the reference SplitMix64 generator seeded with 0.
    r = SplitMix64(0)
    assert [r.next_u64() for _ in range(3)] == [
        0xE220A8397B1DCDAF, 0x6E789E6AA1B965F4, 0x06C45D188009454F]


def test_bounded_draws_and_permutation():
    r = SplitMix64(123)
    x = r.integers(3, 7, 4000)
    assert x.min() == 3 and x.max() == 7
    counts = np.bincount(x - 3)
    assert (np.abs(counts - 800) < 120).all()
    p = SplitMix64(5).permutation(range(1, 101))
    assert sorted(p.tolist()) == list(range(1, 101))


def test_round_half_away():
    x = np.array([0.5, 1.5, 2.4999999, 2.5, 0.49999999999999994, 7.0])
    assert round_half_away(x).tolist() == [1.0, 2.0, 2.0, 3.0, 0.0, 7.0]


def test_instance_recipe():
    a = make_instance(30, 1, 10, seed=7, Q=40)
    b = make_instance(30, 1, 10, seed=7, Q=40)
    assert (a.tour == b.tour).all() and (a.dist == b.dist).all()
    assert sorted(a.tour.tolist()) == list(range(1, 31))
    assert (a.dist == a.dist.T).all() and (np.diag(a.dist) == 0).all()
    assert tuple(a.coords[0]) == (500, 500)
    assert a.coords[1:].min() >= 0 and a.coords[1:].max() <= 1000
    assert a.mu.min() >= 1 and a.mu.max() <= 10
    inst = make_instance(40, 1, 10, seed=1, q_from_mean=10)
    assert inst.Q == (10 * int(inst.mu.sum()) + 20) // 40


def test_columns_are_counter_based():
    inst = make_instance(25, 1, 30, seed=2, Q=200)
    full = demand_matrix(inst.mu, inst.region, KIND_CORRELATED, 99, 300, dtype=np.int16)
    pick = np.array([0, 17, 299, 150])
    sub = demand_columns(inst.mu, inst.region, KIND_CORRELATED, 99, pick, np.int16)
    assert (sub == full[:, pick]).all()
    shifted = demand_matrix(inst.mu, inst.region, KIND_CORRELATED, 99, 100, s0=200,
                            dtype=np.int16, chunk=33)
    assert (shifted == full[:, 200:]).all()


def test_standard_normals():
    s = np.arange(200_000)
    z = std_normal(7, s, 3, DOM_E)
    assert abs(z.mean()) < 0.01 and abs(z.var() - 1) < 0.015
    assert abs(((z ** 4).mean()) - 3) < 0.06           # normal kurtosis


def test_correlated_structure():
    S = 100_000
    s = np.arange(S)[None, :]
    f = std_normal(11, s, np.arange(4)[:, None], DOM_F)
    e = std_normal(11, s, np.arange(3)[:, None], DOM_E)
    y_a = 0.6 * f[2] + 0.8 * e[0]
    y_b = 0.6 * f[2] + 0.8 * e[1]     # same quadrant as a
    y_c = 0.6 * f[1] + 0.8 * e[2]     # another quadrant
    assert abs(np.corrcoef(y_a, y_b)[0, 1] - 0.36) < 0.015
    assert abs(np.corrcoef(y_a, y_c)[0, 1]) < 0.015
    assert abs(np.exp(0.3 * y_a - 0.045).mean() - 1.0) < 0.004   # mean preserving


def test_demand_moments():
    mu = np.array([5, 10, 20, 30])
    region = np.array([0, 1, 2, 3])
    d = demand_matrix(mu, region, KIND_CORRELATED, 5, 60_000, dtype=np.int32).astype(float)
    assert np.allclose(d.mean(1), mu, rtol=0.01)
    dn = demand_matrix(mu, region, KIND_NORMAL, 5, 60_000, dtype=np.int32).astype(float)
    assert np.allclose(dn.mean(1), mu, rtol=0.01)
    assert np.allclose(dn.std(1), np.sqrt((0.3 * mu) ** 2 + 1 / 12), rtol=0.03)
    assert dn.min() >= 0


@pytest.mark.parametrize("name", ["plain-n50", "corr-n200", "million-n1000"])
def test_named_workloads(name):
    w = workload(name, S=64)
    inst = w.instances[0]
    assert {"plain-n50": (50, 40, 50), "corr-n200": (200, 150, 40),
            "million-n1000": (1000, 200, 60)}[name] == (inst.n, inst.Q, inst.L)
    D = demand_matrix(inst.mu, inst.region, w.kind, w.scen_seeds[0], 64, dtype=w.dtype)
    assert D.shape == (inst.n, 64) and D.dtype == w.dtype


def test_batched_workload_sizes():
    w = workload("batched-512", S=8, T=6)
    ns = [inst.n for inst in w.instances]
    assert all(100 <= n <= 1000 for n in ns) and len(set(ns)) > 1
    for inst in w.instances:
        assert inst.L == inst.n and inst.mu.max() <= 10
        assert inst.Q == (10 * int(inst.mu.sum()) + inst.n // 2) // inst.n
