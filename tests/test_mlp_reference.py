"""Pins for the FP64 surrogate reference (oracle/mlp_reference.py): its
hand-written gradient against central finite differences of its forward
pass, and its bf16 rounding against the bit patterns of the format."""
import numpy as np

from oracle import mlp_reference as M


def small_case(seed=0, T=6, n=9):
    rng = np.random.default_rng(seed)
    tours = np.stack([rng.permutation(np.arange(1, n + 1)) for _ in range(T)])
    cust = np.column_stack([rng.integers(0, 1001, n), rng.integers(0, 1001, n),
                            rng.integers(1, 20, n), rng.uniform(0.5, 5, n)]).astype(np.float64)
    pts = np.vstack([[500, 500], cust[:, :2]])
    dist = np.floor(np.sqrt(((pts[:, None] - pts[None]) ** 2).sum(-1)) + 0.5)
    p = rng.normal(0, 0.3, M.NPARAMS)
    target = rng.normal(0, 1, T)
    return tours, cust, dist, p, target


def test_gradient_matches_finite_differences():
    tours, cust, dist, p, target = small_case()
    phi, t = M.features(tours, cust, dist, Q=32.0)
    loss, g, _ = M.loss_and_grad(p, phi, t, target)
    rng = np.random.default_rng(1)
    idx = np.concatenate([rng.choice(np.arange(M.OFF_W1, M.OFF_B1), 25), rng.choice(np.arange(M.OFF_B1, M.OFF_W2), 10),
                          rng.choice(np.arange(M.OFF_W2, M.OFF_B2), 25), rng.choice(np.arange(M.OFF_B2, M.OFF_W3), 10),
                          rng.choice(np.arange(M.OFF_W3, M.OFF_B3), 10), [M.OFF_B3]])
    h = 1e-6
    for i in idx:
        q = p.copy()
        q[i] += h
        lp = M.loss_and_grad(q, phi, t, target)[0]
        q[i] -= 2 * h
        lm = M.loss_and_grad(q, phi, t, target)[0]
        fd = (lp - lm) / (2 * h)
        assert abs(fd - g[i]) <= 1e-5 * max(1.0, abs(fd)), (i, fd, g[i])


def test_features_by_hand():
    cust = np.array([[0, 0, 4, 1], [1000, 0, 8, 2], [0, 1000, 16, 4]], dtype=np.float64)
    dist = np.array([[0, 3, 4, 5], [3, 0, 6, 7], [4, 6, 0, 8], [5, 7, 8, 0]], dtype=np.float64)
    phi, t = M.features(np.array([[2, 3, 1]]), cust, dist, Q=16.0)
    # cumulative mu / Q along the tour: 8/16, 24/16, 28/16 -> fractional parts .5, .5, .75
    assert np.allclose(phi[0, :, 4], [0.5, 0.5, 0.75])
    assert np.allclose(phi[0, :, 0], [1.0, 0.0, 0.0]) and np.allclose(phi[0, :, 2], [0.5, 1.0, 0.25])
    # closed tour 0 -> 2 -> 3 -> 1 -> 0: 4 + 8 + 7 + 3 = 22
    assert np.isclose(t[0], 22 / (500 * 3))


def test_bf16_rounding():
    x = np.array([1.0, 1.00390625, 1.005859375, -3.14159, 65504.0, 1e-3], dtype=np.float32)
    r = M.to_bf16(x)
    # 1 + 2^-8 is a tie between 1 and 1 + 2^-7: ties go to the even mantissa (1.0)
    assert r[0] == 1.0 and r[1] == 1.0 and r[2] == 1.0078125
    assert abs(r[3] + 3.140625) < 1e-12
    bits = r.astype(np.float32).view(np.uint32)
    assert (bits & 0xFFFF == 0).all()


def test_bf16_pair():
    """A feature carried as two bfloat16 numbers: exact for values of at most
    16 significant bits, within 2^-16 relative otherwise, and both parts are
    bfloat16 bit patterns."""
    exact = np.array([1.0 + 2.0 ** -12, 0.75 + 2.0 ** -15, -(3.0 + 2.0 ** -10)], dtype=np.float32)
    assert np.array_equal(M.to_bf16_pair(exact), exact.astype(np.float64))
    rng = np.random.default_rng(5)
    v = rng.uniform(-2.0, 2.0, 1000).astype(np.float32)
    pair = M.to_bf16_pair(v)
    assert np.all(np.abs(pair - v) <= np.abs(v) * 2.0 ** -16)
    # one bfloat16 alone is off by up to 2^-9 relative; the pair is far closer
    assert np.abs(M.to_bf16(v) - v).max() > 100 * np.abs(pair - v).max()
    hi = M.to_bf16(v)
    lo = M.to_bf16(v.astype(np.float64) - hi)
    for part in (hi, lo):
        assert (part.astype(np.float32).view(np.uint32) & 0xFFFF == 0).all()
    assert np.array_equal(hi + lo, pair)
