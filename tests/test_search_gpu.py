"""GPU tests of the local-search pieces: the many-tours Split, neighbour
moves, top-k, the surrogate network's kernels (against the FP64 reference)
and what the trained surrogate gains over unscreened neighbour choice."""
import numpy as np
import pytest

import oracle
from oracle import mlp_reference as M
from synth import demand_matrix, make_instance, workload

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


def apply_move(tour, t, a, b):
    tour = list(tour)
    if t == 0:
        lo, hi = min(a, b), max(a, b)
        tour[lo:hi + 1] = tour[lo:hi + 1][::-1]
        return tour
    c = tour.pop(a)
    tour.insert(b, c)
    return tour


def test_split_eval_tours_matches_oracle(sp, cv):
    w = workload("corr-n200", S=3001)
    inst = w.instances[0]
    D = demand_matrix(inst.mu, inst.region, w.kind, w.scen_seeds[0], 3001, dtype=np.int16)
    D[11, 7] = inst.Q + 3
    rng = np.random.default_rng(0)
    tours = np.stack([inst.tour] + [rng.permutation(np.arange(1, inst.n + 1)) for _ in range(9)]).astype(np.int32)
    dT = torch.from_numpy(tours).cuda()
    dD = torch.from_numpy(D).cuda()
    mean = torch.empty(10, dtype=torch.float64, device="cuda")
    sums = torch.empty(10, dtype=torch.int64, device="cuda")
    inf = torch.empty(10, dtype=torch.int64, device="cuda")
    cv.cvrpsd_split_eval_tours(sp.ctx, dT, inst.dist, dD, inst.Q, inst.L, mean=mean, sums=sums, infeasible=inf)
    for t in range(10):
        _, ws, wi, _ = oracle.split_costs(tours[t], inst.dist, D, inst.Q, inst.L)
        assert (int(sums[t]), int(inf[t])) == (ws, wi)
        assert float(mean[t]) == ws / (3001 - wi)


def test_split_eval_tours_surrogate_size(sp, cv):
    """The search's exact evaluation at its own size: 8 tours of the
    surrogate-n200 instance under all 65,536 scenarios, exactly as the
    oracle sums them."""
    w = workload("surrogate-n200")
    inst, S = w.instances[0], w.S
    D = demand_matrix(inst.mu, inst.region, w.kind, w.scen_seeds[0], S, dtype=np.int16)
    rng = np.random.default_rng(3)
    tours = np.stack([inst.tour] + [rng.permutation(np.arange(1, inst.n + 1)) for _ in range(7)]).astype(np.int32)
    sums = torch.empty(8, dtype=torch.int64, device="cuda")
    inf = torch.empty(8, dtype=torch.int64, device="cuda")
    cv.cvrpsd_split_eval_tours(sp.ctx, torch.from_numpy(tours).cuda(), inst.dist, torch.from_numpy(D).cuda(),
                               inst.Q, inst.L, sums=sums, infeasible=inf)
    for t in range(8):
        _, ws, wi, _ = oracle.split_costs(tours[t], inst.dist, D, inst.Q, inst.L, nthreads=8)
        assert (int(sums[t]), int(inf[t])) == (ws, wi)


def test_neighbors_and_gather(sp, cv):
    rng = np.random.default_rng(2)
    n = 37
    base = rng.permutation(np.arange(1, n + 1)).astype(np.int32)
    from paper_2511_18022_gb300.search import random_moves
    moves = random_moves(rng, 500, n)
    moves[:3] = [[0, 5, 5], [1, 0, n - 1], [1, n - 1, 0]]
    out = torch.empty((500, n), dtype=torch.int32, device="cuda")
    cv.cvrpsd_neighbors(sp.ctx, torch.from_numpy(base).cuda(), torch.from_numpy(moves).cuda(), out)
    got = out.cpu().numpy()
    for m in range(500):
        assert got[m].tolist() == apply_move(base, *moves[m]), m
    idx = torch.tensor([499, 0, 17], dtype=torch.int32, device="cuda")
    g = torch.empty((3, n), dtype=torch.int32, device="cuda")
    cv.cvrpsd_gather_tours(sp.ctx, out, idx, g)
    assert (g.cpu().numpy() == got[[499, 0, 17]]).all()


@pytest.mark.parametrize("M,k", [(4096, 64), (1000, 1000), (5, 1), (3000, 17)])
def test_topk(sp, cv, M, k):
    rng = np.random.default_rng(M)
    s = rng.normal(size=M).astype(np.float32)
    s[rng.integers(0, M, M // 10)] = 0.25                # ties
    if M > 10:
        s[3] = np.nan
    out = torch.empty(k, dtype=torch.int32, device="cuda")
    cv.cvrpsd_topk(sp.ctx, torch.from_numpy(s).cuda(), k, out)
    key = np.where(np.isnan(s), np.inf, s)
    want = np.lexsort((np.arange(M), key))[:k]
    assert out.cpu().numpy().tolist() == want.tolist()


@pytest.mark.parametrize("T,case", [(1, "better"), (7, "tie"), (300, "tie"), (64, "worse"), (33, "nan"),
                                    (513, "equal")])
def test_accept_best(sp, cv, T, case):
    """cvrpsd_accept_best against the rule written out on the host: the
    cheapest candidate (first of equal costs, NaN never), taken only if
    strictly below the current cost; the trace holds the cost after."""
    rng = np.random.default_rng(T)
    n = 37
    tours = rng.integers(1, 1000, size=(T, n)).astype(np.int32)
    cost = rng.uniform(100, 200, T)
    cur0 = np.arange(1, n + 1, dtype=np.int32)
    cc0 = 150.0
    if case == "better":
        cost[0] = 99.0
    elif case == "tie":
        cost[T // 3] = cost[T - 1] = 50.0            # equal minima: the first wins
    elif case == "worse":
        cost[:] = rng.uniform(151, 200, T)
    elif case == "nan":
        cost[:] = np.nan
        cost[5] = 120.0
    elif case == "equal":
        cost[:] = rng.uniform(150.5, 200, T)
        cost[200] = cc0                               # not strictly cheaper
    key = np.where(np.isnan(cost), np.inf, cost)
    b = int(np.argmin(key))
    take = key[b] < cc0
    want_cur = tours[b] if take else cur0
    want_c = key[b] if take else cc0
    d_cur = torch.from_numpy(cur0.copy()).cuda()
    d_cc = torch.tensor([cc0], dtype=torch.float64, device="cuda")
    trace = torch.full((1,), -1.0, dtype=torch.float64, device="cuda")
    d_tours = torch.from_numpy(tours).cuda()
    cv.cvrpsd_accept_best(sp.ctx, d_tours, torch.from_numpy(cost).cuda(), d_cur, d_cc, trace=trace)
    assert d_cur.cpu().numpy().tolist() == want_cur.tolist()
    assert d_cc.item() == want_c and trace.item() == want_c
    with pytest.raises(cv.CvrpsdError):
        cv.cvrpsd_accept_best(sp.ctx, d_tours, torch.from_numpy(cost).cuda(), d_tours[0], d_cc)


def surrogate_case(cv, sp, T=48, n=60, seed=0):
    inst = make_instance(n, 5, 20, seed=seed, Q=64)
    rng = np.random.default_rng(seed)
    cust = np.column_stack([inst.coords[1:, 0], inst.coords[1:, 1], inst.mu,
                            rng.uniform(1, 6, n)]).astype(np.float32)
    sur = cv.Surrogate(sp.ctx, cust, inst.dist, Q=64.0, seed=seed + 1)
    tours = np.stack([rng.permutation(np.arange(1, n + 1)) for _ in range(T)]).astype(np.int32)
    target = rng.normal(size=T).astype(np.float32)
    return inst, cust, sur, tours, target


def test_surrogate_forward_matches_reference(sp, cv):
    inst, cust, sur, tours, _ = surrogate_case(cv, sp)
    p = sur.params()
    phi, t = M.features(tours, cust, inst.dist, Q=64.0)   # Q = 2^6 keeps the features exact in fp32
    want, _ = M.forward(p, phi, t, bf16=True)
    out = torch.empty(len(tours), dtype=torch.float32, device="cuda")
    sur.predict(torch.from_numpy(tours).cuda(), out)
    assert np.allclose(out.cpu().numpy(), want, rtol=1e-4, atol=1e-4)
    sur.close()


def test_surrogate_scaled_length_matches_reference(sp, cv):
    inst, cust, sur, tours, _ = surrogate_case(cv, sp, seed=9)
    sur.set_scale(30000.0, 1024.0)
    p = sur.params()
    phi, t = M.features(tours, cust, inst.dist, Q=64.0, len_mean=30000.0, len_sd=1024.0)
    want, _ = M.forward(p, phi, t, bf16=True)
    out = torch.empty(len(tours), dtype=torch.float32, device="cuda")
    sur.predict(torch.from_numpy(tours).cuda(), out)
    assert np.allclose(out.cpu().numpy(), want, rtol=1e-4, atol=1e-4)
    sur.close()


def test_surrogate_gradients_match_reference(sp, cv):
    inst, cust, sur, tours, target = surrogate_case(cv, sp, seed=3)
    p = sur.params()
    phi, t = M.features(tours, cust, inst.dist, Q=64.0)
    wloss, wg, _ = M.loss_and_grad(p, phi, t, target, bf16=True)
    g, loss = sur.gradients(torch.from_numpy(tours).cuda(), torch.from_numpy(target).cuda())
    assert abs(loss - wloss) <= 1e-4 * max(1.0, wloss)
    for lo, hi in ((M.OFF_W1, M.OFF_B1), (M.OFF_B1, M.OFF_W2), (M.OFF_W2, M.OFF_B2), (M.OFF_B2, M.OFF_W3),
                   (M.OFF_W3, M.OFF_B3), (M.OFF_B3, M.NPARAMS)):
        scale = np.abs(wg[lo:hi]).max() + 1e-12
        assert np.abs(g[lo:hi] - wg[lo:hi]).max() <= 1e-3 * scale, (lo, hi)
    sur.close()


def test_surrogate_checkpoint_resume(sp, cv, tmp_path):
    """A checkpoint restores parameters, Adam moments, step and input scale
    exactly, and training resumed from it follows the uninterrupted run."""
    inst, cust, sur, tours, target = surrogate_case(cv, sp, T=256, seed=4)
    sur.set_scale(20000.0, 900.0)
    dT, dY = torch.from_numpy(tours).cuda(), torch.from_numpy(target).cuda()
    for _ in range(3):
        sur.train_step(dT, dY, 1e-3)
    path = tmp_path / "sur.ckpt"
    sur.save(path)
    blob = path.read_bytes()
    other = cv.Surrogate(sp.ctx, cust, inst.dist, Q=64.0, seed=99)     # different initial weights
    assert not np.array_equal(other.params(), sur.params())
    other.load(path)
    assert other.state() == blob                                        # exact restore
    assert np.array_equal(other.params(), sur.params())
    for _ in range(4):
        sur.train_step(dT, dY, 1e-3)
        other.train_step(dT, dY, 1e-3)
    a, b = sur.params(), other.params()
    ckpt = np.frombuffer(blob, dtype=np.float32, count=M.NPARAMS, offset=32)
    assert np.abs(a - ckpt).max() > 1e-4                                # training moved on
    # the two runs differ only by the order of floating-point atomics in the
    # gradient sums: almost all parameters agree to rounding, and no update
    # can differ by more than Adam's step bound (lr per step)
    d = np.abs(a - b)
    assert np.percentile(d, 99) <= 1e-6 and d.max() <= 2 * 4 * 1e-3
    # a checkpoint of a network for another n is refused
    inst2, cust2, sur2, _, _ = surrogate_case(cv, sp, n=23, T=8, seed=6)
    with pytest.raises(cv.CvrpsdError):
        sur2.load_state(blob)
    for s in (sur, other, sur2):
        s.close()


def test_training_reduces_loss(sp, cv):
    inst, cust, sur, tours, _ = surrogate_case(cv, sp, T=512, seed=5)
    dT = torch.from_numpy(tours).cuda()
    phi, t = M.features(tours, cust, inst.dist, Q=64.0)
    lens = t * 500.0 * inst.n
    sur.set_scale(float(lens.mean()), float(lens.std()))
    y = torch.tensor(((lens - lens.mean()) / lens.std()).astype(np.float32)).cuda()   # learnable target
    _, l0 = sur.gradients(dT, y)
    for _ in range(200):
        sur.train_step(dT, y, 3e-3)
    _, l1 = sur.gradients(dT, y)
    assert l1 < 0.2 * l0
    sur.close()


def test_surrogate_screening_beats_random_choice(sp, cv):
    """The trained surrogate's top-64 of 4096 neighbours contain clearly
    cheaper tours (by the exact Split) than 64 unscreened neighbours."""
    from paper_2511_18022_gb300 import search
    w = workload("surrogate-n200", S=4096)
    inst = w.instances[0]
    D = torch.empty((inst.n, w.S), dtype=torch.int16, device="cuda")
    sp.gen_demand(w.scen_seeds[0], cv.GEN_CORRELATED, inst.mu, inst.region, D)
    cust = search.customer_features(inst, D[:, :4096].cpu().numpy())
    tours, costs = search.training_set(sp.ctx, inst, D, 24_000, seed=1)
    sur = cv.Surrogate(sp.ctx, cust, inst.dist, Q=float(inst.Q), seed=7)
    scale, mae = search.train_surrogate(sur, tours, costs, dist=inst.dist, epochs=10)
    assert mae < 0.5 * float(costs.std().item())
    rng = np.random.default_rng(3)
    ev = search.Evaluator(sp.ctx, inst, D)
    base = tours[int(torch.argmin(costs).item())].clone()
    gains = []
    for _ in range(8):
        moves = torch.from_numpy(search.random_moves(rng, 4096, inst.n)).cuda()
        cand = torch.empty((4096, inst.n), dtype=torch.int32, device="cuda")
        cv.cvrpsd_neighbors(sp.ctx, base, moves, cand)
        scores = torch.empty(4096, dtype=torch.float32, device="cuda")
        sur.predict(cand, scores)
        idx = torch.empty(64, dtype=torch.int32, device="cuda")
        cv.cvrpsd_topk(sp.ctx, scores, 64, idx)
        top = torch.empty((64, inst.n), dtype=torch.int32, device="cuda")
        cv.cvrpsd_gather_tours(sp.ctx, cand, idx, top)
        screened = ev(top).clone()
        unscreened = ev(cand[:64].contiguous()).clone()
        gains.append(float(unscreened.mean() - screened.mean()))
    assert np.mean(gains) > 0 and sum(g > 0 for g in gains) >= 6
    sur.close()


def test_more_training_scenarios_generalise_better(sp, cv):
    """Section 4.2's observation on a synthetic instance: a tour optimised on
    one scenario does worse on held-out scenarios than one optimised on a
    thousand."""
    from paper_2511_18022_gb300 import search
    w = workload("surrogate-n200", S=1000)
    inst = w.instances[0]
    D_train = torch.empty((inst.n, 1000), dtype=torch.int16, device="cuda")
    sp.gen_demand(w.scen_seeds[0], cv.GEN_CORRELATED, inst.mu, inst.region, D_train)
    D_test = torch.empty((inst.n, 100_000), dtype=torch.int16, device="cuda")
    sp.gen_demand(w.scen_seeds[0] + 5, cv.GEN_CORRELATED, inst.mu, inst.region, D_test)
    rows = search.oos_study(sp.ctx, inst, D_train, D_test, [1, 1000], iterations=150, seed=2)
    (s1, in1, out1), (s2, in2, out2) = rows
    assert out2 < out1


def test_local_search_matches_host_accept_rule(sp, cv):
    """The device-side choice and acceptance of LocalSearch against a host
    replica: same seeded moves, neighbours built on the host from the moves'
    definition, exact costs from the oracle, the best neighbour accepted only
    if strictly cheaper. Same final tour, same cost trace (non-increasing),
    and the reported cost is the exact cost of the final tour."""
    from paper_2511_18022_gb300 import search
    inst = make_instance(60, 1, 10, seed=13, Q=40, L=15)
    S = 257
    D = demand_matrix(inst.mu, inst.region, 1, 5, S, dtype=np.int16)
    dD = torch.from_numpy(D).cuda()
    start = np.random.default_rng(2).permutation(np.arange(1, inst.n + 1)).astype(np.int32)
    k, iters = 16, 100
    # a trace chunk of 7 costs: the device trace rolls over 14 times
    ls = search.LocalSearch(sp.ctx, inst, dD, start, k=k, seed=77, moves_block=8, trace_chunk=7)
    for _ in range(iters):
        ls.step()
    ls.flush()

    def cost(t):
        _, s, inf, _ = oracle.split_costs(np.asarray(t, np.int32), inst.dist, D, inst.Q, inst.L)
        return s / (S - inf)

    rng = np.random.default_rng(77)
    cur, cur_c, trace = list(start), cost(start), []
    block = []
    for _ in range(iters):
        if not block:
            block = [search.random_moves(rng, k, inst.n) for _ in range(8)]
        moves = block.pop(0)
        cands = [apply_move(cur, *(int(x) for x in m)) for m in moves]
        cs = [cost(c) for c in cands]
        b = int(np.argmin(cs))
        if cs[b] < cur_c:
            cur, cur_c = cands[b], cs[b]
        trace.append(cur_c)
    assert ls.cur.cpu().tolist() == cur
    assert ls.log.costs == trace
    assert all(b <= a for a, b in zip(trace, trace[1:]))
    assert ls.cur_cost == cost(ls.cur.cpu().numpy())


def test_screened_search_against_plain_split_search(sp, cv):
    """The surrogate-screened search (screen M neighbours, split the k best)
    against the plain-Split search that splits all M neighbours exactly, same
    moves and start, reduced scale: at least 10x the candidate tours per
    second, and within the same wall time a final SAA cost within 0.5 % of
    the plain search's."""
    from paper_2511_18022_gb300 import search
    w = workload("surrogate-n200", S=8192)
    inst = w.instances[0]
    D = torch.empty((inst.n, w.S), dtype=torch.int16, device="cuda")
    sp.gen_demand(w.scen_seeds[0], cv.GEN_CORRELATED, inst.mu, inst.region, D)
    cust = search.customer_features(inst, D[:, :4096].cpu().numpy())
    tours, costs = search.training_set(sp.ctx, inst, D, 40_000, seed=1)
    sur = cv.Surrogate(sp.ctx, cust, inst.dist, Q=float(inst.Q), seed=7)
    scale, _ = search.train_surrogate(sur, tours, costs, dist=inst.dist, epochs=8)
    start = np.random.default_rng(5).permutation(np.arange(1, inst.n + 1)).astype(np.int32)
    plain = search.LocalSearch(sp.ctx, inst, D, start, M=2048, seed=9, exact_all=True)
    plain.run(60)
    screened = search.LocalSearch(sp.ctx, inst, D, start, surrogate=sur, M=2048, k=32, seed=9, retrain_every=25,
                                  scale=scale)
    screened.run(100_000, seconds=plain.log.seconds)
    assert screened.log.candidates_per_s >= 10 * plain.log.candidates_per_s
    assert screened.cur_cost <= 1.005 * plain.cur_cost
    q = search.neighbourhood_quality(sp.ctx, inst, D, sur, scale, screened.cur.cpu().numpy(), M=2048, k=32)
    assert q["spearman"] > 0.3
    sur.close()


def test_screened_search_exploration_slots(sp, cv):
    """With `explore` slots the k exact evaluations are the k - explore best
    by the surrogate plus the iteration's last `explore` random neighbours:
    the cost trace stays non-increasing, the reported cost is the exact cost
    of the final tour, and bad settings are refused."""
    from paper_2511_18022_gb300 import search
    inst = make_instance(60, 1, 10, seed=13, Q=40, L=15)
    S = 257
    D = demand_matrix(inst.mu, inst.region, 1, 5, S, dtype=np.int16)
    dD = torch.from_numpy(D).cuda()
    cust = search.customer_features(inst, D)
    sur = cv.Surrogate(sp.ctx, cust, inst.dist, Q=float(inst.Q), seed=3)
    start = np.random.default_rng(2).permutation(np.arange(1, inst.n + 1)).astype(np.int32)
    with pytest.raises(ValueError):
        search.LocalSearch(sp.ctx, inst, dD, start, surrogate=sur, M=256, k=16, explore=16)
    with pytest.raises(ValueError):
        search.LocalSearch(sp.ctx, inst, dD, start, k=16, explore=4)
    ls = search.LocalSearch(sp.ctx, inst, dD, start, surrogate=sur, M=256, k=16, seed=4, explore=4)
    log = ls.run(80)
    assert all(b <= a for a, b in zip(log.costs, log.costs[1:]))
    _, s, inf, _ = oracle.split_costs(ls.cur.cpu().numpy(), inst.dist, D, inst.Q, inst.L)
    assert ls.cur_cost == s / (S - inf)
    assert sorted(ls.cur.cpu().tolist()) == list(range(1, inst.n + 1))
    sur.close()
