"""Local search over giant tours with the exact GPU Split as the arbiter and an
optional learned surrogate that screens neighbours.

Each iteration draws random 2-opt / relocate moves of the current tour
(seeded host RNG), and the library's kernels do the rest on the device:

* build the neighbour tours;
* screen them with the surrogate and keep the k best scores, or, without a
  surrogate, keep k random neighbours;
* evaluate those k tours exactly under every scenario;
* accept the best one if it improves the current SAA cost.

The exact Split stays the arbiter: the surrogate only decides which
neighbours get evaluated. This module sequences calls and holds no arithmetic
of the Split or of the network.
"""
from __future__ import annotations

import time
from dataclasses import dataclass, field

import numpy as np

from . import (Surrogate, cvrpsd_accept_best, cvrpsd_gather_tours, cvrpsd_neighbors, cvrpsd_split_eval_tours,
               cvrpsd_topk)


def random_moves(rng: np.random.Generator, M: int, n: int) -> np.ndarray:
    """M moves (type, a, b): half 2-opt segment reversals, half relocations."""
    t = rng.integers(0, 2, M)
    a = rng.integers(0, n, M)
    b = rng.integers(0, n - 1, M)
    b = b + (b >= a)                      # b != a
    return np.stack([t, a, b], axis=1).astype(np.int32)


def customer_features(inst, D_host_sample: np.ndarray) -> np.ndarray:
    """(x, y, mean demand, demand sd) per customer, from a sample of scenario
    columns [n][s] (the statistics the surrogate sees)."""
    d = D_host_sample.astype(np.float64)
    return np.column_stack([inst.coords[1:, 0], inst.coords[1:, 1], d.mean(axis=1),
                            d.std(axis=1)]).astype(np.float32)


class Evaluator:
    """Exact SAA costs of device tours of one instance."""

    def __init__(self, ctx, inst, D):
        import torch
        self.ctx, self.inst, self.D = ctx, inst, D
        self._mean = torch.empty(0, dtype=torch.float64, device=D.device)

    def __call__(self, tours):
        import torch
        T = int(tours.shape[0])
        if self._mean.numel() < T:
            self._mean = torch.empty(T, dtype=torch.float64, device=tours.device)
        out = self._mean[:T]
        cvrpsd_split_eval_tours(self.ctx, tours, self.inst.dist, self.D, self.inst.Q, self.inst.L, mean=out)
        return out


@dataclass
class SearchLog:
    costs: list = field(default_factory=list)     # current SAA cost after each iteration
    screened: int = 0                             # candidate tours considered
    evaluated: int = 0                            # tours split exactly
    seconds: float = 0.0

    @property
    def candidates_per_s(self) -> float:
        return self.screened / self.seconds if self.seconds else 0.0


class LocalSearch:
    """Best-improvement local search from `start` (host int array of ids).

    An iteration never waits for the device: the moves of the next
    `moves_block` iterations are drawn on the host and copied at once, the
    best evaluated neighbour is chosen and accepted on the device
    (cvrpsd_accept_best), and the per-iteration costs, kept on the device in
    chunks of `trace_chunk`, are read back when run() ends."""

    def __init__(self, ctx, inst, D, start, *, surrogate: Surrogate | None = None, M: int = 4096, k: int = 64,
                 seed: int = 0, retrain_every: int = 0, scale=(0.0, 1.0), lr: float = 2e-4,
                 moves_block: int = 64, exact_all: bool = False, explore: int = 0, trace_chunk: int = 1024):
        """Three modes: with a surrogate, screen M neighbours and split the k
        best exactly; with exact_all, split all M neighbours exactly (the
        plain-Split search the screened one is measured against: same moves
        for the same seed); otherwise split k random neighbours. `explore`
        (screened mode) gives that many of the k exact evaluations to
        neighbours the surrogate did not pick: the last `explore` of the
        iteration's random moves."""
        import torch
        self.ctx, self.inst, self.D = ctx, inst, D
        self.n = inst.n
        if surrogate is not None and exact_all:
            raise ValueError("exact_all splits every neighbour: no surrogate")
        self.exact_all = exact_all
        self.M = M if (surrogate is not None or exact_all) else k
        k = self.M if exact_all else k
        self.k = k
        if not 0 <= explore < k or (explore and surrogate is None):
            raise ValueError("explore needs a surrogate and 0 <= explore < k")
        self.explore = explore
        self.sur = surrogate
        self.rng = np.random.default_rng(seed)
        self.eval = Evaluator(ctx, inst, D)
        dev = D.device
        self.cur = torch.tensor(np.asarray(start, dtype=np.int32), device=dev)
        self.cur_cost_t = self.eval(self.cur.view(1, -1))[:1].clone()     # device [1]
        self.moves_block = moves_block
        self._moves_host = torch.empty((moves_block, self.M, 3), dtype=torch.int32).pin_memory()
        self._moves = torch.empty((moves_block, self.M, 3), dtype=torch.int32, device=dev)
        self._moves_copied = torch.cuda.Event()
        self._mi = moves_block
        self.cand = torch.empty((self.M, self.n), dtype=torch.int32, device=dev)
        self.top = torch.empty((k, self.n), dtype=torch.int32, device=dev)
        self.idx = torch.empty(k, dtype=torch.int32, device=dev)
        self.scores = torch.empty(self.M, dtype=torch.float32, device=dev)
        self.retrain_every = retrain_every
        self.scale = scale
        self.lr = lr
        self.new_tours, self.new_costs = [], []
        self._trace = []                  # device chunks of the cost trace
        self._trace_chunk = max(1, int(trace_chunk))
        self._tpos = self._trace_chunk
        self.log = SearchLog()

    @property
    def cur_cost(self) -> float:
        return float(self.cur_cost_t[0].item())

    def _next_moves(self):
        import torch
        if self._mi == self.moves_block:
            # the previous block's copy must have left the pinned buffer
            self._moves_copied.synchronize()
            blk = np.stack([random_moves(self.rng, self.M, self.n) for _ in range(self.moves_block)])
            self._moves_host.copy_(torch.from_numpy(blk))
            self._moves.copy_(self._moves_host, non_blocking=True)
            self._moves_copied.record()
            self._mi = 0
        m = self._moves[self._mi]
        self._mi += 1
        return m

    def step(self):
        import torch
        cvrpsd_neighbors(self.ctx, self.cur, self._next_moves(), self.cand)
        if self.sur is not None:
            self.sur.predict(self.cand, self.scores)
            kt = self.k - self.explore
            cvrpsd_topk(self.ctx, self.scores, kt, self.idx)
            cvrpsd_gather_tours(self.ctx, self.cand, self.idx[:kt], self.top)
            if self.explore:
                self.top[kt:].copy_(self.cand[self.M - self.explore:])
            chosen = self.top
        elif self.exact_all:
            chosen = self.cand
        else:
            chosen = self.cand[: self.k]
        costs = self.eval(chosen)
        # the cheapest candidate replaces the current tour if strictly
        # cheaper; the cost after the step goes to the device trace
        if self._tpos == self._trace_chunk:
            self._trace.append(torch.empty(self._trace_chunk, dtype=torch.float64, device=costs.device))
            self._tpos = 0
        cvrpsd_accept_best(self.ctx, chosen, costs, self.cur, self.cur_cost_t,
                           trace=self._trace[-1][self._tpos:self._tpos + 1])
        self._tpos += 1
        self.log.screened += self.M
        self.log.evaluated += self.k
        if self.sur is not None and self.retrain_every:
            self.new_tours.append(chosen.clone())
            self.new_costs.append(costs.to(torch.float32).clone())
            if len(self.new_tours) >= self.retrain_every:
                tours = torch.cat(self.new_tours)
                target = (torch.cat(self.new_costs) - self.scale[0]) / self.scale[1]
                for _ in range(4):
                    self.sur.train_step(tours, target, self.lr)
                self.new_tours, self.new_costs = [], []

    def run(self, iterations: int, seconds: float | None = None) -> SearchLog:
        """`iterations` steps, or with `seconds` as many as fit in that wall
        time (at most `iterations`; the clock is checked every 32 steps)."""
        import torch
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for it in range(iterations):
            self.step()
            if seconds is not None and it % 32 == 31:
                torch.cuda.synchronize()
                if time.perf_counter() - t0 >= seconds:
                    break
        torch.cuda.synchronize()
        self.log.seconds += time.perf_counter() - t0
        self.flush()
        return self.log

    def flush(self):
        """Move the device-side cost trace of the steps taken so far into
        log.costs (step() alone only appends to the device trace)."""
        import torch
        if self._trace:
            last = self._trace[-1][:self._tpos]
            self.log.costs.extend(torch.cat(self._trace[:-1] + [last]).tolist())
            self._trace = []
            self._tpos = self._trace_chunk

    @property
    def iterations(self) -> int:
        return self.log.screened // self.M


def _ranks(x: np.ndarray) -> np.ndarray:
    """Average ranks (ties share their mean rank), 0-based."""
    order = np.argsort(x, kind="stable")
    r = np.empty(len(x), dtype=np.float64)
    r[order] = np.arange(len(x), dtype=np.float64)
    xs = x[order]
    i = 0
    while i < len(x):
        j = i
        while j + 1 < len(x) and xs[j + 1] == xs[i]:
            j += 1
        if j > i:
            r[order[i:j + 1]] = (i + j) / 2.0
        i = j + 1
    return r


def spearman(a, b) -> float:
    """Spearman rank correlation of two equally long sequences."""
    ra, rb = _ranks(np.asarray(a, dtype=np.float64)), _ranks(np.asarray(b, dtype=np.float64))
    ra -= ra.mean()
    rb -= rb.mean()
    den = float(np.sqrt((ra * ra).sum() * (rb * rb).sum()))
    return float((ra * rb).sum() / den) if den > 0 else float("nan")


def neighbourhood_quality(ctx, inst, D, sur: Surrogate, scale, tour, *, M: int = 4096, k: int = 64,
                          seed: int = 0) -> dict:
    """How well the surrogate ranks the M neighbours of one tour (what the
    screen decides): exact SAA costs of all M by the GPU Split, surrogate
    predictions in cost units, and their mean absolute error, Spearman rank
    correlation, the share of the exact top-k among the surrogate's top-k,
    and whether the exact best is in the surrogate's top-k."""
    import torch
    dev = D.device
    rng = np.random.default_rng(seed)
    moves = torch.from_numpy(random_moves(rng, M, inst.n)).to(dev)
    base = torch.as_tensor(np.asarray(tour, dtype=np.int32), device=dev)
    cand = torch.empty((M, inst.n), dtype=torch.int32, device=dev)
    cvrpsd_neighbors(ctx, base, moves, cand)
    exact = Evaluator(ctx, inst, D)(cand).cpu().numpy().astype(np.float64)
    pred_t = torch.empty(M, dtype=torch.float32, device=dev)
    sur.predict(cand, pred_t)
    pred = pred_t.cpu().numpy().astype(np.float64) * scale[1] + scale[0]
    top_pred = set(np.argsort(pred, kind="stable")[:k].tolist())
    top_exact = np.argsort(exact, kind="stable")[:k].tolist()
    return {"mae": float(np.abs(pred - exact).mean()), "spearman": spearman(pred, exact),
            "recall_at_k": len(top_pred.intersection(top_exact)) / k,
            "best_in_top_k": bool(int(np.argmin(exact)) in top_pred),
            "exact_spread": float(exact.std()), "k": k, "M": M}


def training_set(ctx, inst, D, count: int, seed: int = 0, chain: int = 64, chunk: int = 4096):
    """`count` (tour, exact SAA cost) pairs: neighbours of a chain of base
    tours that improves step by step from a random permutation (so the set
    spans random to locally improved tours). Returns device tensors."""
    import torch
    rng = np.random.default_rng(seed)
    dev = D.device
    n = inst.n
    ev = Evaluator(ctx, inst, D)
    base = torch.tensor(rng.permutation(np.arange(1, n + 1)).astype(np.int32), device=dev)
    base_cost = float(ev(base.view(1, -1))[0].item())
    per_base = max(1, count // chain)
    tours = torch.empty((count, n), dtype=torch.int32, device=dev)
    costs = torch.empty(count, dtype=torch.float64, device=dev)
    filled = 0
    while filled < count:
        m = min(per_base, count - filled)
        moves = torch.from_numpy(random_moves(rng, m, n)).to(dev)
        cvrpsd_neighbors(ctx, base, moves, tours[filled:filled + m])
        for a in range(filled, filled + m, chunk):
            b = min(filled + m, a + chunk)
            costs[a:b] = ev(tours[a:b])
        block = costs[filled:filled + m]
        j = int(torch.argmin(block).item())
        if float(block[j].item()) < base_cost:       # move the base downhill
            base = tours[filled + j].clone()
            base_cost = float(block[j].item())
        filled += m
    return tours, costs


def tour_lengths(tours_host: np.ndarray, dist: np.ndarray) -> np.ndarray:
    """Closed lengths (depot, tour, depot) of host tours [T][n]."""
    t = np.asarray(tours_host, dtype=np.int64)
    d = np.asarray(dist, dtype=np.int64)
    return d[0, t[:, 0]] + d[t[:, -1], 0] + d[t[:, :-1], t[:, 1:]].sum(axis=1)


def train_surrogate(sur: Surrogate, tours, costs, *, dist=None, epochs: int = 8, batch: int = 1024,
                    lr: float = 1e-3, seed: int = 0, holdout: float = 0.1):
    """Fit the surrogate to standardised costs (the tour-length input is
    standardised over the same tours when `dist` is given); returns (mean, sd)
    of the costs and the held-out mean absolute error in cost units."""
    import torch
    N = int(tours.shape[0])
    if dist is not None:
        lens = tour_lengths(tours.cpu().numpy(), dist).astype(np.float64)
        sur.set_scale(float(lens.mean()), float(lens.std() + 1e-9))
    g = torch.Generator(device="cpu").manual_seed(seed)
    perm = torch.randperm(N, generator=g).to(tours.device)
    n_hold = int(N * holdout)
    hold, train = perm[:n_hold], perm[n_hold:]
    c32 = costs.to(torch.float32)
    mean, sd = float(c32[train].mean().item()), float(c32[train].std().item())
    target = (c32 - mean) / sd
    steps = 0
    total = epochs * ((len(train) + batch - 1) // batch)
    for ep in range(epochs):
        order = train[torch.randperm(len(train), generator=g).to(tours.device)]
        for a in range(0, len(order), batch):
            ix = order[a:a + batch]
            rate = lr * (0.1 + 0.9 * (1.0 - steps / total))    # linear decay to 10 %
            sur.train_step(tours[ix].contiguous(), target[ix].contiguous(), rate)
            steps += 1
    pred = torch.empty(n_hold, dtype=torch.float32, device=tours.device)
    sur.predict(tours[hold].contiguous(), pred)
    mae = float(((pred * sd + mean) - c32[hold]).abs().mean().item())
    return (mean, sd), mae


def oos_study(ctx, inst, D_train, D_test, S_list, *, iterations: int = 400, seed: int = 0, k: int = 64,
              repeats: int = 1):
    """Out-of-sample effect of the scenario count (the study of Section 4.2
    on a synthetic instance): for each S in S_list, local search with the
    exact Split on the first S training scenarios; the final tour is then
    split under the held-out scenarios D_test. With repeats > 1 every S runs
    that many searches (start and move seeds seed, seed+1, ...) and the row
    holds the means. Returns rows (S, in-sample SAA cost, out-of-sample SAA
    cost)."""
    test_eval = Evaluator(ctx, inst, D_test)
    rows = []
    for S in S_list:
        Dtr = D_train[:, :S].contiguous()
        ins, outs = [], []
        for r in range(repeats):
            sd = seed + 1000 * r
            start = np.random.default_rng(sd).permutation(np.arange(1, inst.n + 1)).astype(np.int32)
            ls = LocalSearch(ctx, inst, Dtr, start, k=k, seed=sd + 1)
            ls.run(iterations)
            ins.append(ls.cur_cost)
            outs.append(float(test_eval(ls.cur.view(1, -1))[0].item()))
        rows.append((int(S), float(np.mean(ins)), float(np.mean(outs))))
    return rows
