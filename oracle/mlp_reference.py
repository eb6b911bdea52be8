"""FP64 reference of the tour-cost surrogate network (test infrastructure).

TEST INFRASTRUCTURE ONLY: the GPU tests use it to check the library's BF16
training and inference kernels; the library never imports it. The network is
not part of the paper's method: it screens local-search neighbours before
the exact Split evaluates them.

Network (width H = 256), for a tour sigma_1..sigma_n of an instance with
customer features (x, y, mean demand mu, demand sd), capacity Q and distances c
(with bf16=True the weights are rounded to bfloat16 first and each feature
is carried as a bfloat16 pair, hi = bf16(v) plus lo = bf16(v - hi), v the
feature in float32):
    phi_k = (x/1000, y/1000, mu/Q, sd/Q, frac(sum_{t<=k} mu_{sigma_t} / Q))
    h_k   = relu(W1 phi_k + b1)
    z     = (1/n) sum_k h_k
    t     = (c(0, sigma_1) + sum_k c(sigma_k, sigma_{k+1}) + c(sigma_n, 0) - m) / sd
            (m, sd given; by default m = 0 and sd = 500 n)
    u     = relu(W2 [z; t] + b2)
    y     = w3 . u + b3
Loss over a batch: mean_b (y_b - target_b)^2. Gradients are the chain rule
written out by hand (`backward`); `tests/test_mlp_reference.py` pins them to
central finite differences of `forward`.
"""
from __future__ import annotations

import numpy as np

H = 256
IN1 = 5
IN2 = H + 1
OFF_W1 = 0
OFF_B1 = OFF_W1 + H * IN1
OFF_W2 = OFF_B1 + H
OFF_B2 = OFF_W2 + H * IN2
OFF_W3 = OFF_B2 + H
OFF_B3 = OFF_W3 + H
NPARAMS = OFF_B3 + 1


def unpack(p):
    p = np.asarray(p, dtype=np.float64)
    return (p[OFF_W1:OFF_B1].reshape(H, IN1), p[OFF_B1:OFF_W2], p[OFF_W2:OFF_B2].reshape(H, IN2),
            p[OFF_B2:OFF_W3], p[OFF_W3:OFF_B3], p[OFF_B3])


def to_bf16(x):
    """Round float32 values to bfloat16 (round to nearest, ties to even) and
    return them as float64."""
    b = np.asarray(x, dtype=np.float32).view(np.uint32).astype(np.uint64)
    r = ((b + 0x7FFF + ((b >> 16) & 1)) >> 16) << 16
    return r.astype(np.uint32).view(np.float32).astype(np.float64)


def to_bf16_pair(x):
    """hi + lo with hi = bf16(v), lo = bf16(v - hi), v = float32(x): the two
    bfloat16 numbers a feature is carried as (about 16 significant bits)."""
    v = np.asarray(x, dtype=np.float32).astype(np.float64)
    hi = to_bf16(v)
    return hi + to_bf16(v - hi)


def features(tours, cust, dist, Q, len_mean=0.0, len_sd=None):
    """phi [T][n][5] and t [T] for tours [T][n] (customer ids 1..n)."""
    tours = np.asarray(tours, dtype=np.int64)
    cust = np.asarray(cust, dtype=np.float64)
    dist = np.asarray(dist, dtype=np.float64)
    T, n = tours.shape
    c = cust[tours - 1]                                   # [T][n][4]
    mu = c[:, :, 2] / Q
    cum = np.cumsum(mu, axis=1)
    phi = np.stack([c[:, :, 0] / 1000.0, c[:, :, 1] / 1000.0, mu, c[:, :, 3] / Q, cum - np.floor(cum)], axis=2)
    legs = dist[0, tours[:, 0]] + dist[tours[:, -1], 0] + dist[tours[:, :-1], tours[:, 1:]].sum(axis=1)
    return phi, (legs - len_mean) / (500.0 * n if len_sd is None else len_sd)


def forward(p, phi, t, bf16=False):
    """Network outputs and the intermediates the backward pass needs. With
    bf16 the weights are rounded to bfloat16 and the per-position features
    replaced by their bfloat16 pairs (the library's operands); everything else
    stays float64."""
    W1, b1, W2, b2, w3, b3 = unpack(p)
    if bf16:
        W1, b1, W2, b2, w3 = (to_bf16(a) for a in (W1, b1, W2, b2, w3))
        b3 = to_bf16(np.array([b3]))[0]
        phi = to_bf16_pair(phi)
    pre = np.einsum("tkf,jf->tkj", phi, W1) + b1          # [T][n][H]
    z = np.maximum(pre, 0.0).mean(axis=1)                # [T][H]
    zt = np.concatenate([z, t[:, None]], axis=1)          # [T][H+1]
    v = zt @ W2.T + b2
    u = np.maximum(v, 0.0)
    y = u @ w3 + b3
    return y, dict(pre=pre, zt=zt, v=v, u=u, W2=W2, w3=w3)


def loss_and_grad(p, phi, t, target, bf16=False):
    y, c = forward(p, phi, t, bf16)
    if bf16:
        phi = to_bf16_pair(phi)
    T, n, _ = phi.shape
    err = y - np.asarray(target, dtype=np.float64)
    loss = float((err ** 2).mean())
    dy = 2.0 * err / T
    g = np.zeros(NPARAMS)
    g[OFF_W3:OFF_B3] = dy @ c["u"]
    g[OFF_B3] = dy.sum()
    du = np.outer(dy, c["w3"]) * (c["v"] > 0)
    g[OFF_W2:OFF_B2] = (du.T @ c["zt"]).reshape(-1)
    g[OFF_B2:OFF_W3] = du.sum(axis=0)
    dzt = du @ c["W2"]
    dpre = (dzt[:, None, :H] / n) * (c["pre"] > 0)        # [T][n][H]
    g[OFF_W1:OFF_B1] = np.einsum("tkj,tkf->jf", dpre, phi).reshape(-1)
    g[OFF_B1:OFF_W2] = dpre.sum(axis=(0, 1))
    return loss, g, y
