"""Float64 reference of the k-th-count predictor network.

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__.py``).  The paper has no
learned component; this network seeds the c-PQ AuditThreshold (Sec. 3.3.1)
with a predicted k-th count.  Definitions used on both sides:

  features  x[b] = scale * #{query keywords with df = 0}                 b = 0
            x[b] = scale * #{query keywords with floor(log2 df) = b - 1}  b >= 1
            (b clipped to 63; df = posting-list length, scale = 1/32)
  network   pre = W1 x + b1 (128), h = relu(pre), y = w2 . h + b2
            W1 128x64, w2 128 held in bfloat16 for the forward pass
  loss      L = (1/B) sum_j 0.5 (y_j - t_j)^2, t = k-th count
  optimiser Adam (Kingma & Ba 2015) on float32 master weights

Everything here runs in float64 on the given (already bf16-rounded) weights.
"""
from __future__ import annotations

import numpy as np

N_FEATURES = 64
N_HIDDEN = 128
FEATURE_SCALE = 1.0 / 32.0


def floor_log2(v: np.ndarray) -> np.ndarray:
    """floor(log2 v) for integers v >= 1, by repeated halving."""
    v = np.asarray(v, dtype=np.uint64).copy()
    out = np.zeros(v.shape, dtype=np.int64)
    while np.any(v > 1):
        big = v > 1
        out += big
        v = np.where(big, v >> np.uint64(1), v)
    return out


def features(df_per_keyword: np.ndarray, q_off: np.ndarray) -> np.ndarray:
    """Histogram features of each query from the df of its keywords."""
    df = np.asarray(df_per_keyword, dtype=np.uint64)
    q_off = np.asarray(q_off, dtype=np.int64)
    bins = np.where(df == 0, 0, np.minimum(floor_log2(np.maximum(df, 1)) + 1, N_FEATURES - 1))
    n_q = len(q_off) - 1
    x = np.zeros((n_q, N_FEATURES), dtype=np.float64)
    for q in range(n_q):
        b = bins[q_off[q]:q_off[q + 1]]
        np.add.at(x[q], b, 1.0)
    return x * FEATURE_SCALE


def bf16_round(a: np.ndarray) -> np.ndarray:
    """Round float32 values to the nearest bfloat16 (ties to even), returned as
    float32.  bfloat16 keeps the top 16 bits of the float32 encoding."""
    a32 = np.asarray(a, dtype=np.float32)
    u = np.ascontiguousarray(a32).reshape(-1).view(np.uint32).astype(np.uint64)
    lsb = (u >> np.uint64(16)) & np.uint64(1)
    r = ((u + np.uint64(0x7FFF) + lsb) & np.uint64(0xFFFF0000)).astype(np.uint32)
    r = np.where(np.isnan(a32.reshape(-1)), np.uint32(0x7FC00000), r)
    return r.view(np.float32).reshape(a32.shape)


def forward(x, W1, b1, w2, b2):
    """Returns (y, cache)."""
    x = np.asarray(x, np.float64)
    pre = x @ np.asarray(W1, np.float64).T + np.asarray(b1, np.float64)
    h = np.maximum(pre, 0.0)
    y = h @ np.asarray(w2, np.float64) + float(b2)
    return y, (x, pre, h)


def loss(y, t) -> float:
    y = np.asarray(y, np.float64)
    t = np.asarray(t, np.float64)
    return float(np.mean(0.5 * (y - t) ** 2))


def backward(y, t, cache, W1, w2):
    """Gradients of ``loss`` w.r.t. (W1, b1, w2, b2)."""
    x, pre, h = cache
    B = len(y)
    dy = (np.asarray(y, np.float64) - np.asarray(t, np.float64)) / B
    g_w2 = h.T @ dy
    g_b2 = float(dy.sum())
    dh = np.outer(dy, np.asarray(w2, np.float64))
    dpre = dh * (pre > 0.0)
    g_W1 = dpre.T @ x
    g_b1 = dpre.sum(axis=0)
    return g_W1, g_b1, g_w2, g_b2


def adam(theta, g, m, v, step, lr=1e-3, beta1=0.9, beta2=0.999, eps=1e-8):
    """One Adam update; returns (theta, m, v).  ``step`` counts from 1."""
    m = beta1 * m + (1.0 - beta1) * g
    v = beta2 * v + (1.0 - beta2) * g * g
    mhat = m / (1.0 - beta1 ** step)
    vhat = v / (1.0 - beta2 ** step)
    return theta - lr * mhat / (np.sqrt(vhat) + eps), m, v
