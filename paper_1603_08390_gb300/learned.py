"""Learned AuditThreshold seeds: data, training and calibration driver.

The k-th-count network (``genie_mlp_*`` in the C ABI) is trained on pairs
(query features -> k-th match count) that the plain search produces, then
seeds the Gate of the seeded search.  Everything that touches a query or a
weight runs in libgenie.so; this module only sequences the calls and picks
the safety margin from held-out predictions.
"""
from __future__ import annotations

from typing import Optional

import numpy as np
import torch

from . import genie, runner


def kth_counts(res: dict, k: int) -> np.ndarray:
    """t_k per query from a search result: the count at rank k, 0 if fewer
    than k objects matched."""
    return np.where(res["n_valid"] >= k, res["counts"][:, k - 1], 0).astype(np.float32)


def training_pairs(index: genie.Index, q_off: np.ndarray, q_kw: np.ndarray, k: int,
                   batch: int = 4096):
    """Features (device, [n, 64] float32) and k-th counts (device, [n]) of the
    given queries, computed by the plain search in batches."""
    n = len(q_off) - 1
    feats = torch.empty((n, genie.N_FEATURES), dtype=torch.float32, device="cuda")
    targets = np.empty(n, dtype=np.float32)
    q_off = q_off.astype(np.int64)
    for a in range(0, n, batch):
        b = min(n, a + batch)
        off = (q_off[a:b + 1] - q_off[a]).astype(np.uint32)
        kw = q_kw[q_off[a]:q_off[b]]
        qs = genie.genie_make_queries(index, runner.to_dev(off), runner.to_dev(kw), b - a)
        out = runner.search(index, qs, k)
        genie.genie_queries_export(qs, d_features=feats[a:b])
        targets[a:b] = kth_counts(out.host(), k)
        qs.close()
    return feats, torch.from_numpy(targets).cuda()


def calibrate_margin(mlp: genie.MLP, feats: torch.Tensor, targets: torch.Tensor,
                     fail_rate: float = 0.01) -> float:
    """Smallest margin whose seeds floor(y - margin) exceed the true k-th count
    on at most ``fail_rate`` of the held-out queries (an over-high seed costs a
    rerun; a low one only costs Gate work)."""
    n = feats.shape[0]
    y = torch.empty(n, dtype=torch.float32, device="cuda")
    mlp.forward(feats, n, y)
    torch.cuda.synchronize()
    excess = (y.cpu().numpy().astype(np.float64) - targets.cpu().numpy() - 1.0)
    # seed > t  <=>  floor(y - m) >= t + 1  <=>  m <= y - t - 1
    return float(max(0.0, np.quantile(excess, 1.0 - fail_rate) + 1e-3))


def train_predictor(index: genie.Index, train_q_off: np.ndarray, train_q_kw: np.ndarray, k: int,
                    epochs: int = 30, batch: int = 256, lr: float = 2e-3, seed: int = 7,
                    holdout: float = 0.1, fail_rate: float = 0.01) -> dict:
    """Label training queries with the plain search, train the network on the
    GPU and calibrate its margin on a held-out slice."""
    feats, targets = training_pairs(index, train_q_off, train_q_kw, k)
    n = feats.shape[0]
    n_val = max(1, int(n * holdout))
    n_tr = n - n_val
    mlp = genie.MLP(seed)
    loss = mlp.train(feats[:n_tr], targets[:n_tr], n_tr, epochs, batch, lr)
    margin = calibrate_margin(mlp, feats[n_tr:], targets[n_tr:], fail_rate)
    return {"mlp": mlp, "train_loss": loss, "margin": margin, "n_train": n_tr, "n_val": n_val,
            "target_mean": float(targets.mean().item())}


def seeded_search(index: genie.Index, queries: genie.Queries, mlp: genie.MLP, margin: float, k,
                  stats: Optional[torch.Tensor] = None, out: Optional[runner.Outputs] = None,
                  stream=None) -> runner.Outputs:
    """Seeds from the network, then the exact seeded search (verify + rerun)."""
    seeds = torch.empty(queries.n_queries, dtype=torch.int32, device="cuda")
    mlp.seeds(queries, margin, seeds, stream)
    opts = genie.make_opts(d_seed=seeds, d_stats=stats)
    return runner.search(index, queries, k, opts=opts, out=out, stream=stream)
