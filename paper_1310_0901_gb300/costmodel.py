"""Fitting the learned batch-split cost model.

cg_tune_batch measures, for one batch, the level-kernel time of every
candidate segment size (dry runs, the shadow is untouched).  Measurements
over many batches give samples (batch features, log2 segment KiB) ->
log2 ms, on which the network is fitted with the library's own GPU kernels
(cg_mlp_fit).  Installed with Context.set_cost_model, it picks the split of
batches that no tuned entry matches.
"""
from __future__ import annotations

import numpy as np

from . import CANDIDATES_KIB, batch_features, mlp_fit


def measure(ctx, batches, repeats: int = 2) -> list[dict]:
    """Per batch: its features and the dry-run ms of every candidate."""
    out = []
    for reqs in batches:
        _, ms = ctx.tune_batch(reqs, CANDIDATES_KIB, repeats, remember=False)
        out.append({"features": batch_features(reqs), "ms": ms})
    return out


def samples(measured: list[dict]) -> tuple[np.ndarray, np.ndarray]:
    """Targets are log2 ms relative to the batch's mean over the candidates:
    only the shape over segment sizes decides the choice, and removing each
    batch's overall scale keeps it from dominating the fit."""
    xs, ts = [], []
    for m in measured:
        logs = {k: np.log2(max(v, 1e-3)) for k, v in m["ms"].items()}
        mean = float(np.mean(list(logs.values())))
        for kib, lg in logs.items():
            xs.append(np.concatenate([m["features"], [np.log2(kib)]]))
            ts.append(lg - mean)
    return np.asarray(xs, np.float32), np.asarray(ts, np.float32)


def fit(measured: list[dict], hidden: int = 32, epochs: int = 3000, lr: float = 3e-3,
        seed: int = 0):
    x, t = samples(measured)
    return mlp_fit(x, t, hidden, epochs, lr, seed)


def predict(weights: np.ndarray, features: np.ndarray, kib: int, hidden: int) -> float:
    """The installed model's prediction (the same arithmetic the library
    uses to choose; here only for reporting)."""
    d = len(features) + 1
    mu, sd = weights[:d], weights[d:2 * d]
    o = 2 * d
    W1 = weights[o:o + d * hidden].reshape(d, hidden)
    b1 = weights[o + d * hidden:o + d * hidden + hidden]
    w2 = weights[o + d * hidden + hidden:o + d * hidden + 2 * hidden]
    b2 = weights[-1]
    x = (np.concatenate([features, [np.log2(kib)]]) - mu) / sd
    return float(np.maximum(x @ W1 + b1, 0) @ w2 + b2)
