"""Learned codec selector workflow: training rows from fields, seeded initial weights,
training on the GPU, and size regret against exhaustive and heuristic selection.

Every numeric step runs in the library's kernels (api.selector_rows, selector_train,
compress); this module only allocates buffers and orders the calls.
"""
from __future__ import annotations

import numpy as np
import torch

from . import api


def init_weights(seed: int, device="cuda") -> torch.Tensor:
    """Seeded uniform (He-style) initial parameters in the packed layout
    W1[32][8] b1[32] W2[32][32] b2[32] W3[3][32] b3[3]; biases start at zero."""
    rng = np.random.default_rng(seed)
    w1 = rng.uniform(-1, 1, (32, 8)) * np.sqrt(6.0 / 8)
    w2 = rng.uniform(-1, 1, (32, 32)) * np.sqrt(6.0 / 32)
    w3 = rng.uniform(-1, 1, (3, 32)) * np.sqrt(6.0 / 32) * 0.1
    flat = np.concatenate([w1.ravel(), np.zeros(32), w2.ravel(), np.zeros(32), w3.ravel(), np.zeros(3)])
    assert flat.size == api.MLP_PARAMS
    return torch.from_numpy(flat.astype(np.float32)).to(device)


def collect_rows(fields, device="cuda"):
    """Training rows of every block of every field, concatenated in field order.
    `fields`: iterable of (CUDA field tensor or zero-argument callable returning one,
    eb, eb_mode).  Callables let the caller generate each field on demand."""
    items = list(fields)
    shapes = []
    for f, _, _ in items:
        shapes.append(tuple(f.shape) if isinstance(f, torch.Tensor) else None)
    parts = []
    for (f, eb, mode), shp in zip(items, shapes):
        x = f if isinstance(f, torch.Tensor) else f()
        parts.append(api.selector_rows(x, eb, mode))
        del x
    out = {k: torch.cat([p[k] for p in parts]) for k in ("feat", "target", "sizes", "valid")}
    return out


def train(rows, seed: int = 0, steps: int = 3000, lr: float = 3e-3):
    """Weights trained by full-batch Adam on the valid rows; returns (weights, loss before,
    loss after)."""
    w = init_weights(seed, rows["feat"].device)
    loss0, _ = api.selector_grad(w, rows["feat"], rows["target"], rows["valid"])
    loss = api.selector_train(w, rows["feat"], rows["target"], rows["valid"], steps=steps, lr=lr)
    loss1, _ = api.selector_grad(w, rows["feat"], rows["target"], rows["valid"])
    return w, loss0, loss1


def evaluate(weights, fields, selectors=("learned", "exhaustive", "heuristic")):
    """Total archive bytes per selector over `fields` ((tensor or callable, eb, mode)),
    and the learned selector's size regret against exhaustive and its gain over the
    paper's heuristic."""
    tot = {s: 0 for s in selectors}
    n_in = 0
    for f, eb, mode in fields:
        x = f if isinstance(f, torch.Tensor) else f()
        n_in += 4 * x.numel()
        for s in selectors:
            _, nb, _ = api.compress(x, eb, mode, select=s, weights=weights if s == "learned" else None)
            tot[s] += nb
        del x
    rep = {"bytes": tot, "input_bytes": n_in}
    if "learned" in tot and "exhaustive" in tot:
        rep["regret_vs_exhaustive"] = tot["learned"] / tot["exhaustive"] - 1.0
    if "learned" in tot and "heuristic" in tot:
        rep["gain_vs_heuristic"] = tot["heuristic"] / tot["learned"] - 1.0
        rep["heuristic_regret_vs_exhaustive"] = (tot["heuristic"] / tot["exhaustive"] - 1.0
                                                 if "exhaustive" in tot else None)
    return rep
