"""Training data and training of the learned vertex-activity predictor.

Traces come from plain runs of the library with trace recording on: each
sample is the 8-feature vector a vertex had when it was selected for
evaluation and whether it then moved.  Only vertices of at least
MIN_DEGREE entries are recorded, the same vertices the predictor later
decides for: skipping pays only where a re-evaluation scans a long row, and
below that degree the inference would cost about as much as the scan.
Training uses the library's own tensor-core kernels (louvain_mlp_train,
Adam on the mean binary cross-entropy).  The default model is trained on
R-MAT graphs of scales 20, 21 and 22 (seeds 101, 102, 103; edge factor 16)
and stored next to this file, with the settings it is meant for, by running
``python -m paper_2501_19004_gb300.predictor``.
"""
from __future__ import annotations

import json
import os
import sys
import time

import numpy as np

from . import graphgen as gg
from . import louvain as lv

HERE = os.path.dirname(os.path.abspath(__file__))
MODEL_FILE = os.path.join(HERE, "predictor_rmat20-22.f32")
TRAINING_GRAPHS = ((20, 101), (21, 102), (22, 103))
MIN_DEGREE = 1024
# run settings the stored model is meant for (louvain_config fields)
SETTINGS = dict(learned_min_degree=MIN_DEGREE, skip_threshold=0.2, learned_fallback=3, learned_skip_clears=1)


def collect_traces(graph, cap: int = 4_000_000, rate: float = 0.25, min_degree: int = 0):
    """(features [k][8] float32, labels [k] float32) from one plain run; with
    min_degree only vertices of at least that degree are recorded."""
    import torch
    cfg = lv.Config(trace_capacity=cap, trace_rate=rate, learned_min_degree=min_degree)
    with lv.Louvain(lv.DeviceCSR.from_host(graph), cfg) as ctx:
        ctx.run()
        X, Y = lv.louvain_traces(ctx.ctx, cap)
    torch.cuda.synchronize()
    return X, Y


def initial_params(seed: int = 0) -> np.ndarray:
    """He-initialised weights (seeded numpy), zero biases."""
    rng = np.random.default_rng(seed)
    p = np.zeros(lv.louvain_model_size(), dtype=np.float32)
    p[0:256] = rng.normal(0, np.sqrt(2.0 / 8), 256)
    p[288:1312] = rng.normal(0, np.sqrt(2.0 / 32), 1024)
    p[1344:1376] = rng.normal(0, np.sqrt(1.0 / 32), 32)
    return p


def train(X, Y, epochs: int = 8, batch: int = 8192, lr: float = 3e-3, seed: int = 0):
    """Adam training on the device; returns (params float32, per-epoch losses)."""
    import torch
    p = torch.from_numpy(initial_params(seed)).cuda()
    losses = lv.louvain_mlp_train(p, torch.from_numpy(np.ascontiguousarray(X)).cuda(),
                                  torch.from_numpy(np.ascontiguousarray(Y)).cuda(), epochs=epochs, batch=batch,
                                  lr=lr, seed=seed)
    return p.cpu().numpy(), losses


def train_default(epochs: int = 30, verbose: bool = False):
    Xs, Ys = [], []
    for scale, seed in TRAINING_GRAPHS:
        t0 = time.time()
        g = gg.rmat(scale, 16, seed=seed)
        X, Y = collect_traces(g, rate=1.0, min_degree=MIN_DEGREE)
        Xs.append(X)
        Ys.append(Y)
        if verbose:
            print(f"scale {scale}: {X.shape[0]} samples, moved {Y.mean():.3f} ({time.time() - t0:.1f} s)",
                  file=sys.stderr)
    X = np.concatenate(Xs)
    Y = np.concatenate(Ys)
    params, losses = train(X, Y, epochs=epochs, batch=2048)
    info = {"samples": int(X.shape[0]), "positive_rate": float(Y.mean()), "losses": [float(v) for v in losses],
            "graphs": [f"rmat{s}-ef16-seed{sd}" for s, sd in TRAINING_GRAPHS], "settings": SETTINGS}
    return params, info


def load_default():
    """The stored default model, or None."""
    if not os.path.exists(MODEL_FILE):
        return None
    p = np.fromfile(MODEL_FILE, dtype=np.float32)
    return p if p.shape[0] == lv.louvain_model_size() else None


def default_config(model=None, **over) -> "lv.Config":
    """A learned-mode Config with the stored model and the settings it was
    trained for (keyword arguments override them)."""
    kw = dict(SETTINGS)
    kw.update(over)
    return lv.Config(mode=lv.MODE_LEARNED, model=load_default() if model is None else model, **kw)


if __name__ == "__main__":
    out = sys.argv[1] if len(sys.argv) > 1 else MODEL_FILE
    params, info = train_default(verbose=True)
    params.astype(np.float32).tofile(out)
    with open(out + ".json", "w") as f:
        json.dump(info, f, indent=1)
    print(json.dumps(info))
