"""CPU oracle of the learned vertex-activity predictor (8 -> 32 -> 32 -> 1 MLP).

TEST INFRASTRUCTURE ONLY (tests, smoke check, CPU baseline); the product path
never imports it and it shares no code with the CUDA kernels.

The paper has no predictor; its definition is the library's, written out
in include/louvain.h (above louvain_mlp_forward): parameters W1[8][32],
b1[32], W2[32][32], b2[32], w3[32], b3 in one flat float vector; the
inputs, the weights and the hidden ReLU outputs are rounded to bf16 (round
to nearest even) and products are summed exactly here (fp64; the device
sums in fp32).  Loss: mean binary cross-entropy of sigmoid(logit).  The
backward pass restates the header's definition: of the back-propagated
deltas exactly two are rounded to bf16, dz2 where it enters dW2 = h1^T dz2
and dh1 = dz2 W2^T, and dz1 where it enters dW1 = x^T dz1; bias and w3
gradients use the unrounded deltas.  With bf16=False everything is plain
fp64 (used to pin the gradient against finite differences).
"""
from __future__ import annotations

import numpy as np

N_PARAMS = 8 * 32 + 32 + 32 * 32 + 32 + 32 + 1
_SL = {
    "W1": (0, 256, (8, 32)),
    "b1": (256, 288, (32,)),
    "W2": (288, 1312, (32, 32)),
    "b2": (1312, 1344, (32,)),
    "w3": (1344, 1376, (32,)),
    "b3": (1376, 1377, ()),
}


def unpack(p):
    p = np.asarray(p, dtype=np.float64)
    out = {}
    for k, (a, b, shp) in _SL.items():
        out[k] = p[a:b].reshape(shp) if shp else p[a]
    return out


def pack(d):
    p = np.zeros(N_PARAMS, dtype=np.float64)
    for k, (a, b, shp) in _SL.items():
        p[a:b] = np.asarray(d[k], dtype=np.float64).reshape(-1)
    return p


def bf16_round(a):
    """Round to the nearest bfloat16 (ties to even), returned as float64.
    Implemented on the float32 bit pattern: keep the high 16 bits after adding
    0x7FFF plus the lowest kept bit."""
    a32 = np.ascontiguousarray(np.asarray(a, dtype=np.float32))
    bits = a32.view(np.uint32).astype(np.uint64)
    lsb = (bits >> np.uint64(16)) & np.uint64(1)
    r = ((bits + np.uint64(0x7FFF) + lsb) & np.uint64(0xFFFF0000)).astype(np.uint32)
    return r.view(np.float32).astype(np.float64)


def forward(params, X, bf16: bool = True):
    """Logits of the rows of X [n][8]; also returns the intermediates."""
    P = unpack(params)
    X = np.asarray(X, dtype=np.float64)
    rb = bf16_round if bf16 else (lambda a: np.asarray(a, dtype=np.float64))
    xb, W1, W2, w3 = rb(X), rb(P["W1"]), rb(P["W2"]), rb(P["w3"])
    z1 = xb @ W1 + P["b1"]
    h1 = rb(np.maximum(z1, 0.0))
    z2 = h1 @ W2 + P["b2"]
    h2 = rb(np.maximum(z2, 0.0))
    logit = h2 @ w3 + P["b3"]
    return logit, dict(xb=xb, W1=W1, W2=W2, w3=w3, z1=z1, h1=h1, z2=z2, h2=h2)


def bce_loss(logit, Y):
    """Mean binary cross-entropy of sigmoid(logit) (numerically stable form)."""
    logit = np.asarray(logit, dtype=np.float64)
    Y = np.asarray(Y, dtype=np.float64)
    return float(np.mean(np.maximum(logit, 0) - logit * Y + np.log1p(np.exp(-np.abs(logit)))))


def gradient(params, X, Y, bf16: bool = True):
    """(gradient vector, mean loss) of the mean BCE over the rows of X."""
    X = np.asarray(X, dtype=np.float64)
    Y = np.asarray(Y, dtype=np.float64)
    n = X.shape[0]
    rb = bf16_round if bf16 else (lambda a: np.asarray(a, dtype=np.float64))
    logit, c = forward(params, X, bf16)
    p = 1.0 / (1.0 + np.exp(-logit))
    dl = (p - Y) / n
    g = {}
    g["b3"] = dl.sum()
    g["w3"] = c["h2"].T @ dl
    dz2 = dl[:, None] * c["w3"][None, :] * (c["z2"] > 0)
    g["b2"] = dz2.sum(0)
    dz2b = rb(dz2)
    g["W2"] = c["h1"].T @ dz2b
    dh1 = dz2b @ c["W2"].T
    dz1 = dh1 * (c["z1"] > 0)
    g["b1"] = dz1.sum(0)
    g["W1"] = c["xb"].T @ rb(dz1)
    return pack(g), bce_loss(logit, Y)


def init_params(seed: int = 0, scale: float = 1.0):
    """He-style random initial parameters from a seeded numpy generator."""
    rng = np.random.default_rng(seed)
    d = {
        "W1": rng.normal(0, scale * np.sqrt(2.0 / 8), (8, 32)),
        "b1": np.zeros(32),
        "W2": rng.normal(0, scale * np.sqrt(2.0 / 32), (32, 32)),
        "b2": np.zeros(32),
        "w3": rng.normal(0, scale * np.sqrt(1.0 / 32), 32),
        "b3": 0.0,
    }
    return pack(d).astype(np.float32)

