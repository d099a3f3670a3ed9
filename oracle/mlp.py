"""FP64 reference of the learned opening criterion's network -- TEST INFRASTRUCTURE ONLY.

The learned criterion is not in the paper (which uses the fixed-theta test of Sec. 3.1); it
predicts, from 8 features of a (sink cell, source cell) pair, the log10 of the force error that
accepting the pair as a cell-cell interaction would make.

Network: x (8) -> h1 = relu(W1 x + b1) (64) -> h2 = relu(W2 h1 + b2) (64)
         -> h3 = relu(W3 h2 + b3) (64) -> y = w4 . h3 + b4.
Loss: mean squared error 0.5 * mean((y - label)^2).

Flat parameter layout (shared with the C ABI, float32 there):
    W1 [64 x 8] row-major, b1 [64], W2 [64 x 64], b2 [64], W3 [64 x 64], b3 [64], w4 [64], b4 [1]
    followed by the feature normalisation: mean [8], inv_std [8]  (x = (f - mean) * inv_std),
    and N_SUR floats of a surrogate bound that only the walk uses (zero here).
"""
from __future__ import annotations

import numpy as np

H = 64
F = 8
SIZES = [("W1", (H, F)), ("b1", (H,)), ("W2", (H, H)), ("b2", (H,)), ("W3", (H, H)), ("b3", (H,)),
         ("w4", (H,)), ("b4", (1,))]
N_WEIGHTS = sum(int(np.prod(s)) for _, s in SIZES)  # 8961
N_SUR = 12  # the surrogate bound (alpha, beta, r_lo, r_hi, gamma[8]), which only the walk uses
N_PARAMS = N_WEIGHTS + 2 * F + N_SUR


def unpack(flat):
    flat = np.asarray(flat, dtype=np.float64)
    out, o = {}, 0
    for name, shape in SIZES:
        k = int(np.prod(shape))
        out[name] = flat[o:o + k].reshape(shape)
        o += k
    out["mean"] = flat[o:o + F]
    out["inv_std"] = flat[o + F:o + 2 * F]
    out["surrogate"] = flat[o + 2 * F:o + 2 * F + N_SUR]
    return out


def pack(p):
    sur = np.asarray(p.get("surrogate", np.zeros(N_SUR)), dtype=np.float64)
    return np.concatenate([np.asarray(p[name], dtype=np.float64).reshape(-1) for name, _ in SIZES] +
                          [np.asarray(p["mean"], dtype=np.float64), np.asarray(p["inv_std"], dtype=np.float64), sur])


def forward(flat, feats):
    """feats (B, 8) raw features -> predictions (B,), with the activations for backward."""
    p = unpack(flat)
    x = (np.asarray(feats, dtype=np.float64) - p["mean"]) * p["inv_std"]
    z1 = x @ p["W1"].T + p["b1"]
    h1 = np.maximum(z1, 0.0)
    z2 = h1 @ p["W2"].T + p["b2"]
    h2 = np.maximum(z2, 0.0)
    z3 = h2 @ p["W3"].T + p["b3"]
    h3 = np.maximum(z3, 0.0)
    y = h3 @ p["w4"] + p["b4"][0]
    return y, (x, z1, h1, z2, h2, z3, h3)


def loss(flat, feats, labels):
    y, _ = forward(flat, feats)
    r = y - np.asarray(labels, dtype=np.float64)
    return 0.5 * float(np.mean(r * r))


def grad(flat, feats, labels):
    """Gradient of the loss with respect to the network weights (first N_WEIGHTS entries)."""
    p = unpack(flat)
    y, (x, z1, h1, z2, h2, z3, h3) = forward(flat, feats)
    B = y.shape[0]
    dy = (y - np.asarray(labels, dtype=np.float64)) / B
    g = {"w4": h3.T @ dy, "b4": np.array([dy.sum()])}
    d3 = np.outer(dy, p["w4"]) * (z3 > 0)
    g["W3"] = d3.T @ h2
    g["b3"] = d3.sum(axis=0)
    d2 = (d3 @ p["W3"]) * (z2 > 0)
    g["W2"] = d2.T @ h1
    g["b2"] = d2.sum(axis=0)
    d1 = (d2 @ p["W2"]) * (z1 > 0)
    g["W1"] = d1.T @ x
    g["b1"] = d1.sum(axis=0)
    return np.concatenate([g[name].reshape(-1) for name, _ in SIZES])


def bf16(a):
    """Round to bfloat16 (nearest even) and back to float64."""
    a32 = np.asarray(a, dtype=np.float32)
    u = a32.view(np.uint32).astype(np.uint64)
    r = ((u + 0x7FFF + ((u >> 16) & 1)) >> 16) << 16
    return r.astype(np.uint32).view(np.float32).astype(np.float64)


def forward_bf16(flat, feats):
    """Inference as the tensor-core path computes it: normalised inputs, weights and hidden
    activations rounded to bfloat16, products accumulated in higher precision, biases in FP32."""
    p = unpack(flat)
    x = bf16((np.asarray(feats, dtype=np.float32) - p["mean"].astype(np.float32)) * p["inv_std"].astype(np.float32))
    h = x
    for W, b in (("W1", "b1"), ("W2", "b2"), ("W3", "b3")):
        h = bf16(np.maximum(h @ bf16(p[W]).T + p[b], 0.0))
    return h @ bf16(p["w4"]) + p["b4"][0]
