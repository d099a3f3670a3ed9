"""Pins of the FP64 reference network of the learned criterion: its gradient against central
finite differences of its loss, and its bfloat16 rounding against the format's definition."""
import numpy as np

from oracle import mlp


def _params(seed=0):
    rng = np.random.default_rng(seed)
    flat = np.zeros(mlp.N_PARAMS)
    flat[:mlp.N_WEIGHTS] = 0.3 * rng.standard_normal(mlp.N_WEIGHTS)
    p = mlp.unpack(flat)
    p["mean"][:] = rng.standard_normal(8)
    p["inv_std"][:] = 0.5 + rng.random(8)
    return mlp.pack(p)


def test_gradient_matches_central_differences():
    rng = np.random.default_rng(1)
    flat = _params(1)
    feats = rng.standard_normal((40, 8))
    labels = rng.standard_normal(40)
    g = mlp.grad(flat, feats, labels)
    idx = rng.choice(mlp.N_WEIGHTS, 60, replace=False)
    h = 1e-6
    for i in idx:
        fp, fm = flat.copy(), flat.copy()
        fp[i] += h
        fm[i] -= h
        fd = (mlp.loss(fp, feats, labels) - mlp.loss(fm, feats, labels)) / (2 * h)
        assert abs(fd - g[i]) <= 1e-6 * max(1.0, abs(g[i])) + 1e-9


def test_zero_network_predicts_the_output_bias():
    flat = np.zeros(mlp.N_PARAMS)
    p = mlp.unpack(flat)
    p["b4"][0] = -3.25
    p["inv_std"][:] = 1.0
    y, _ = mlp.forward(mlp.pack(p), np.ones((5, 8)))
    assert np.all(y == -3.25)


def test_bf16_rounding():
    # bfloat16 keeps 8 significand bits: 1 + 2^-8 is a tie and rounds to even (1.0); 1 + 3*2^-8 rounds up
    v = np.array([1.0, 1.0 + 2.0 ** -8, 1.0 + 3 * 2.0 ** -8, -2.5, 3.0e38])
    r = mlp.bf16(v)
    assert r[0] == 1.0 and r[1] == 1.0 and r[2] == 1.0 + 2.0 ** -6 and r[3] == -2.5
    assert np.all(np.abs(r[:4] - v[:4]) <= 2.0 ** -8 * np.abs(v[:4]))
