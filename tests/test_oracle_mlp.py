"""Pins of the CPU oracle of the learned predictor's MLP: bf16 rounding
against torch's bfloat16 conversion (a library routine), the fp64 gradient
against central finite differences, closed-form special cases, and the bf16
gradient against the fp64 one within bf16 precision."""
import numpy as np
import pytest

from oracle import mlp


def test_bf16_round_matches_torch():
    torch = pytest.importorskip("torch")
    rng = np.random.default_rng(0)
    vals = np.concatenate([rng.normal(0, 1, 4000), rng.normal(0, 1e-3, 1000), rng.normal(0, 1e4, 1000),
                           [0.0, -0.0, 1.0, 1.00390625, 1.005859375, 1.0 + 2**-9, -3.14159, 65504.0, 1e-30]])
    want = torch.tensor(vals, dtype=torch.float32).to(torch.bfloat16).to(torch.float64).numpy()
    assert np.array_equal(mlp.bf16_round(vals), want)


def test_fp64_gradient_matches_finite_differences():
    rng = np.random.default_rng(1)
    p = mlp.init_params(3).astype(np.float64)
    p[mlp._SL["b1"][0]:mlp._SL["b1"][1]] = rng.normal(0, 0.1, 32)
    p[mlp._SL["b2"][0]:mlp._SL["b2"][1]] = rng.normal(0, 0.1, 32)
    X = rng.normal(0, 1, (24, 8))
    Y = (rng.random(24) < 0.4).astype(np.float64)
    g, _ = mlp.gradient(p, X, Y, bf16=False)
    h = 1e-6
    idx = np.concatenate([rng.choice(mlp.N_PARAMS, 200, replace=False), [mlp.N_PARAMS - 1]])
    for k in idx:
        pp, pm = p.copy(), p.copy()
        pp[k] += h
        pm[k] -= h
        fd = (mlp.bce_loss(mlp.forward(pp, X, False)[0], Y) - mlp.bce_loss(mlp.forward(pm, X, False)[0], Y)) / (2 * h)
        assert abs(fd - g[k]) <= 1e-6 + 1e-5 * abs(fd), (k, fd, g[k])


def test_special_cases():
    p = np.zeros(mlp.N_PARAMS)
    p[-1] = 0.7  # only b3
    rng = np.random.default_rng(2)
    X = rng.normal(0, 1, (50, 8))
    Y = (rng.random(50) < 0.5).astype(np.float64)
    logit, _ = mlp.forward(p, X)
    assert np.all(logit == 0.7)
    g, loss = mlp.gradient(p, X, Y)
    s = 1 / (1 + np.exp(-0.7))
    assert abs(g[-1] - np.mean(s - Y)) < 1e-15
    assert np.all(g[:-1] == 0)
    assert abs(loss - np.mean(-(Y * np.log(s) + (1 - Y) * np.log(1 - s)))) < 1e-12


def test_bf16_gradient_close_to_fp64():
    rng = np.random.default_rng(4)
    p = mlp.init_params(5)
    X = rng.normal(0, 1, (256, 8))
    Y = (rng.random(256) < 0.3).astype(np.float64)
    g64, l64 = mlp.gradient(p, X, Y, bf16=False)
    g16, l16 = mlp.gradient(p, X, Y, bf16=True)
    assert abs(l64 - l16) < 2e-2 * max(1.0, l64)
    assert np.linalg.norm(g16 - g64) <= 3e-2 * np.linalg.norm(g64)
