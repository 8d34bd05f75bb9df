"""Pins of the oracle MLP: bfloat16 rounding, features, float64 gradients
against central finite differences, and that Adam training fits a seeded
synthetic function better than a constant."""
import math

import numpy as np
import pytest

import workloads as W
from workloads.synth import SyntheticGPU
from oracle import mlp, space


def test_bf16_rounding():
    x = np.float32([1.0, 1.0 + 2 ** -8, 1.0 + 2 ** -7, 1.0 + 3 * 2 ** -8, -2.5, 0.0, 65504.0])
    r = mlp.bf16(x)
    # 1 + 2^-8 is a tie -> even (1.0); 1 + 3*2^-8 is a tie -> even (1 + 2^-6)
    assert list(r) == [1.0, 1.0, 1.0 + 2 ** -7, 1.0 + 2 ** -6, -2.5, 0.0, 65536.0]
    y = np.random.default_rng(0).standard_normal(1000).astype(np.float32)
    rb = mlp.bf16(y)
    assert np.all(rb.view(np.uint32) & 0xFFFF == 0)
    assert np.all(np.abs(rb - y) <= np.abs(y) * 2 ** -8)


def test_features():
    vals = [[1, 2, 4], [7], [0, 1]]
    x = mlp.features(vals, [[2, 0, 1], [0, 0, 0]])
    assert x.shape == (2, 16)
    np.testing.assert_array_equal(x[0, :6], [0, 0, 1, 1, 0, 1])
    np.testing.assert_array_equal(x[1, :6], [1, 0, 0, 1, 1, 0])
    assert x[0, 6] == 1.0 and x[1, 6] == -1.0 and x[0, 7] == 0.0 and x[0, 8] == 1.0


def test_gelu_against_closed_form():
    z = np.linspace(-4, 4, 41)
    ref = np.array([0.5 * v * (1 + math.erf(v / math.sqrt(2))) for v in z])
    np.testing.assert_allclose(mlp.gelu(z), ref, rtol=1e-14, atol=1e-15)
    h = 1e-6
    fd = (mlp.gelu(z + h) - mlp.gelu(z - h)) / (2 * h)
    np.testing.assert_allclose(mlp.gelu_grad(z), fd, rtol=1e-7, atol=1e-9)


def test_gradients_match_finite_differences():
    rng = np.random.default_rng(1)
    F, K, n = 16, 5, 7
    p = mlp.init_params(F, K, seed=3)
    for k in p:
        p[k] = p[k].astype(np.float64)
        if k.startswith("b"):
            p[k] = rng.standard_normal(p[k].shape) * 0.1
    x = rng.standard_normal((n, F))
    t = rng.standard_normal((n, K))
    _, g = mlp.loss_and_grads(p, x, t, mode="f64")
    h = 1e-6
    for name in ("W1", "b1", "W2", "b3", "W4", "b4"):
        for _ in range(6):
            idx = tuple(int(rng.integers(0, s)) for s in p[name].shape)
            old = p[name][idx]
            p[name][idx] = old + h
            lp = mlp.loss_and_grads(p, x, t, mode="f64")[0]
            p[name][idx] = old - h
            lm = mlp.loss_and_grads(p, x, t, mode="f64")[0]
            p[name][idx] = old
            fd = (lp - lm) / (2 * h)
            assert abs(g[name][idx] - fd) <= 1e-6 * max(1.0, abs(fd)), (name, idx, g[name][idx], fd)


def test_bf16_path_close_to_f64():
    rng = np.random.default_rng(2)
    F, K, n = 32, 8, 64
    p = mlp.init_params(F, K, seed=5)
    x = mlp.bf16(rng.standard_normal((n, F)).astype(np.float32))
    y16, _ = mlp.forward(p, x)
    y64, _ = mlp.forward(p, x, mode="f64")
    assert np.max(np.abs(y16 - y64)) < 0.05 * np.max(np.abs(y64)) + 0.05


def test_training_fits_synthetic_counters():
    desc = W.space_tiny_block_tile()
    roles = W.layout(16)
    gpu = SyntheticGPU(desc, roles, seed=0)
    valid = space.enumerate_valid(desc)
    dig = space.decode(desc.radices, valid)
    C, _ = gpu.evaluate(dig)
    ranges = gpu.counter_ranges()
    x = mlp.features(desc.values, dig)
    t = (C / ranges).astype(np.float32)
    p = mlp.init_params(x.shape[1], 16, seed=0)
    opt = mlp.Adam(p)
    rng = np.random.default_rng(0)
    base = float(np.mean((t - t.mean(axis=0)) ** 2))
    for _ in range(150):
        b = rng.choice(len(x), size=256, replace=False)
        loss, g = mlp.loss_and_grads(p, x[b], t[b])
        opt.step(p, g)
    y, _ = mlp.forward(p, x)
    final = float(np.mean((y - t) ** 2))
    assert final < 0.5 * base
