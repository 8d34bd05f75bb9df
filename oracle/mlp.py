"""The learned counter model: a small MLP surrogate (oracle).

It stands in for the per-counter trees of Section 3.3 (which the paper builds
with regression trees or least-squares models): a function from a
configuration's parameters to its counter vector, fitted on the profiles the
method samples.  Architecture and numerics (the readings of this build):

  features   one-hot digit of every parameter, then the parameter's value
             as u = 2 (log2(1 + v) - lo) / (hi - lo) - 1 in [-1, 1] (0 for a
             one-valued parameter), zero padding to F (a multiple of 16)
  layers     z1 = x W1^T + b1, a1 = GELU(z1); z2, a2; z3, a3 (width 256);
             y = a3 W4^T + b4; prediction = y * range (per counter)
  GELU       erf form, 0.5 z (1 + erf(z / sqrt 2)) (Hendrycks & Gimpel 2016)
  BF16       x, the weights and the activations a1..a3 are rounded to bfloat16
             (round to nearest even); products accumulate in float32; biases,
             pre-activations, y and predictions are float32
  loss       mean over the batch and the K counters of (y - t / range)^2
  backward   g_y = 2 (y - t/range) / (n K); the operands of every backward
             product (g_y, g_z1..g_z3) are rounded to bfloat16; bias gradients
             sum the float32 values; g_z = (g_a) * GELU'(z)
  optimiser  Adam (Kingma & Ba 2015), lr 1e-3, beta (0.9, 0.999), eps 1e-8,
             float32 master weights, bias-corrected moments

``mode="f64"`` runs the same network without any rounding in float64; it is
what the finite-difference pin checks.  Accumulation order differs from the
tensor cores', so GPU parity is within a tolerance, not bit-exact.
"""
from __future__ import annotations

import math
from typing import Dict, List

import numpy as np
from scipy.special import erf

HIDDEN = 256


def bf16(x) -> np.ndarray:
    """Round float32 values to bfloat16 (nearest even), returned as float32."""
    a = np.ascontiguousarray(x, dtype=np.float32)
    u = a.view(np.uint32).astype(np.uint64)
    r = (u + 0x7FFF + ((u >> 16) & 1)) & 0xFFFF0000
    out = r.astype(np.uint32).view(np.float32)
    nan = np.isnan(a)
    if nan.any():
        out = np.where(nan, a, out)
    return out.reshape(np.shape(x))


def u_table(values: List[List[int]]) -> List[np.ndarray]:
    out = []
    for vals in values:
        lv = np.log2(1.0 + np.asarray(vals, dtype=np.float64))
        lo, hi = lv.min(), lv.max()
        out.append(np.zeros_like(lv) if hi == lo else 2.0 * (lv - lo) / (hi - lo) - 1.0)
    return out


def n_features(radices: List[int]) -> int:
    f = sum(radices) + len(radices)
    return (f + 15) // 16 * 16


def features(values: List[List[int]], digits) -> np.ndarray:
    """Feature rows [n, F] (float32, bfloat16-exact)."""
    d = np.atleast_2d(np.asarray(digits, dtype=np.int64))
    radices = [len(v) for v in values]
    F = n_features(radices)
    x = np.zeros((d.shape[0], F), dtype=np.float32)
    off = 0
    rows = np.arange(d.shape[0])
    for j, r in enumerate(radices):
        x[rows, off + d[:, j]] = 1.0
        off += r
    ut = u_table(values)
    for j in range(len(radices)):
        x[:, off + j] = bf16(ut[j][d[:, j]].astype(np.float32))
    return x


def init_params(F: int, K: int, seed: int) -> Dict[str, np.ndarray]:
    """He-style normal initialisation from a seeded generator (float32)."""
    rng = np.random.default_rng([int(seed), 0x3177])
    dims = [(HIDDEN, F), (HIDDEN, HIDDEN), (HIDDEN, HIDDEN), (K, HIDDEN)]
    p = {}
    for i, (o, n_in) in enumerate(dims, 1):
        p["W%d" % i] = (rng.standard_normal((o, n_in)) * math.sqrt(2.0 / n_in)).astype(np.float32)
        p["b%d" % i] = np.zeros(o, dtype=np.float32)
    return p


def gelu(z):
    return 0.5 * z * (1.0 + erf(z / math.sqrt(2.0)))


def gelu_grad(z):
    return 0.5 * (1.0 + erf(z / math.sqrt(2.0))) + z * np.exp(-0.5 * z * z) / math.sqrt(2.0 * math.pi)


def forward(p, x, mode: str = "bf16"):
    """Returns (y, cache).  y: [n, K] float32 (scaled outputs)."""
    if mode == "f64":
        a = np.asarray(x, dtype=np.float64)
        cache = {"a0": a}
        for i in (1, 2, 3):
            z = a @ p["W%d" % i].astype(np.float64).T + p["b%d" % i].astype(np.float64)
            cache["z%d" % i] = z
            a = gelu(z)
            cache["a%d" % i] = a
        y = a @ p["W4"].astype(np.float64).T + p["b4"].astype(np.float64)
        return y, cache
    a = np.asarray(x, dtype=np.float32)
    cache = {"a0": a}
    for i in (1, 2, 3):
        w = bf16(p["W%d" % i]).astype(np.float64)
        z = (a.astype(np.float64) @ w.T).astype(np.float32) + p["b%d" % i]
        cache["z%d" % i] = z
        a = bf16(gelu(z.astype(np.float64)).astype(np.float32))
        cache["a%d" % i] = a
    w4 = bf16(p["W4"]).astype(np.float64)
    y = (a.astype(np.float64) @ w4.T).astype(np.float32) + p["b4"]
    return y, cache


def loss_and_grads(p, x, t_scaled, mode: str = "bf16"):
    """Mean-squared loss on scaled outputs and the gradient of every parameter."""
    y, c = forward(p, x, mode)
    n, K = y.shape
    f64 = mode == "f64"
    dt = np.float64 if f64 else np.float32
    t = np.asarray(t_scaled, dtype=dt)
    diff = y.astype(dt) - t
    loss = float(np.mean(diff.astype(np.float64) ** 2))
    g = (2.0 / (n * K)) * diff
    g = g.astype(dt)
    grads = {}
    rnd = (lambda v: v) if f64 else (lambda v: bf16(v))
    for i in (4, 3, 2, 1):
        a_prev = c["a%d" % (i - 1)]
        gb = rnd(g)
        grads["W%d" % i] = (gb.astype(np.float64).T @ np.asarray(a_prev, dtype=np.float64)).astype(dt)
        grads["b%d" % i] = g.astype(np.float64).sum(axis=0).astype(dt)
        if i > 1:
            w = p["W%d" % i].astype(np.float64) if f64 else bf16(p["W%d" % i]).astype(np.float64)
            ga = (gb.astype(np.float64) @ w).astype(dt)
            z = c["z%d" % (i - 1)]
            g = (ga * gelu_grad(np.asarray(z, dtype=np.float64))).astype(dt)
    return loss, grads


class Adam:
    def __init__(self, params, lr=1e-3, b1=0.9, b2=0.999, eps=1e-8):
        self.lr, self.b1, self.b2, self.eps = lr, b1, b2, eps
        self.m = {k: np.zeros_like(v) for k, v in params.items()}
        self.v = {k: np.zeros_like(v) for k, v in params.items()}
        self.t = 0

    def step(self, params, grads):
        self.t += 1
        c1 = 1.0 - self.b1 ** self.t
        c2 = 1.0 - self.b2 ** self.t
        for k in params:
            g = grads[k].astype(np.float32)
            self.m[k] = (self.b1 * self.m[k] + (1.0 - self.b1) * g).astype(np.float32)
            self.v[k] = (self.b2 * self.v[k] + (1.0 - self.b2) * g * g).astype(np.float32)
            mh = self.m[k] / np.float32(c1)
            vh = self.v[k] / np.float32(c2)
            params[k] = (params[k] - np.float32(self.lr) * mh / (np.sqrt(vh) + np.float32(self.eps))).astype(np.float32)


def predict(p, values, digits, ranges) -> np.ndarray:
    y, _ = forward(p, features(values, digits))
    return (y * np.asarray(ranges, dtype=np.float32)).astype(np.float32)
