"""Regression trees (oracle; test infrastructure).

Section 3.3.2: one regression tree per counter, built top-down and greedily
(ID3 with standard-deviation reduction, equivalently the largest drop of the
sum of squared errors), nodes testing tuning parameters, leaves holding the
predicted counter value.

Readings (the paper allows "two or more branches"): binary splits on the
ordinal digit, "digit > threshold" goes right; split score = SSE reduction in
float64; ties go to the lowest feature, then the lowest threshold; a node
becomes a leaf at the depth limit, when it holds one sample, when its targets
are all equal, or when no split separates its samples; the leaf value is the
float64 mean rounded to float32.

Parity: prediction is exact (integer compares, stored float32 leaves); pinned
by hand-traced trees.  The fitter is pinned by exact recovery of
piecewise-constant targets and by brute force on tiny inputs.
"""
from __future__ import annotations

from typing import List

import numpy as np


def predict_tree(tree: dict, digits: np.ndarray) -> np.ndarray:
    """Follow child pointers from the root until a leaf, for every row."""
    d = np.atleast_2d(np.asarray(digits, dtype=np.int64))
    node = np.zeros(d.shape[0], dtype=np.int64)
    feat, thr = tree["feature"], tree["threshold"]
    left, right = tree["left"], tree["right"]
    rows = np.arange(d.shape[0])
    while True:
        inner = feat[node] >= 0
        if not inner.any():
            break
        f = np.where(inner, feat[node], 0)
        go_right = d[rows, f] > thr[node]
        nxt = np.where(go_right, right[node], left[node])
        node = np.where(inner, nxt, node)
    return tree["value"][node].astype(np.float32)


def predict(model: dict, digits: np.ndarray) -> np.ndarray:
    """Counter vectors [n, K] (float32) of the given digit rows."""
    d = np.atleast_2d(np.asarray(digits, dtype=np.int64))
    return np.stack([predict_tree(t, d) for t in model["trees"]], axis=1)


def _sse(y: np.ndarray) -> float:
    if y.size == 0:
        return 0.0
    m = y.mean()
    return float(((y - m) ** 2).sum())


def fit_tree(digits: np.ndarray, y: np.ndarray, depth: int, radices: List[int]) -> dict:
    """Greedy CART on ordinal digits (see module docstring for the rules)."""
    d = np.atleast_2d(np.asarray(digits, dtype=np.int64))
    y = np.asarray(y, dtype=np.float64)
    feat, thr, left, right, val = [], [], [], [], []

    def new():
        feat.append(-1); thr.append(0); left.append(-1); right.append(-1); val.append(0.0)
        return len(feat) - 1

    def build(idx: np.ndarray, level: int) -> int:
        i = new()
        yy = y[idx]
        val[i] = float(np.float32(yy.mean()))
        if level == depth or idx.size <= 1 or np.all(yy == yy[0]):
            return i
        parent = _sse(yy)
        best = None
        for f in range(d.shape[1]):
            col = d[idx, f]
            for t in range(radices[f] - 1):
                m = col > t
                nr = int(m.sum())
                if nr == 0 or nr == idx.size:
                    continue
                gain = parent - (_sse(yy[~m]) + _sse(yy[m]))
                if best is None or gain > best[0]:
                    best = (gain, f, t)
        if best is None:
            return i
        _, f, t = best
        m = d[idx, f] > t
        feat[i], thr[i] = f, t
        li = build(idx[~m], level + 1)
        ri = build(idx[m], level + 1)
        left[i], right[i] = li, ri
        return i

    build(np.arange(d.shape[0]), 0)
    return {"feature": np.asarray(feat, np.int32), "threshold": np.asarray(thr, np.int32),
            "left": np.asarray(left, np.int32), "right": np.asarray(right, np.int32),
            "value": np.asarray(val, np.float32)}


def fit_model(digits, Y, depth: int, radices: List[int], roles: List[int]) -> dict:
    Y = np.asarray(Y)
    return {"roles": list(roles), "depth": int(depth),
            "trees": [fit_tree(digits, Y[:, k], depth, radices) for k in range(Y.shape[1])]}


def tree_depth(tree: dict) -> int:
    """Longest root-to-leaf path length (edges)."""
    def rec(i):
        if tree["feature"][i] < 0:
            return 0
        return 1 + max(rec(tree["left"][i]), rec(tree["right"][i]))
    return rec(0)
