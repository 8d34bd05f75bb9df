"""Random regression-tree ensembles in a neutral pointer-based form.

A tree is a dict of equal-length arrays indexed by node id (root = 0):
``feature`` (int32, -1 at a leaf), ``threshold`` (int32; a configuration goes
right when its digit of ``feature`` is greater than it), ``left`` / ``right``
(int32 child ids, -1 at a leaf) and ``value`` (float32 leaf value, unused at
internal nodes).  A model is ``{"roles": [...], "depth": D, "trees": [...]}``
with one tree per counter.  These random ensembles are inputs for parity
cases; fitted ensembles come from the fitters.
"""
from __future__ import annotations

from typing import List

import numpy as np


def random_tree(rng: np.random.Generator, radices: List[int], depth: int,
                p_leaf: float = 0.08, p_zero: float = 0.05,
                p_dead: float = 0.03, scale: float = 8000.0) -> dict:
    feat, thr, left, right, val = [], [], [], [], []

    def new():
        feat.append(-1); thr.append(0); left.append(-1); right.append(-1); val.append(0.0)
        return len(feat) - 1

    def leaf_value():
        if rng.random() < p_zero:
            return 0.0
        # wide magnitude spread, non-negative like counters
        return float(np.float32(scale * rng.random() ** 3 + 1e-3 * rng.random()))

    def build(level: int) -> int:
        i = new()
        if level == depth or (level > 0 and rng.random() < p_leaf):
            val[i] = leaf_value()
            return i
        f = int(rng.integers(0, len(radices)))
        r = radices[f]
        if rng.random() < p_dead:
            t = int(rng.integers(max(0, r - 1), 16))      # right child unreachable
        else:
            t = int(rng.integers(0, max(1, r - 1)))
        feat[i], thr[i] = f, t
        li = build(level + 1)
        ri = build(level + 1)
        left[i], right[i] = li, ri
        return i

    build(0)
    return {"feature": np.asarray(feat, np.int32), "threshold": np.asarray(thr, np.int32),
            "left": np.asarray(left, np.int32), "right": np.asarray(right, np.int32),
            "value": np.asarray(val, np.float32)}


def random_model(radices: List[int], roles: List[int], depth: int, seed: int,
                 **kw) -> dict:
    rng = np.random.default_rng([int(seed), 0x7EE5])
    return {"roles": list(roles), "depth": int(depth),
            "trees": [random_tree(rng, radices, depth, **kw) for _ in roles]}
