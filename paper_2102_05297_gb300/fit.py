"""Model creation: one regression tree per counter (Section 3.3.2), or a
least-squares polynomial per counter and binary-parameter subspace (Section
3.3.1, ``fit_lsq``).

Host-side tooling, off the search step: it turns sampled profiles (digits of
the sampled configurations and their measured counters) into the tree
ensemble that ``ktune_model_load`` reads.  Trees are grown level by level:
for every open node and every parameter, digit histograms of the node's
samples give the sum of squared errors of each split "digit > t"; the split
with the largest error reduction is taken (ties to the lowest parameter, then
the lowest threshold).  A node becomes a leaf at the depth limit, with one
sample, with all targets equal, or when no split separates its samples; its
value is the float64 mean rounded to float32.
"""
from __future__ import annotations

from typing import List

import numpy as np


def fit_tree(digits: np.ndarray, y: np.ndarray, depth: int, radices: List[int]) -> dict:
    X = np.asarray(digits, dtype=np.int64)
    y = np.asarray(y, dtype=np.float64)
    n, P = X.shape
    feat, thr, left, right, val = [], [], [], [], []

    def new(v):
        feat.append(-1); thr.append(0); left.append(-1); right.append(-1); val.append(v)
        return len(feat) - 1

    node_id = np.zeros(n, dtype=np.int64)      # position of each sample among open nodes
    open_nodes = [new(float(np.float32(y.mean())) if n else 0.0)]
    for level in range(depth + 1):
        m = len(open_nodes)
        if m == 0:
            break
        cnt = np.bincount(node_id, minlength=m).astype(np.float64)
        s1 = np.bincount(node_id, weights=y, minlength=m)
        mean = s1 / np.maximum(cnt, 1)
        yc = y - mean[node_id]                   # centred targets: stable SSE sums
        sse = np.bincount(node_id, weights=yc * yc, minlength=m)
        ymin = np.full(m, np.inf); np.minimum.at(ymin, node_id, y)
        ymax = np.full(m, -np.inf); np.maximum.at(ymax, node_id, y)
        can = (cnt > 1) & (ymin < ymax) & (level < depth)
        best_gain = np.full(m, -np.inf)
        best_f = np.full(m, -1, dtype=np.int64)
        best_t = np.zeros(m, dtype=np.int64)
        for f in range(P):
            R = radices[f]
            if R < 2:
                continue
            key = node_id * R + X[:, f]
            hc = np.bincount(key, minlength=m * R).reshape(m, R)
            h1 = np.bincount(key, weights=yc, minlength=m * R).reshape(m, R)
            h2 = np.bincount(key, weights=yc * yc, minlength=m * R).reshape(m, R)
            cl, sl, ql = np.cumsum(hc, 1)[:, :-1], np.cumsum(h1, 1)[:, :-1], np.cumsum(h2, 1)[:, :-1]
            cr, sr, qr = cnt[:, None] - cl, -sl, sse[:, None] - ql   # centred: total sum is 0
            with np.errstate(divide="ignore", invalid="ignore"):
                e = (ql - sl * sl / cl) + (qr - sr * sr / cr)
            gain = sse[:, None] - e
            gain = np.where((cl > 0) & (cr > 0), gain, -np.inf)
            t = np.argmax(gain, axis=1)             # first maximum = lowest threshold
            g = gain[np.arange(m), t]
            better = g > best_gain                  # strict: ties keep the lower feature
            best_gain = np.where(better, g, best_gain)
            best_f = np.where(better, f, best_f)
            best_t = np.where(better, t, best_t)
        split = can & (best_f >= 0) & np.isfinite(best_gain)
        next_nodes = []
        child_of = np.full((m, 2), -1, dtype=np.int64)
        for j in range(m):
            if not split[j]:
                continue
            i = open_nodes[j]
            f, t = int(best_f[j]), int(best_t[j])
            sel = node_id == j
            go = X[sel, f] > t
            ys = y[sel]
            li = new(float(np.float32(ys[~go].mean())))
            ri = new(float(np.float32(ys[go].mean())))
            feat[i], thr[i], left[i], right[i] = f, t, li, ri
            child_of[j] = (len(next_nodes), len(next_nodes) + 1)
            next_nodes += [li, ri]
        if not next_nodes:
            break
        alive = split[node_id]
        f_s = best_f[node_id]
        go_right = np.zeros(n, dtype=bool)
        go_right[alive] = X[alive, f_s[alive]] > best_t[node_id[alive]]
        new_id = np.where(go_right, child_of[node_id, 1], child_of[node_id, 0])
        keep = alive
        X, y, node_id = X[keep], y[keep], new_id[keep]
        n = len(y)
        open_nodes = next_nodes
    return {"feature": np.asarray(feat, np.int32), "threshold": np.asarray(thr, np.int32),
            "left": np.asarray(left, np.int32), "right": np.asarray(right, np.int32),
            "value": np.asarray(val, np.float32)}


def fit_model(digits, Y, depth: int, radices: List[int], roles: List[int]) -> dict:
    """Per-counter trees for the counter layout ``roles``."""
    Y = np.asarray(Y)
    return {"roles": list(roles), "depth": int(depth),
            "trees": [fit_tree(digits, Y[:, k], depth, radices) for k in range(Y.shape[1])]}


def init_mlp(F: int, K: int, hidden: int = 256, seed: int = 0) -> dict:
    """Seeded starting parameters of the MLP counter model (host tooling, as
    the tree fitter is): every weight uniform in +-1/sqrt(fan_in) (the
    classic fan-in scaling), biases zero."""
    rng = np.random.default_rng(seed)

    def w(rows, cols):
        b = 1.0 / np.sqrt(cols)
        return rng.uniform(-b, b, size=(rows, cols)).astype(np.float32)

    return {"W1": w(hidden, F), "b1": np.zeros(hidden, np.float32),
            "W2": w(hidden, hidden), "b2": np.zeros(hidden, np.float32),
            "W3": w(hidden, hidden), "b3": np.zeros(hidden, np.float32),
            "W4": w(K, hidden), "b4": np.zeros(K, np.float32)}


def lsq_shape(values: List[List[int]]):
    """Binary parameters (subspace bits, first most significant), regressors
    (three or more values) and their u per digit: log2(1 + v) mapped linearly
    onto [-1, 1] over the parameter's values."""
    binary = [j for j, v in enumerate(values) if len(v) == 2]
    regs = [j for j, v in enumerate(values) if len(v) > 2]
    u = {}
    for j in regs:
        l = np.log2(np.asarray(values[j], dtype=np.float64) + 1.0)
        u[j] = (l - l.min()) * (2.0 / (l.max() - l.min())) - 1.0
    return binary, regs, u


def fit_lsq(values: List[List[int]], digits: np.ndarray, Y: np.ndarray, roles: List[int]) -> dict:
    """Least-squares model of counters Y [n][K] measured at the configurations
    with digits [n][P]: per subspace of the binary parameters, each counter
    regressed on 1, u_a, u_a^2 and u_a u_b (a < b) of the m regressors
    (T = 1 + 2m + m(m-1)/2 terms, in that order), minimum-norm solution; a
    subspace without samples takes the fit over all samples.  Coefficients
    are returned as float32 [2^nb][K][T]."""
    binary, regs, u = lsq_shape(values)
    D = np.asarray(digits, dtype=np.int64)
    Y = np.asarray(Y, dtype=np.float64).reshape(len(D), -1)
    U = np.column_stack([u[j][D[:, j]] for j in regs]) if regs else np.zeros((len(D), 0))
    m = U.shape[1]
    pairs = [(a, b) for a in range(m) for b in range(a + 1, m)]
    X = np.column_stack([np.ones(len(D))] + [U[:, a] for a in range(m)] + [U[:, a] * U[:, a] for a in range(m)]
                        + [U[:, a] * U[:, b] for a, b in pairs])
    sub = np.zeros(len(D), dtype=np.int64)
    for j in binary:
        sub = (sub << 1) | D[:, j]
    everything = np.linalg.lstsq(X, Y, rcond=None)[0].T
    coef = np.empty((1 << len(binary), Y.shape[1], X.shape[1]))
    for g in range(coef.shape[0]):
        r = np.flatnonzero(sub == g)
        coef[g] = np.linalg.lstsq(X[r], Y[r], rcond=None)[0].T if len(r) else everything
    return {"kind": "lsq", "roles": list(roles), "coef": coef.astype(np.float32)}
