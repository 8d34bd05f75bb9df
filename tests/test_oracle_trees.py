"""Pins of the oracle's regression trees: hand-traced walks, exact recovery of
piecewise-constant targets, brute-force best split."""
import itertools

import numpy as np

from oracle import trees


def _tree(nodes):
    """nodes: list of (feature, threshold, left, right, value)."""
    f, t, l, r, v = zip(*nodes)
    return {"feature": np.array(f, np.int32), "threshold": np.array(t, np.int32),
            "left": np.array(l, np.int32), "right": np.array(r, np.int32),
            "value": np.array(v, np.float32)}


def test_hand_traced_depth3():
    # root: d1 > 1 ?  left: d0 > 0 ? (leaf 10 | leaf 20)   right: d2 > 2 ? (leaf 30 | d0 > 2 ? (40 | 50))
    t = _tree([(1, 1, 1, 2, 0), (0, 0, 3, 4, 0), (2, 2, 5, 6, 0), (-1, 0, -1, -1, 10.0),
               (-1, 0, -1, -1, 20.0), (-1, 0, -1, -1, 30.0), (0, 2, 7, 8, 0),
               (-1, 0, -1, -1, 40.0), (-1, 0, -1, -1, 50.0)])
    digits = np.array([[0, 0, 0], [1, 1, 9], [0, 2, 2], [5, 3, 3], [2, 3, 3], [3, 2, 5]])
    expect = [10, 20, 30, 50, 40, 50]
    np.testing.assert_array_equal(trees.predict_tree(t, digits), np.float32(expect))
    assert trees.tree_depth(t) == 3


def test_single_leaf_tree():
    t = _tree([(-1, 0, -1, -1, 7.5)])
    np.testing.assert_array_equal(trees.predict_tree(t, np.zeros((4, 2))), np.float32([7.5] * 4))


def test_fit_recovers_piecewise_constant():
    radices = [4, 3, 5]
    digits = np.array(list(itertools.product(*[range(r) for r in radices])))
    y = np.where(digits[:, 0] > 1, 100.0, 10.0) + np.where(digits[:, 2] > 3, 1.0, 0.0)
    t = trees.fit_tree(digits, y, depth=3, radices=radices)
    np.testing.assert_array_equal(trees.predict_tree(t, digits), y.astype(np.float32))
    # pure nodes stop early: two splits suffice
    assert trees.tree_depth(t) == 2


def test_fit_root_split_is_brute_force_best():
    rng = np.random.default_rng(3)
    radices = [3, 4, 2]
    digits = np.stack([rng.integers(0, r, size=40) for r in radices], axis=1)
    y = rng.normal(size=40) * 5 + digits[:, 1] * 2.0
    t = trees.fit_tree(digits, y, depth=1, radices=radices)
    best = None
    n = len(y)
    for f, r in enumerate(radices):
        for thr in range(r - 1):
            m = digits[:, f] > thr
            if m.all() or (~m).all():
                continue
            # within-group variance form of the error, computed independently
            err = np.var(y[m]) * m.sum() + np.var(y[~m]) * (~m).sum()
            if best is None or err < best[0] - 1e-9:
                best = (err, f, thr)
    assert (int(t["feature"][0]), int(t["threshold"][0])) == (best[1], best[2])
    m = digits[:, best[1]] > best[2]
    assert t["value"][t["left"][0]] == np.float32(y[~m].mean())
    assert t["value"][t["right"][0]] == np.float32(y[m].mean())


def test_fit_ties_lowest_feature_then_threshold():
    # two identical features: the split must use feature 0
    digits = np.array([[0, 0], [1, 1], [2, 2], [0, 0], [2, 2]])
    y = np.array([1.0, 5.0, 5.0, 1.0, 5.0])
    t = trees.fit_tree(digits, y, depth=1, radices=[3, 3])
    assert (t["feature"][0], t["threshold"][0]) == (0, 0)


def test_fit_depth_limit_and_leaf_rounding():
    rng = np.random.default_rng(1)
    digits = rng.integers(0, 4, size=(200, 3))
    y = rng.normal(size=200) * 1000 + 0.1
    t = trees.fit_tree(digits, y, depth=4, radices=[4, 4, 4])
    assert trees.tree_depth(t) <= 4
    assert t["value"].dtype == np.float32
