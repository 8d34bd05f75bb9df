"""The library-side tree fitter against the oracle's fitter and exact cases."""
import itertools

import numpy as np

from oracle import trees as otrees
from paper_2102_05297_gb300 import fit


def test_fit_matches_oracle_on_random_data():
    rng = np.random.default_rng(0)
    radices = [3, 5, 2, 4]
    X = np.stack([rng.integers(0, r, size=400) for r in radices], axis=1)
    for k in range(4):
        y = rng.normal(size=400) * 100 + X[:, k % 4] * 30.0
        a = fit.fit_tree(X, y, 6, radices)
        b = otrees.fit_tree(X, y, 6, radices)
        Xa = np.array(list(itertools.product(*[range(r) for r in radices])))
        np.testing.assert_array_equal(otrees.predict_tree(a, Xa), otrees.predict_tree(b, Xa))


def test_fit_recovers_piecewise_constant():
    radices = [4, 3, 5, 2]
    X = np.array(list(itertools.product(*[range(r) for r in radices])))
    y = np.where(X[:, 2] > 2, 7.0, 1.0) * np.where(X[:, 0] > 0, 3.0, 1.0)
    t = fit.fit_tree(X, y, 4, radices)
    np.testing.assert_array_equal(otrees.predict_tree(t, X), y.astype(np.float32))
    assert otrees.tree_depth(t) == 2


def test_fit_depth_limit():
    rng = np.random.default_rng(2)
    X = rng.integers(0, 8, size=(3000, 6))
    t = fit.fit_tree(X, rng.normal(size=3000), 5, [8] * 6)
    assert otrees.tree_depth(t) == 5
