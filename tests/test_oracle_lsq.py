"""Pins of the least-squares counter model oracle (Section 3.3.1): the term
count; exact recovery of a target that is itself a member of the model class;
the normal equations of the least-squares fit on noisy data; the subspace
split by binary parameters; and the fallback for a subspace without samples."""
import itertools

import numpy as np

from oracle import lsq

VALUES = [[0, 1], [1, 2, 4, 8], [3, 6, 9], [0, 1], [8, 16, 32, 64, 128], [5]]


def all_digits(values):
    return np.array(list(itertools.product(*[range(len(v)) for v in values])), dtype=np.int64)


def test_design_and_term_count():
    d = lsq.design(VALUES)
    assert d["binary"] == [0, 3] and d["regs"] == [1, 2, 4] and d["n_sub"] == 4
    m = 3
    assert d["T"] == 1 + 2 * m + m * (m - 1) // 2 == 10
    # u spans [-1, 1] on log2(1 + v)
    np.testing.assert_allclose(d["u"][1][[0, -1]], [-1.0, 1.0])
    lv = np.log2(1.0 + np.array([3, 6, 9.0]))
    np.testing.assert_allclose(d["u"][2], 2 * (lv - lv[0]) / (lv[-1] - lv[0]) - 1)


def test_terms_by_hand():
    d = lsq.design(VALUES)
    dig = np.array([[1, 2, 0, 0, 4, 0]])
    u1, u2, u4 = d["u"][1][2], d["u"][2][0], d["u"][4][4]
    expect = [1, u1, u2, u4, u1 * u1, u2 * u2, u4 * u4, u1 * u2, u1 * u4, u2 * u4]
    np.testing.assert_allclose(lsq.terms(d, dig)[0], expect)
    assert lsq.subspace(d, dig)[0] == 2          # digits (1, 0) of the binary parameters 0, 3


def test_exact_recovery_of_a_model_member():
    rng = np.random.default_rng(0)
    d = lsq.design(VALUES)
    C = rng.standard_normal((d["n_sub"], 3, d["T"]))
    dig = all_digits(VALUES)
    Y = lsq.predict(VALUES, C, dig)
    C2 = lsq.fit(VALUES, dig, Y)
    np.testing.assert_allclose(C2, C, atol=1e-9)
    np.testing.assert_allclose(lsq.predict(VALUES, C2, dig), Y, atol=1e-9)


def test_normal_equations_on_noisy_targets():
    rng = np.random.default_rng(1)
    d = lsq.design(VALUES)
    dig = all_digits(VALUES)
    Y = rng.standard_normal((len(dig), 2)) * 10 + np.sin(dig[:, [1]] * dig[:, [4]])
    C = lsq.fit(VALUES, dig, Y)
    X = lsq.terms(d, dig)
    sub = lsq.subspace(d, dig)
    for g in range(d["n_sub"]):
        r = sub == g
        resid = Y[r] - X[r] @ C[g].T
        np.testing.assert_allclose(X[r].T @ resid, 0.0, atol=1e-8)   # X^T (y - X c) = 0


def test_subspaces_are_separate_models():
    d = lsq.design(VALUES)
    dig = all_digits(VALUES)
    Y = (7.0 * dig[:, 0] + 3.0 * dig[:, 3] + 1.0)[:, None]           # depends on binaries only
    C = lsq.fit(VALUES, dig, Y)
    for g, (b0, b3) in enumerate([(0, 0), (0, 1), (1, 0), (1, 1)]):
        np.testing.assert_allclose(C[g, 0, 0], 7.0 * b0 + 3.0 * b3 + 1.0, atol=1e-9)
        np.testing.assert_allclose(C[g, 0, 1:], 0.0, atol=1e-9)


def test_empty_subspace_takes_the_global_fit():
    d = lsq.design(VALUES)
    dig = all_digits(VALUES)
    keep = lsq.subspace(d, dig) != 3
    Y = (dig[:, 1] * 2.0 + 1.0)[:, None]
    C = lsq.fit(VALUES, dig[keep], Y[keep])
    glob = np.linalg.lstsq(lsq.terms(d, dig[keep]), Y[keep], rcond=None)[0].T
    np.testing.assert_allclose(C[3], glob)
