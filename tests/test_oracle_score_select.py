"""Pins of Eq. score, Eq. score_normalization, the integer weights, Philox
and the weighted draws."""
import os

import numpy as np
import pytest

from oracle import score, select

GOLD = os.path.join(os.path.dirname(__file__), "golden")


# ---- Eq. score ---------------------------------------------------------------
def test_score_hand_case():
    delta = [-0.5, 0.25, 0.0]
    A = [100.0, 10.0, 5.0]
    a = [[50.0, 30.0, 1.0]]
    # -0.5 * (50-100)/150 + 0.25 * (30-10)/40 ; counter 2 has no Delta
    s = score.score_def(A, a, delta)[0]
    assert s == pytest.approx(1.0 / 6.0 + 0.125, abs=1e-15)


def test_score_direction():
    """A candidate that lowers a counter the expert system wants lowered, or
    raises one it wants raised, scores positive."""
    assert score.score_def([100.0], [[50.0]], [-1.0])[0] > 0
    assert score.score_def([100.0], [[150.0]], [-1.0])[0] < 0
    assert score.score_def([100.0], [[150.0]], [+1.0])[0] > 0


def test_score_pc_used_excludes_zero_predictions():
    assert score.score_def([0.0, 10.0], [[5.0, 10.0]], [-1.0, -1.0])[0] == 0.0
    assert score.score_def([5.0], [[0.0]], [-1.0])[0] == 0.0
    assert score.score_fp32([0.0], [[5.0]], [-1.0])[0] == 0.0


@pytest.mark.parametrize("seed", range(4))
def test_score_antisymmetry_bound_and_fp32(seed):
    rng = np.random.default_rng(seed)
    K = 32
    A = (rng.random(K) * 8000).astype(np.float32)
    C = (rng.random((500, K)) * 8000).astype(np.float32)
    C[rng.random((500, K)) < 0.05] = 0
    d = np.where(rng.random(K) < 0.4, 0.0, rng.uniform(-1, 1, K))
    s = score.score_def(A, C, d)
    # antisymmetry: swapping profiled and candidate negates each term exactly
    for i in range(20):
        back = score.score_def(C[i], A[None, :], d)[0]
        assert back == -s[i]
    assert np.all(np.abs(s) <= np.abs(d).sum() + 1e-12)
    assert np.all(score.score_def(A, A[None, :], d) == 0)
    s32 = score.score_fp32(A, C, d.astype(np.float32))
    # three roundings per term plus K additions: < (K + 3) 2^-24 sum|delta|
    bound = (K + 3) * 2.0 ** -24 * np.abs(d).sum()
    assert np.all(np.abs(s32.astype(np.float64) - s) <= bound)


# ---- Eq. score_normalization and the weights ------------------------------
def test_normalisation_end_points():
    s = np.float32([0.5, 0.0, -0.25, -0.3, -0.1, 0.25])
    out = select.normalise_fp32(s, s_min=-0.3, s_max=0.5)
    assert out[0] == 256.0                      # s = s_max
    assert out[1] == 1.0                        # s = 0
    assert out[2] == np.float32(1e-4)           # s = gamma
    assert out[3] == np.float32(1e-4)           # s < gamma
    assert out[4] == pytest.approx((1 - (-0.1) / -0.3) ** 8, rel=1e-6)
    assert out[5] == pytest.approx(1.5 ** 8, rel=1e-6)
    # s_min above gamma: the lowest score reaches the 1e-4 floor
    out = select.normalise_fp32(np.float32([-0.2, -0.1]), -0.2, 0.3)
    assert out[0] == np.float32(1e-4)
    assert out[1] == pytest.approx(0.5 ** 8, rel=1e-6)
    # all scores zero: s_min = s_max = 0
    assert np.all(select.normalise_fp32(np.float32([0, 0]), 0.0, 0.0) == 1.0)


def test_normalisation_fp32_vs_def():
    rng = np.random.default_rng(0)
    s = rng.uniform(-0.6, 0.9, 2000).astype(np.float32)
    a = select.normalise_fp32(s, s.min(), s.max())
    b = select.normalise_def(s.astype(np.float64), float(s.min()), float(s.max()))
    np.testing.assert_allclose(a, b, rtol=3e-6)


def test_quantise():
    w = select.quantise(np.float32([1e-4, 1.0, 256.0, 0.5]))
    assert list(w) == [105, 1 << 20, 1 << 28, 1 << 19]


# ---- Philox4x32-10 -----------------------------------------------------------
def test_philox_known_answers():
    rows = [l.split() for l in open(os.path.join(GOLD, "philox4x32_10_kat.txt"))
            if l.strip() and not l.startswith("#")]
    assert len(rows) == 3
    for r in rows:
        v = [int(x, 16) for x in r]
        assert select.philox4x32_10(tuple(v[:4]), tuple(v[4:6])) == v[6:10]


def test_scaled_draw_range():
    assert select.scaled_draw(0, 10) == 0
    assert select.scaled_draw((1 << 64) - 1, 10) == 9
    assert select.scaled_draw(1 << 63, 10) == 5


# ---- weighted draws --------------------------------------------------------
def test_draws_without_replacement():
    w = np.array([0, 5, 0, 7, 1, 0, 3], dtype=np.uint64)
    got = select.weighted_draws(w, 10, seed=9, search_id=0, step=0)
    assert sorted(got) == [1, 3, 4, 6]
    assert len(set(got)) == len(got)


def test_draw_is_first_prefix_above_r():
    w = np.array([3, 0, 2, 5], dtype=np.uint64)
    u = select.uniform_u64(5, 1, 2, 0, 0)
    r = select.scaled_draw(u, 10)
    expect = [0, 0, 0, 2, 2, 3, 3, 3, 3, 3][r]
    assert select.weighted_draws(w, 1, 5, 1, 2) == [expect]


def test_draw_frequencies_chi_square():
    scipy = pytest.importorskip("scipy.stats")
    w = np.array([105, 1 << 20, 3 << 20, 1 << 18, 7 << 19, 1 << 20], dtype=np.uint64)
    n = 30000
    hits = np.zeros(len(w))
    total = int(w.sum())
    csum = np.cumsum(w.astype(object))
    for step in range(n):
        r = select.scaled_draw(select.uniform_u64(1, 0, step, 0, 0), total)
        hits[next(i for i, c in enumerate(csum) if c > r)] += 1
    exp = n * w.astype(np.float64) / total
    chi2 = ((hits - exp) ** 2 / exp).sum()
    assert chi2 < scipy.chi2.ppf(0.999, len(w) - 1)


def test_topk_ties_to_lower_raw():
    s = np.float32([0.5, 0.9, 0.5, 0.9, 0.1])
    raw = np.array([40, 30, 10, 20, 0])
    assert select.topk(s, raw, 3) == [3, 1, 2]
