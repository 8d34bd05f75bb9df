"""Pins of the oracle's space enumeration: brute force over the cross product
with constraints written as plain Python predicates (not bytecode)."""
import itertools
import json
import os

import numpy as np
import pytest

import workloads as W
from oracle import space

GOLD = os.path.join(os.path.dirname(__file__), "golden")


def brute(values, pred):
    """Valid raw indices by nested iteration, last parameter fastest."""
    out = []
    for raw, combo in enumerate(itertools.product(*values)):
        if pred(combo):
            out.append(raw)
    return np.asarray(out, dtype=np.int64)


def test_tiny_block_tile_closed_form():
    d = W.space_tiny_block_tile()
    # block * tile_x * tile_y <= 4096, counted directly
    n = 0
    for b in [32, 64, 128, 256, 512, 1024]:
        for tx in [1, 2, 4, 8]:
            for ty in [1, 2, 4, 8]:
                if b * tx * ty <= 4096:
                    n += 1
    n *= 4 * 2 * 3
    assert n == 1824
    assert space.count_valid(d) == n
    np.testing.assert_array_equal(
        space.enumerate_valid(d), brute(d.values, lambda c: c[0] * c[1] * c[2] <= 4096))


def test_last_parameter_fastest():
    radices = [3, 4, 5]
    assert space.strides(radices) == [20, 5, 1]
    np.testing.assert_array_equal(space.decode(radices, [0, 1, 5, 20, 59]),
                                  [[0, 0, 0], [0, 0, 1], [0, 1, 0], [1, 0, 0], [2, 3, 4]])
    raw = np.arange(60)
    np.testing.assert_array_equal(space.encode(radices, space.decode(radices, raw)), raw)


@pytest.mark.parametrize("seed", range(6))
def test_random_constraints_vs_python(seed):
    rng = np.random.default_rng(seed)
    P = int(rng.integers(2, 5))
    values = []
    for _ in range(P):
        r = int(rng.integers(2, 6))
        values.append(sorted(int(x) for x in rng.choice(np.arange(-6, 40), size=r, replace=False)))
    a, b = (int(x) for x in rng.choice(P, size=2, replace=False))
    c = int(rng.integers(-50, 200))
    x = values[a][0]
    # v_a % v_b == 0  (C truncation; zero divisor -> 0)
    code = W.c_divides(a, b)
    def cmod(u, v):
        if v == 0:
            return 0
        q = abs(u) // abs(v)
        q = -q if (u < 0) != (v < 0) else q
        return u - q * v
    # v_a * v_b <= c, v_a == x -> v_b <= 10, and (v_a - v_b) / 3 > -2 via DIV
    code += W.c_product_le([a, b], c) + W.c_implies_le(a, x, b, 10)
    code += [W.OP_VAL, a, W.OP_VAL, b, W.OP_SUB, W.OP_CONST, 3, W.OP_DIV, W.OP_CONST, -2,
             W.OP_GT, W.OP_REQUIRE]
    def tdiv(u, v):
        if v == 0:
            return 0
        q = abs(u) // abs(v)
        return -q if (u < 0) != (v < 0) else q
    def pred(cv):
        return (cmod(cv[a], cv[b]) == 0 and cv[a] * cv[b] <= c
                and (cv[a] != x or cv[b] <= 10) and tdiv(cv[a] - cv[b], 3) > -2)
    d = W.SpaceDesc("t", ["p%d" % j for j in range(P)], values, code)
    np.testing.assert_array_equal(space.enumerate_valid(d, chunk=7), brute(values, pred))


def test_logic_ops_and_const64():
    values = [[0, 1, 2], [0, 3], [5, 7]]
    code = [W.OP_VAL, 0, W.OP_VAL, 1, W.OP_AND, W.OP_VAL, 2, W.OP_CONST, 7, W.OP_EQ,
            W.OP_OR, W.OP_REQUIRE]
    code += [W.OP_VAL, 0, W.OP_NOT, W.OP_NOT, W.OP_VAL, 1, W.OP_GE, W.OP_REQUIRE]
    code += W.const64(1 << 40) + [W.OP_VAL, 2, W.OP_MUL] + W.const64(6 << 40) + [W.OP_LT, W.OP_REQUIRE]
    d = W.SpaceDesc("t", ["a", "b", "c"], values, code)
    def pred(cv):
        return (((cv[0] != 0 and cv[1] != 0) or cv[2] == 7) and int(cv[0] != 0) >= cv[1]
                and (cv[2] << 40) < (6 << 40))
    np.testing.assert_array_equal(space.enumerate_valid(d), brute(values, pred))


@pytest.mark.parametrize("code", [[W.OP_ADD, W.OP_REQUIRE], [W.OP_VAL, 5, W.OP_REQUIRE],
                                  [W.OP_VAL, 0], [99], [W.OP_CONST]])
def test_bad_bytecode_rejected(code):
    d = W.SpaceDesc("t", ["a", "b"], [[1, 2], [3, 4]], code)
    with pytest.raises(ValueError):
        space.check_bytecode(d)


def test_frozen_counts_consistent():
    """The committed descriptors parse and their stored counts are plausible
    (exact counts are recomputed by the oracle in the slow test below)."""
    with open(os.path.join(GOLD, "space_counts.json")) as f:
        counts = json.load(f)
    for name, c in counts.items():
        if name == "tiny_block_tile":
            continue
        d = W.load_space(name)
        space.check_bytecode(d)
        assert d.n_raw == c["n_raw"]
        rng = np.random.default_rng(0)
        raw = rng.integers(0, d.n_raw, size=20000)
        frac = space.is_valid_raw(d, raw).mean()
        assert abs(frac * d.n_raw - c["n_valid"]) < 0.08 * d.n_raw + 50
