"""Seeded synthetic inputs shared by the oracle, the tests and the benchmark.

This module holds data and random generators only: tuning-space descriptors,
the counter layouts, a seeded synthetic "GPU" that stands in for a real
profiler, and random tree ensembles for parity cases.  It contains none of the
search method's arithmetic (no decoding, constraint filtering, bottleneck
analysis, scoring or selection); both the CPU oracle and the CUDA library take
what it produces as plain input.

Interface constants defined here (counter roles, constraint opcodes) are the
shared data format of the library's descriptors; each side implements its own
interpretation of them.
"""
from __future__ import annotations

import json
import os
from dataclasses import dataclass, field
from typing import List

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))

# ---------------------------------------------------------------------------
# Counter roles: the 24 counters of the paper's counter table (Section 3.4,
# Table "tab:pcs"), in table order, plus the "global" thread-count
# pseudo-counter (Section 3.4.2) and an inert role for counters that the
# expert system does not read (stand-ins for stall-reason counters, which the
# paper leaves unused, Section 3.8).
# ---------------------------------------------------------------------------
ROLE_NAMES = [
    "DRAM_RT", "DRAM_WT", "L2_RT", "L2_WT", "TEX_RWT", "LOC_O", "SHR_LT",
    "SHR_WT", "INST_F32", "INST_F64", "INST_INT", "INST_MISC", "INST_LDST",
    "INST_CONT", "INST_BCONV", "INST_EXE", "INST_ISSUE_U", "DRAM_U", "L2_U",
    "TEX_U", "SHR_U", "SM_E", "WARP_E", "WARP_NP_E", "GLOBAL", "INERT",
]
ROLE = {n: i for i, n in enumerate(ROLE_NAMES)}
N_ROLES = len(ROLE_NAMES)

LAYOUT_16 = [ROLE[n] for n in (
    "DRAM_RT", "DRAM_WT", "L2_RT", "L2_WT", "TEX_RWT", "SHR_LT", "SHR_WT",
    "INST_F32", "INST_INT", "INST_LDST", "INST_EXE", "INST_ISSUE_U",
    "DRAM_U", "L2_U", "TEX_U", "SHR_U")]
LAYOUT_32 = list(range(25)) + [ROLE["INERT"]] * 7
LAYOUT_40 = list(range(25)) + [ROLE["INERT"]] * 15


def layout(k: int) -> List[int]:
    """Counter roles of the K=16 / 32 / 40 synthetic counter vectors."""
    return {16: LAYOUT_16, 32: LAYOUT_32, 40: LAYOUT_40}[k]


# ---------------------------------------------------------------------------
# Constraint bytecode: a stack program over int64 parameter values.  A program
# is a sequence of expressions; each REQUIRE pops one value and the
# configuration is valid only if every popped value is non-zero.
# DIV and MOD truncate toward zero (C semantics); a zero divisor yields 0.
# Arithmetic wraps modulo 2^64 (two's complement).
# ---------------------------------------------------------------------------
OP_VAL, OP_CONST = 1, 2            # VAL j: push value of parameter j; CONST c
OP_ADD, OP_SUB, OP_MUL, OP_DIV, OP_MOD = 3, 4, 5, 6, 7
OP_EQ, OP_NE, OP_LT, OP_LE, OP_GT, OP_GE = 8, 9, 10, 11, 12, 13
OP_AND, OP_OR, OP_NOT = 14, 15, 16
OP_REQUIRE = 17
OP_CONST64 = 18                    # CONST64 lo hi: push (hi << 32) | (lo & 0xffffffff)
OPS_WITH_ARG = (OP_VAL, OP_CONST)  # one argument word; CONST64 takes two
MAX_STACK = 16


@dataclass
class SpaceDesc:
    """A tuning space: per-parameter ascending value lists and constraints."""
    name: str
    param_names: List[str]
    values: List[List[int]]
    bytecode: List[int] = field(default_factory=list)

    @property
    def n_params(self) -> int:
        return len(self.values)

    @property
    def radices(self) -> List[int]:
        return [len(v) for v in self.values]

    @property
    def n_raw(self) -> int:
        n = 1
        for r in self.radices:
            n *= r
        return n

    def to_json(self) -> dict:
        return {"name": self.name, "param_names": self.param_names,
                "values": self.values, "bytecode": self.bytecode}

    @staticmethod
    def from_json(d: dict) -> "SpaceDesc":
        return SpaceDesc(d["name"], list(d["param_names"]),
                         [list(map(int, v)) for v in d["values"]],
                         list(map(int, d["bytecode"])))


def load_space(name: str) -> SpaceDesc:
    """Load a frozen descriptor from workloads/spaces/<name>.json."""
    with open(os.path.join(HERE, "spaces", name + ".json")) as f:
        return SpaceDesc.from_json(json.load(f))


# Constraint builders (bytecode emitters) -------------------------------------
def c_divides(a: int, b: int) -> List[int]:
    """v_a % v_b == 0."""
    return [OP_VAL, a, OP_VAL, b, OP_MOD, OP_CONST, 0, OP_EQ, OP_REQUIRE]


def c_product_le(params: List[int], bound: int) -> List[int]:
    """prod v_j <= bound."""
    code = [OP_VAL, params[0]]
    for j in params[1:]:
        code += [OP_VAL, j, OP_MUL]
    return code + const64(bound) + [OP_LE, OP_REQUIRE]


def const64(c: int) -> List[int]:
    """CONST64 instruction pushing the int64 constant c."""
    c &= (1 << 64) - 1
    lo, hi = c & 0xFFFFFFFF, c >> 32
    to_i32 = lambda x: x - (1 << 32) if x >= (1 << 31) else x
    return [OP_CONST64, to_i32(lo), to_i32(hi)]


def c_implies_le(a: int, x: int, b: int, y: int) -> List[int]:
    """v_a == x  ->  v_b <= y."""
    return [OP_VAL, a, OP_CONST, x, OP_NE, OP_VAL, b, OP_CONST, y, OP_LE,
            OP_OR, OP_REQUIRE]


def c_sum_le(params: List[int], bound: int) -> List[int]:
    """sum v_j <= bound."""
    code = [OP_VAL, params[0]]
    for j in params[1:]:
        code += [OP_VAL, j, OP_ADD]
    return code + [OP_CONST, bound, OP_LE, OP_REQUIRE]


def space_tiny_block_tile() -> SpaceDesc:
    """The 6-parameter space {block, tile_x, tile_y, unroll, use_smem, vec}
    with block * tile_x * tile_y <= 4096 (2,304 raw, 1,824 valid)."""
    vals = [[32, 64, 128, 256, 512, 1024], [1, 2, 4, 8], [1, 2, 4, 8],
            [1, 2, 4, 8], [0, 1], [1, 2, 4]]
    return SpaceDesc("tiny_block_tile", ["block", "tile_x", "tile_y", "unroll",
                                         "use_smem", "vec"], vals,
                     c_product_le([0, 1, 2], 4096))
