"""Tuning space: decode, constraints, enumeration (oracle; test infrastructure).

Section 1 defines the tuning space as the cross product of the parameters'
value sets pruned by constraints; Algorithm 1 takes it as an array TS of all
configurations.  Reading used here: a configuration's raw index is its
mixed-radix number with the LAST parameter varying fastest, and TS lists the
valid configurations in ascending raw order.
"""
from __future__ import annotations

from typing import List

import numpy as np

import workloads as W


def strides(radices: List[int]) -> List[int]:
    """Mixed-radix place values, last parameter fastest."""
    out = [1] * len(radices)
    for j in range(len(radices) - 2, -1, -1):
        out[j] = out[j + 1] * radices[j + 1]
    return out


def decode(radices: List[int], raw) -> np.ndarray:
    """Digits d_j = (raw // stride_j) mod radix_j, shape [n, P] (int64)."""
    raw = np.atleast_1d(np.asarray(raw, dtype=np.int64))
    st = strides(radices)
    return np.stack([(raw // st[j]) % radices[j] for j in range(len(radices))], axis=1)


def encode(radices: List[int], digits) -> np.ndarray:
    """Inverse of decode: raw = sum_j d_j * stride_j."""
    d = np.atleast_2d(np.asarray(digits, dtype=np.int64))
    st = strides(radices)
    return sum(d[:, j] * st[j] for j in range(len(radices)))


def check_bytecode(desc: W.SpaceDesc) -> None:
    """Structural validation: known opcodes, arguments present, parameter
    indices in range, no stack underflow or overflow, empty stack at end."""
    code, depth, i = desc.bytecode, 0, 0
    while i < len(code):
        op = code[i]
        if op == W.OP_VAL:
            if i + 1 >= len(code) or not 0 <= code[i + 1] < desc.n_params:
                raise ValueError("bad VAL")
            depth += 1; i += 2
        elif op == W.OP_CONST:
            if i + 1 >= len(code):
                raise ValueError("bad CONST")
            depth += 1; i += 2
        elif op == W.OP_CONST64:
            if i + 2 >= len(code):
                raise ValueError("bad CONST64")
            depth += 1; i += 3
        elif W.OP_ADD <= op <= W.OP_OR:
            if depth < 2:
                raise ValueError("stack underflow")
            depth -= 1; i += 1
        elif op == W.OP_NOT:
            if depth < 1:
                raise ValueError("stack underflow")
            i += 1
        elif op == W.OP_REQUIRE:
            if depth < 1:
                raise ValueError("stack underflow")
            depth -= 1; i += 1
        else:
            raise ValueError("unknown opcode %d" % op)
        if depth > W.MAX_STACK:
            raise ValueError("stack overflow")
    if depth != 0:
        raise ValueError("values left on the stack")


def _tdiv(a, b):
    bz = b == 0
    bb = np.where(bz, 1, b)
    q = np.abs(a) // np.abs(bb)
    q = np.where((a < 0) != (bb < 0), -q, q)
    return np.where(bz, 0, q)


def _tmod(a, b):
    return np.where(b == 0, 0, a - _tdiv(a, b) * np.where(b == 0, 1, b))


def valid_mask(desc: W.SpaceDesc, digits: np.ndarray) -> np.ndarray:
    """Evaluate the constraint program for each digit row (stack machine over
    int64 parameter values, wrapping arithmetic, truncating division)."""
    d = np.atleast_2d(np.asarray(digits, dtype=np.int64))
    n = d.shape[0]
    vals = [np.asarray(v, dtype=np.int64) for v in desc.values]
    ok = np.ones(n, dtype=bool)
    stack: list = []
    code, i = desc.bytecode, 0
    with np.errstate(over="ignore"):
        while i < len(code):
            op = code[i]
            if op == W.OP_VAL:
                j = code[i + 1]
                stack.append(vals[j][d[:, j]]); i += 2; continue
            if op == W.OP_CONST:
                stack.append(np.full(n, code[i + 1], dtype=np.int64)); i += 2; continue
            if op == W.OP_CONST64:
                c = (code[i + 1] & 0xFFFFFFFF) | ((code[i + 2] & 0xFFFFFFFF) << 32)
                if c >= 1 << 63:
                    c -= 1 << 64
                stack.append(np.full(n, c, dtype=np.int64)); i += 3; continue
            if op == W.OP_NOT:
                stack.append((stack.pop() == 0).astype(np.int64)); i += 1; continue
            if op == W.OP_REQUIRE:
                ok &= stack.pop() != 0; i += 1; continue
            b = stack.pop(); a = stack.pop()
            if op == W.OP_ADD: r = a + b
            elif op == W.OP_SUB: r = a - b
            elif op == W.OP_MUL: r = a * b
            elif op == W.OP_DIV: r = _tdiv(a, b)
            elif op == W.OP_MOD: r = _tmod(a, b)
            elif op == W.OP_EQ: r = (a == b)
            elif op == W.OP_NE: r = (a != b)
            elif op == W.OP_LT: r = (a < b)
            elif op == W.OP_LE: r = (a <= b)
            elif op == W.OP_GT: r = (a > b)
            elif op == W.OP_GE: r = (a >= b)
            elif op == W.OP_AND: r = (a != 0) & (b != 0)
            elif op == W.OP_OR: r = (a != 0) | (b != 0)
            else:
                raise ValueError("unknown opcode %d" % op)
            stack.append(np.asarray(r, dtype=np.int64)); i += 1
    return ok


def is_valid_raw(desc: W.SpaceDesc, raw) -> np.ndarray:
    return valid_mask(desc, decode(desc.radices, raw))


def enumerate_valid(desc: W.SpaceDesc, chunk: int = 1 << 21) -> np.ndarray:
    """TS: all valid raw indices in ascending order (int64)."""
    check_bytecode(desc)
    out = []
    for lo in range(0, desc.n_raw, chunk):
        raw = np.arange(lo, min(desc.n_raw, lo + chunk), dtype=np.int64)
        out.append(raw[is_valid_raw(desc, raw)])
    return np.concatenate(out) if out else np.zeros(0, np.int64)


def count_valid(desc: W.SpaceDesc, chunk: int = 1 << 21) -> int:
    check_bytecode(desc)
    n = 0
    for lo in range(0, desc.n_raw, chunk):
        raw = np.arange(lo, min(desc.n_raw, lo + chunk), dtype=np.int64)
        n += int(is_valid_raw(desc, raw).sum())
    return n


def values_of(desc: W.SpaceDesc, raw: int) -> List[int]:
    """Parameter values of one configuration."""
    d = decode(desc.radices, [raw])[0]
    return [desc.values[j][d[j]] for j in range(desc.n_params)]
