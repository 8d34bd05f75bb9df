"""Seeded generators of tuning-space structure.

A generated space has parameters of three kinds (powers of two, small linear
ranges, binary flags) and constraints of the kinds tuning spaces use:
divisibility, bounded products and conditional bounds.  The product bounds
are set by one tightness knob ``tau`` in [0, 1]; the committed script
``make_spaces.py`` picks ``tau`` so that the valid count lands near a target
and freezes the result as JSON.
"""
from __future__ import annotations

import math
from typing import List, Tuple

import numpy as np

from . import SpaceDesc, c_divides, c_implies_le, c_product_le


def _values(rng, kind: str, radix: int) -> List[int]:
    if kind == "bin":
        return [0, 1][:radix] if radix <= 2 else list(range(radix))
    if kind == "pow2":
        start = int(rng.integers(0, 4))
        return [1 << (start + i) for i in range(radix)]
    step = int(rng.integers(1, 4))
    start = int(rng.integers(1, 4))
    return [start + step * i for i in range(radix)]


def structure(seed: int, n_params: int, radix_lo: int, radix_hi: int,
              n_div: int, n_prod: int, n_impl: int, raw_lo: float, raw_hi: float):
    """Draw radices (until the raw size is in [raw_lo, raw_hi]), value lists
    and constraint skeletons.  Returns (values, skeleton)."""
    rng = np.random.default_rng([int(seed), 0x59ACE])
    log_target = 0.5 * (math.log(raw_lo) + math.log(raw_hi))
    for _ in range(100000):
        # split log(raw size) among the parameters (Dirichlet shares)
        share = rng.dirichlet(np.ones(n_params))
        radices = [int(min(radix_hi, max(radix_lo, round(math.exp(s * log_target)))))
                   for s in share]
        n_raw = math.prod(radices)
        if raw_lo <= n_raw <= raw_hi:
            break
    else:
        raise RuntimeError("no radix draw in range")
    kinds = []
    for r in radices:
        if r == 2 and rng.random() < 0.5:
            kinds.append("bin")
        elif rng.random() < 0.7:
            kinds.append("pow2")
        else:
            kinds.append("lin")
    values = [_values(rng, k, r) for k, r in zip(kinds, radices)]
    pow2 = [j for j, k in enumerate(kinds) if k == "pow2"]
    nonbin = [j for j, k in enumerate(kinds) if k != "bin"]
    skel = []
    for _ in range(n_div):
        if len(pow2) >= 2:
            a, b = rng.choice(pow2, size=2, replace=False)
            skel.append(("div", int(a), int(b)))
    for _ in range(n_prod):
        m = int(rng.integers(2, 4))
        ps = sorted(int(x) for x in rng.choice(nonbin, size=min(m, len(nonbin)), replace=False))
        skel.append(("prod", ps, float(rng.uniform(0.0, 1.0))))
    for _ in range(n_impl):
        a, b = rng.choice(n_params, size=2, replace=False)
        a, b = int(a), int(b)
        x = values[a][int(rng.integers(0, len(values[a])))]
        y = values[b][int(rng.integers(0, len(values[b])))]
        skel.append(("impl", a, x, b, y))
    return values, skel


def instantiate(name: str, values, skel, tau: float) -> SpaceDesc:
    """Build the descriptor for tightness ``tau`` (larger = more valid)."""
    code = []
    for item in skel:
        if item[0] == "div":
            code += c_divides(item[1], item[2])
        elif item[0] == "prod":
            ps, jitter = item[1], item[2]
            lo = math.log(math.prod(min(values[j]) for j in ps))
            hi = math.log(math.prod(max(values[j]) for j in ps))
            t = min(1.0, max(0.0, tau + 0.15 * (jitter - 0.5)))
            code += c_product_le(ps, int(round(math.exp(lo + t * (hi - lo)))))
        else:
            _, a, x, b, y = item
            code += c_implies_le(a, x, b, y)
    names = ["p%d" % j for j in range(len(values))]
    return SpaceDesc(name, names, [list(v) for v in values], code)
