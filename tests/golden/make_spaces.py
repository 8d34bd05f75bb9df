"""Freeze the synthetic tuning spaces as JSON and their oracle valid counts.

Run once; its outputs (workloads/spaces/*.json, tests/golden/space_counts.json)
are committed.

    python tests/golden/make_spaces.py [--only NAME]

For each space the structure (radices, value lists, constraint skeleton) is
drawn from a fixed seed, and the tightness knob of the product constraints is
bisected until the valid fraction, estimated on 400k random raw indices, puts
the valid count near its target.  The exact valid count of the final
descriptor is then computed by the CPU oracle's enumeration and written, with
the oracle named as its source, to tests/golden/space_counts.json.

Spaces (sizes follow the workloads they stand in for):
  mid_12p      12 parameters, 2-8 values, 5 constraints, ~2.1M valid
  large_16p    16 parameters, 2-16 values, 8 constraints, ~1e8 raw, ~2e7 valid
  batch_<i>    8 spaces, 6-14 parameters, 1e3 .. 5e6 valid (log-uniform)
"""
from __future__ import annotations

import argparse
import json
import math
import os
import sys

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
sys.path.insert(0, ROOT)

import workloads as W                      # noqa: E402
from workloads import spacegen             # noqa: E402
from oracle import space as ospace         # noqa: E402

GOLDEN = os.path.join(HERE, "space_counts.json")
SPACES = os.path.join(ROOT, "workloads", "spaces")


def est_valid(desc, seed=1, n=400_000):
    rng = np.random.default_rng(seed)
    if desc.n_raw <= n:
        return ospace.count_valid(desc)
    raw = rng.integers(0, desc.n_raw, size=n)
    return ospace.is_valid_raw(desc, raw).mean() * desc.n_raw


def tune(name, values, skel, target):
    lo, hi = 0.0, 1.0
    best = None
    for _ in range(30):
        mid = 0.5 * (lo + hi)
        d = spacegen.instantiate(name, values, skel, mid)
        v = est_valid(d)
        if best is None or abs(math.log(v + 1) - math.log(target)) < abs(math.log(best[1] + 1) - math.log(target)):
            best = (mid, v)
        if v < target:
            lo = mid
        else:
            hi = mid
    return spacegen.instantiate(name, values, skel, best[0])


SPECS = {
    "mid_12p": dict(seed=12, n_params=12, radix_lo=2, radix_hi=8, n_div=1, n_prod=3,
                    n_impl=1, raw_lo=4e7, raw_hi=6e7, target=2.1e6),
    "large_16p": dict(seed=16, n_params=16, radix_lo=2, radix_hi=16, n_div=1, n_prod=6,
                      n_impl=1, raw_lo=0.9e8, raw_hi=1.2e8, target=2.0e7),
}


def batch_specs():
    rng = np.random.default_rng(2024)
    out = {}
    for i in range(8):
        target = float(math.exp(rng.uniform(math.log(1e3), math.log(5e6))))
        P = int(rng.integers(6, 15))
        raw = max(target * float(rng.uniform(2.0, 8.0)), 1.6 * 2.0 ** P)
        out["batch_%d" % i] = dict(seed=100 + i, n_params=P, radix_lo=2, radix_hi=16,
                                   n_div=1, n_prod=2, n_impl=1, raw_lo=raw * 0.7,
                                   raw_hi=raw * 1.3, target=target)
    return out


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--only", default=None)
    a = ap.parse_args()
    specs = dict(SPECS)
    specs.update(batch_specs())
    counts = {}
    if os.path.exists(GOLDEN):
        with open(GOLDEN) as f:
            counts = json.load(f)
    for name, sp in specs.items():
        if a.only and name != a.only:
            continue
        sp = dict(sp)
        target = sp.pop("target")
        seed = sp.pop("seed")
        values, skel = spacegen.structure(seed, **sp)
        desc = tune(name, values, skel, target)
        ospace.check_bytecode(desc)
        n_valid = ospace.count_valid(desc)
        with open(os.path.join(SPACES, name + ".json"), "w") as f:
            json.dump(desc.to_json(), f, indent=1)
        counts[name] = {"n_raw": desc.n_raw, "n_valid": n_valid,
                        "source": "oracle.space.count_valid"}
        print(name, "P=%d raw=%d valid=%d (target %.3g)" % (desc.n_params, desc.n_raw, n_valid, target))
    t = W.space_tiny_block_tile()
    counts["tiny_block_tile"] = {"n_raw": t.n_raw, "n_valid": ospace.count_valid(t),
                                 "source": "oracle.space.count_valid"}
    with open(GOLDEN, "w") as f:
        json.dump(counts, f, indent=1, sort_keys=True)


if __name__ == "__main__":
    main()
