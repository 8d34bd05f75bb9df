"""The search on real profiles: Algorithm 1 driven by a profiler instead of a
synthetic performance function.

Each step profiles the current c_profile of a real tunable kernel with
``ncu`` (the Volta-and-newer metrics of the counter table, Table "tab:pcs";
one launch, the GPU's clocks left as they are), converts the counters
(``ncu_counters``), runs ``ktune_step`` on them, times the k configurations it
returns with CUDA events and reports their runtimes (``ktune_report``): the
fastest becomes the next c_profile (Section 3.2's workflow, Algorithm 1).

The kernel (``live/coulomb.cu``) is a direct Coulomb summation on one slice of
a regular grid, with five tuning parameters: block shape BX x BY, grid points
per thread OUT, unrolling of the loop over the charges UNROLL, and staging of
the charges in shared memory SMEM.  The model is a tree ensemble (Section
3.3.2) fitted on ncu profiles of a uniform sample of the space, the paper's
setting of a model built before the search.  For reference every
configuration is timed once, so that the tests a search needs to reach
within 1.1x of the best configuration can be counted and compared with
uniform random draws.

    python -m paper_2102_05297_gb300.live [--seeds 0,1,2] [--out record.json]

Host tooling around the library (the step itself runs in libktune).
"""
from __future__ import annotations

import argparse
import json
import os
import subprocess
import tempfile
import time
from typing import List, Optional, Sequence

import numpy as np

from . import build as _build
from . import ktune as kt
from . import ncu_counters as nc

NAMES = ["BX", "BY", "OUT", "UNROLL", "SMEM"]
VALUES = [[32, 64, 128], [1, 2, 4, 8], [1, 2, 4], [1, 2, 4, 8], [0, 1]]
# constraint bytecode (include/ktune.h opcodes): BX * BY >= 64; OUT * UNROLL <= 16
_VAL, _CONST, _MUL, _LE, _GE, _REQ = 1, 2, 5, 11, 13, 17
BYTECODE = [_VAL, 0, _VAL, 1, _MUL, _CONST, 64, _GE, _REQ,
            _VAL, 2, _VAL, 3, _MUL, _CONST, 16, _LE, _REQ]
ROLES = list(range(25))          # the table's 24 counters and the thread count (GLOBAL)
KERNEL = "coulomb"


def binary() -> str:
    if not os.path.exists(_build.LIVE_BIN):
        raise RuntimeError("the tunable kernel is not built; run `python -m paper_2102_05297_gb300.build`")
    return _build.LIVE_BIN


def cfg_args(rows) -> List[str]:
    return [",".join(str(int(v)) for v in r) for r in rows]


def time_configs(rows, reps: int = 5):
    """Median device time (ms, CUDA events) of `reps` launches of each
    configuration, and each configuration's checksum of the computed grid."""
    r = subprocess.run([binary(), "time", str(reps)] + cfg_args(rows), capture_output=True, text=True)
    if r.returncode:
        raise RuntimeError("timing run failed: " + r.stderr)
    d = json.loads(r.stdout)
    return np.asarray(d["ms"], np.float64), np.asarray(d["checksum"], np.float64)


def profile(rows, roles: Sequence[int] = ROLES, workdir: Optional[str] = None) -> np.ndarray:
    """ncu counters of one launch of each configuration, in the layout of
    `roles`: the program first runs as it is (it must exit 0), then under
    ncu with the layout's metrics."""
    prog = [binary(), "run"] + cfg_args(rows)
    r = subprocess.run(prog, capture_output=True, text=True)
    if r.returncode:
        raise RuntimeError("plain run failed: " + r.stderr)
    fd, path = tempfile.mkstemp(suffix=".csv", dir=workdir)
    os.close(fd)
    try:
        cmd = nc.ncu_command(prog, KERNEL, roles, path, launch_skip=0, launch_count=len(rows))
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode:
            raise RuntimeError("ncu failed: " + r.stdout[-2000:] + r.stderr[-2000:])
        with open(path) as f:
            launches = nc.parse_csv(f.read(), KERNEL)
    finally:
        os.unlink(path)
    if len(launches) != len(rows):
        raise RuntimeError("ncu profiled %d launches, expected %d" % (len(launches), len(rows)))
    return np.stack([nc.counters(v, roles) for v in launches])


def space():
    return kt.Space(VALUES, BYTECODE)


def rows_of(digits) -> np.ndarray:
    return np.array([[VALUES[j][int(d)] for j, d in enumerate(row)] for row in digits], np.int64)


def run(seeds: Sequence[int] = (0, 1, 2), k: int = 5, sample_frac: float = 0.2, depth: int = 8,
        max_tests: int = 120, cores: float = 19456.0, workdir: Optional[str] = None,
        log=print) -> dict:
    from .fit import fit_model
    sp = space()
    n, n_raw = sp.count()
    radices = [len(v) for v in VALUES]
    valid = sp.valid_raw()
    digits = sp.valid_digits()
    rows = rows_of(digits)
    t0 = time.time()
    ms, checks = time_configs(rows)
    best = float(ms.min())
    target = 1.1 * best
    good = int(np.count_nonzero(ms <= target))
    log("space: %d valid of %d; exhaustive timing %.1f s; best %.4f ms, %d within 1.1x"
        % (n, n_raw, time.time() - t0, best, good))
    # the model: trees fitted on ncu profiles of a uniform sample
    rng = np.random.default_rng(12345)
    samp = np.sort(rng.choice(n, size=max(4, int(round(sample_frac * n))), replace=False))
    t0 = time.time()
    C = profile(rows[samp], workdir=workdir)
    prof_s = time.time() - t0
    model = fit_model(digits[samp].astype(np.int64), C, depth, radices, ROLES)
    m = kt.Model(sp, model)
    log("model: depth-%d trees on ncu profiles of %d configurations (%.1f s)" % (depth, len(samp), prof_s))
    pos = {int(r): i for i, r in enumerate(valid)}
    searches = []
    for seed in seeds:
        s = kt.Search(sp, m, k=k, seed=seed, cores=cores)
        cur = pos[s.current()]
        t_cur = float(time_configs(rows[[cur]])[0][0])
        tests, best_seen, steps, ncu_s = 1, t_cur, 0, 0.0
        trace = [(tests, best_seen)]
        while best_seen > target and tests < max_tests:
            t1 = time.time()
            c = profile(rows[[pos[s.current()]]], workdir=workdir)[0]
            ncu_s += time.time() - t1
            raw, _ = s.step(c)
            if len(raw) == 0:
                break
            idx = [pos[int(x)] for x in raw]
            t_pick, _ = time_configs(rows[idx])
            s.report(t_pick)
            tests += len(raw)
            steps += 1
            best_seen = min(best_seen, float(t_pick.min()))
            trace.append((tests, best_seen))
        searches.append({"seed": int(seed), "tests": tests, "steps": steps, "reached": best_seen <= target,
                         "best_ms": best_seen, "ncu_seconds": ncu_s, "trace": trace})
        log("seed %d: %d tests (%d steps) to %.4f ms (%s)" % (seed, tests, steps, best_seen,
                                                          "within 1.1x" if best_seen <= target else "not reached"))
    # uniform random draws without replacement: expected tests to the first of `good`
    random_expect = (n + 1) / (good + 1)
    return {
        "kernel": "direct Coulomb summation, 512 x 512 grid points, 4096 charges (live/coulomb.cu)",
        "space": {"names": NAMES, "values": VALUES, "n_valid": int(n), "n_raw": int(n_raw),
                  "constraints": "BX * BY >= 64; OUT * UNROLL <= 16"},
        "best_ms": best, "within_1_1x": good, "checksums_equal": bool(np.all(checks == checks[0])),
        "model": {"kind": "trees", "depth": depth, "sample": int(len(samp)), "profile_seconds": prof_s},
        "k": k, "searches": searches,
        "median_tests": float(np.median([x["tests"] for x in searches])),
        "random_expected_tests": random_expect,
    }


def main(argv: Optional[Sequence[str]] = None) -> int:
    ap = argparse.ArgumentParser(description="counter-guided search on real ncu profiles")
    ap.add_argument("--seeds", default="0,1,2")
    ap.add_argument("--k", type=int, default=5)
    ap.add_argument("--max-tests", type=int, default=120)
    ap.add_argument("--out", default=None)
    a = ap.parse_args(argv)
    rec = run(seeds=[int(x) for x in a.seeds.split(",")], k=a.k, max_tests=a.max_tests)
    text = json.dumps(rec)
    if a.out:
        with open(a.out, "w") as f:
            f.write(text + "\n")
    print(text)
    return 0


if __name__ == "__main__":
    raise SystemExit(main())
