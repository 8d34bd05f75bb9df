"""A seeded synthetic GPU: counters and runtime of every configuration.

It stands in for the profiler runs of the paper's training and autotuning
phases (Section 3.3, Algorithm 1), whose recorded benchmark data are not
available.  Every "ops" counter is a sigmoid of per-parameter piecewise-linear
terms in the scaled log2 of the parameter value plus four pairwise products;
the runtime is the largest of a few subsystem times (memory levels, issue,
instruction pipes), stretched when too few threads run; and the utilisation
counters are each subsystem's time over that runtime, which ties the measured
stress to the runtime the way the method assumes (Section 3.2).

Inputs are digit tuples (the index of each parameter's value).  Nothing here
implements the search method itself.
"""
from __future__ import annotations

from typing import List

import numpy as np

from . import ROLE, SpaceDesc

# latent channels of the synthetic function
_CH = ["DRAM_RT", "DRAM_WT", "L2_RT", "L2_WT", "TEX_RWT", "LOC_O", "SHR_LT",
       "SHR_WT", "EXE", "F32", "F64", "INT", "MISC", "LDST", "CONT", "BCONV",
       "GLOBAL", "WARP_E", "WARP_NP_E"]
_INST = ["F32", "F64", "INT", "MISC", "LDST", "CONT", "BCONV"]


def _sigmoid(z):
    return 1.0 / (1.0 + np.exp(-z))


class SyntheticGPU:
    """Seeded synthetic performance function over a tuning space.

    ``evaluate(digits)`` returns ``(counters, runtime)``: counters as float32
    in the order of ``roles`` (a counter layout), runtime as float64.
    """

    def __init__(self, space: SpaceDesc, roles: List[int], seed: int = 0,
                 cores: int = 1000):
        self.space = space
        self.roles = list(roles)
        self.cores = cores
        rng = np.random.default_rng([int(seed), 0x5E3D])
        P = space.n_params
        # per-parameter scaled log2(1 + value) in [-1, 1]
        self.u = []
        for vals in space.values:
            lv = np.log2(1.0 + np.asarray(vals, dtype=np.float64))
            lo, hi = lv.min(), lv.max()
            self.u.append(np.zeros_like(lv) if hi == lo else 2.0 * (lv - lo) / (hi - lo) - 1.0)
        n_inert = sum(1 for r in self.roles if r == ROLE["INERT"])
        names = _CH + ["INERT%d" % i for i in range(n_inert)]
        self.tab = {}    # channel -> list over params of per-digit offsets
        self.pairs = {}  # channel -> (a[4], b[4], w[4])
        self.bias = {}
        for ch in names:
            strong = rng.choice(P, size=min(P, 3), replace=False)
            per = []
            for j in range(P):
                scale = 1.2 if j in strong else 0.2
                knots = np.concatenate(([-1.0], np.sort(rng.uniform(-1, 1, 3)), [1.0]))
                ys = rng.normal(0.0, scale, size=5)
                per.append(np.interp(self.u[j], knots, ys))
            self.tab[ch] = per
            a = rng.integers(0, P, size=4)
            b = (a + rng.integers(1, max(2, P), size=4)) % P
            self.pairs[ch] = (a, b, rng.normal(0.0, 0.8, size=4))
            self.bias[ch] = rng.normal(0.0, 0.4)
        self.bias["LOC_O"] -= 2.5
        # capacities from a sample of the unconstrained cross product
        probe = np.stack([rng.integers(0, r, size=4096) for r in space.radices], axis=1)
        raw = self._raw_counters(probe)
        loads = self._loads(raw)
        self.cap = {}
        for m in ("dram", "l2", "tex", "shr", "issue"):
            self.cap[m] = float(np.median(loads[m])) * rng.uniform(0.7, 1.3)

    # -- latent channels ---------------------------------------------------
    def _z(self, ch: str, d: np.ndarray) -> np.ndarray:
        z = np.full(d.shape[0], self.bias[ch])
        for j, t in enumerate(self.tab[ch]):
            z += t[d[:, j]]
        a, b, w = self.pairs[ch]
        for q in range(4):
            z += w[q] * self.u[a[q]][d[:, a[q]]] * self.u[b[q]][d[:, b[q]]]
        return z

    def _raw_counters(self, d: np.ndarray) -> dict:
        d = np.asarray(d, dtype=np.int64)
        c = {}
        for ch in ("DRAM_RT", "DRAM_WT", "L2_RT", "L2_WT", "TEX_RWT", "SHR_LT", "SHR_WT"):
            c[ch] = 8000.0 * (0.05 + 0.95 * _sigmoid(self._z(ch, d)))
        c["LOC_O"] = 100.0 * _sigmoid(self._z("LOC_O", d))
        c["EXE"] = 250.0 * (0.05 + 0.95 * _sigmoid(self._z("EXE", d)))
        # one dominant class (FP32) and the rest shared by the others
        f32 = 0.95 * _sigmoid(self._z("F32", d) + 0.5)
        e = {x: np.exp(self._z(x, d)) for x in _INST if x != "F32"}
        tot = sum(e.values())
        c["F32"] = 32.0 * c["EXE"] * f32
        for x in e:
            c[x] = 32.0 * c["EXE"] * (0.97 - f32) * e[x] / tot
        c["GLOBAL"] = 10.0 ** (3.5 + 3.0 * _sigmoid(self._z("GLOBAL", d)))
        c["WARP_E"] = 100.0 * (0.7 + 0.3 * _sigmoid(self._z("WARP_E", d)))
        c["WARP_NP_E"] = 100.0 * (0.85 + 0.15 * _sigmoid(self._z("WARP_NP_E", d)))
        for ch in self.tab:
            if ch.startswith("INERT"):
                c[ch] = 1000.0 * _sigmoid(self._z(ch, d))
        return c

    @staticmethod
    def _loads(c: dict) -> dict:
        return {"dram": c["DRAM_RT"] + c["DRAM_WT"] + 40.0 * c["LOC_O"],
                "l2": c["L2_RT"] + c["L2_WT"],
                "tex": c["TEX_RWT"],
                "shr": c["SHR_LT"] + c["SHR_WT"],
                "issue": 32.0 * c["EXE"] * (100.0 / c["WARP_E"])}

    # -- public --------------------------------------------------------------
    def evaluate(self, digits: np.ndarray):
        """Counters (float32, layout order) and runtime (float64) per config."""
        d = np.atleast_2d(np.asarray(digits, dtype=np.int64))
        c = self._raw_counters(d)
        L = self._loads(c)
        t = {m: L[m] / self.cap[m] for m in L}
        t_core = np.maximum.reduce(list(t.values()))
        b_par = np.maximum(0.0, 1.0 - c["GLOBAL"] / (5.0 * self.cores))
        runtime = t_core * (1.0 + 0.5 * b_par)
        stress = {
            "INST_ISSUE_U": 100.0 * t["issue"] / t_core,
            "DRAM_U": 100.0 * t["dram"] / t_core,
            "L2_U": 100.0 * t["l2"] / t_core,
            "TEX_U": 100.0 * t["tex"] / t_core,
            "SHR_U": 100.0 * t["shr"] / t_core,
            "SM_E": 100.0 * np.minimum(1.0, c["GLOBAL"] / (2.0 * self.cores)),
        }
        name_of = {"INST_F32": "F32", "INST_F64": "F64", "INST_INT": "INT",
                   "INST_MISC": "MISC", "INST_LDST": "LDST", "INST_CONT": "CONT",
                   "INST_BCONV": "BCONV", "INST_EXE": "EXE"}
        from . import ROLE_NAMES
        out = np.empty((d.shape[0], len(self.roles)), dtype=np.float64)
        inert_i = 0
        for k, r in enumerate(self.roles):
            nm = ROLE_NAMES[r]
            if nm == "INERT":
                out[:, k] = c["INERT%d" % inert_i]
                inert_i += 1
            elif nm in stress:
                out[:, k] = stress[nm]
            elif nm in name_of:
                out[:, k] = c[name_of[nm]]
            else:
                out[:, k] = c[nm]
        return out.astype(np.float32), runtime

    def counter_ranges(self) -> np.ndarray:
        """Nominal full-scale value of each counter (for range-normalised
        errors and MLP output scaling)."""
        from . import ROLE_NAMES
        rng_of = {"LOC_O": 100.0, "INST_EXE": 250.0, "GLOBAL": 1e6, "INERT": 1000.0}
        out = []
        for r in self.roles:
            nm = ROLE_NAMES[r]
            if nm in rng_of:
                out.append(rng_of[nm])
            elif nm.startswith("INST_") and nm != "INST_ISSUE_U":
                out.append(32.0 * 250.0)
            elif nm.endswith("_U") or nm in ("SM_E", "WARP_E", "WARP_NP_E"):
                out.append(100.0)
            else:
                out.append(8000.0)
        return np.asarray(out, dtype=np.float64)


def add_noise(counters: np.ndarray, seed: int, sigma: float = 0.02) -> np.ndarray:
    """Multiplicative Gaussian noise (1 + sigma z) on profiled counters."""
    rng = np.random.default_rng([int(seed), 0x401E])
    z = rng.standard_normal(counters.shape)
    return np.maximum(0.0, counters * (1.0 + sigma * z)).astype(np.float32)


def sample_indices(n: int, fraction: float, seed: int) -> np.ndarray:
    """Sorted uniform sample (without replacement) of round(fraction * n)
    positions out of n, at least one."""
    rng = np.random.default_rng([int(seed), 0x5A3B])
    m = max(1, int(round(fraction * n)))
    return np.sort(rng.choice(n, size=m, replace=False))
