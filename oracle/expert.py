"""Expert system: bottlenecks B and the Delta-PC reaction (oracle).

Section 3.4.1 (Eqs. "global-read", "global-write", "local", "inst_fitted",
"fp32", "maxutil", "issue", "paral") and Section 3.4.2 (memory reaction,
Eq. "fp32_reaction", parallelism reaction).  Float64 throughout, each formula
evaluated left to right as printed.

Readings where the paper is silent or inconsistent:
  * Counters are taken in the Volta-and-newer form: utilisations are
    percentages in [0, 100], so every "X_U / 10" of the equations (written for
    the older 0-10 scale) is read as pct / 100; LOC_O is a percentage too.
  * ins_util = min(1, INST_ISSUE_U / 50) (the Volta+ form).
  * Every bottleneck is clamped to [0, 1] and every Delta to [-1, 1], the
    ranges the paper states for them.
  * RT + WT = 0 gives both memory bottlenecks 0; ins_fitted = 0 gives every
    instruction fraction 0; WARP_E or WARP_NP_E equal to 0 count as 100.
  * The reaction of b_issue goes to INST_ISSUE_U (by analogy with the other
    instruction reactions; the paper files INST_ISSUE_U under Ops).
  * Counters missing from a layout take neutral values: LOC_O = 0, the four
    optional instruction classes = 0, SM_E = WARP_E = WARP_NP_E = 100, and an
    unknown thread count means no parallelism bottleneck.
Parity: pinned by hand-computed cases of every equation.
"""
from __future__ import annotations

from typing import Dict, List

import numpy as np

import workloads as W

INST_CLASSES = ["INST_F32", "INST_F64", "INST_INT", "INST_MISC", "INST_LDST",
                "INST_CONT", "INST_BCONV"]
DEFAULTS = {"LOC_O": 0.0, "INST_F64": 0.0, "INST_MISC": 0.0, "INST_CONT": 0.0,
            "INST_BCONV": 0.0, "SM_E": 100.0, "WARP_E": 100.0, "WARP_NP_E": 100.0}


def _clamp01(x: float) -> float:
    return min(1.0, max(0.0, x))


def counters_by_name(roles: List[int], counters) -> Dict[str, float]:
    """Map a counter vector to role names (first occurrence wins; inert and
    unknown roles are dropped)."""
    pc: Dict[str, float] = {}
    for r, v in zip(roles, counters):
        nm = W.ROLE_NAMES[r]
        if nm != "INERT" and nm not in pc:
            pc[nm] = float(v)
    return pc


def _get(pc: Dict[str, float], name: str) -> float:
    if name in pc:
        return pc[name]
    if name in DEFAULTS:
        return DEFAULTS[name]
    return 0.0


def bottlenecks(pc: Dict[str, float], cores: float) -> Dict[str, float]:
    """B from measured counters (Section 3.4.1)."""
    B: Dict[str, float] = {}

    def mem(name, rt, wt, util):
        r, w, u = _get(pc, rt), _get(pc, wt), _get(pc, util)
        if r + w > 0.0:
            B[name + "_read"] = _clamp01(r / (r + w) * (u / 100.0))
            B[name + "_write"] = _clamp01(w / (r + w) * (u / 100.0))
        else:
            B[name + "_read"] = 0.0
            B[name + "_write"] = 0.0

    mem("dram", "DRAM_RT", "DRAM_WT", "DRAM_U")   # Eqs. global-read / global-write
    mem("l2", "L2_RT", "L2_WT", "L2_U")
    mem("shr", "SHR_LT", "SHR_WT", "SHR_U")
    B["tex"] = _clamp01(_get(pc, "TEX_U") / 100.0)
    # Eq. local
    B["local"] = _clamp01(_get(pc, "LOC_O") / 100.0 * max(
        _get(pc, "DRAM_U") / 100.0, _get(pc, "L2_U") / 100.0, _get(pc, "TEX_U") / 100.0))
    # Eq. inst_fitted
    we = _get(pc, "WARP_E"); we = 100.0 if we == 0.0 else we
    wn = _get(pc, "WARP_NP_E"); wn = 100.0 if wn == 0.0 else wn
    ins_fitted = 32.0 * _get(pc, "INST_EXE") * (100.0 / we) * (100.0 / wn)
    issue_u = _get(pc, "INST_ISSUE_U")
    ins_util = min(1.0, issue_u / 50.0)
    frac = {}
    for x in INST_CLASSES:
        frac[x] = _get(pc, x) / ins_fitted if ins_fitted > 0.0 else 0.0
        B[x] = _clamp01(frac[x] * ins_util)                # Eq. fp32 and analogues
    util_max = max(frac.values())                           # Eq. maxutil
    B["issue"] = _clamp01(util_max * ((100.0 - issue_u) / 100.0))   # Eq. issue
    B["sm"] = _clamp01((100.0 - _get(pc, "SM_E")) / 100.0)
    if "GLOBAL" in pc:                                      # Eq. paral
        threads = pc["GLOBAL"]
        B["paral"] = _clamp01(max(0.0, (cores * 5.0 - threads) / (cores * 5.0)))
    else:
        B["paral"] = 0.0
    return B


def reaction(b: float, inst_reaction: float) -> float:
    """Eq. fp32_reaction."""
    if b <= inst_reaction:
        return 0.0
    return -(b - inst_reaction) / (1.0 - inst_reaction)


def delta_by_name(B: Dict[str, float], inst_reaction: float) -> Dict[str, float]:
    """Delta-PC_ops (Section 3.4.2)."""
    D = {"DRAM_RT": -B["dram_read"], "DRAM_WT": -B["dram_write"],
         "L2_RT": -B["l2_read"], "L2_WT": -B["l2_write"],
         "SHR_LT": -B["shr_read"], "SHR_WT": -B["shr_write"],
         "TEX_RWT": -B["tex"], "LOC_O": -B["local"]}
    for x in INST_CLASSES:
        D[x] = reaction(B[x], inst_reaction)
    D["INST_ISSUE_U"] = reaction(B["issue"], inst_reaction)
    D["SM_E"] = B["sm"]
    D["GLOBAL"] = B["paral"]
    return {k: min(1.0, max(-1.0, v)) for k, v in D.items()}


def delta_vector(roles: List[int], counters, inst_reaction: float = 0.7,
                 cores: float = 1000.0) -> np.ndarray:
    """Delta for each counter slot of the layout (float64); 0 for counters
    without a reaction, for inert counters and for repeated roles."""
    pc = counters_by_name(roles, counters)
    D = delta_by_name(bottlenecks(pc, cores), inst_reaction)
    out = np.zeros(len(roles), dtype=np.float64)
    seen = set()
    for k, r in enumerate(roles):
        nm = W.ROLE_NAMES[r]
        if nm in D and nm not in seen:
            out[k] = D[nm]
            seen.add(nm)
    return out
