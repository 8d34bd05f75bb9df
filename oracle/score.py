"""Configuration score, Section 3.5 Eq. "score" (oracle).

s(c) = sum over p in PC_used of  dpc_p * (pc_p(c) - pc_p(prof)) / (pc_p(c) + pc_p(prof))

with both counter vectors predicted by the model and PC_used the counters with
a Delta entry whose predictions are non-zero for both configurations.

Readings:
  * Sign of the numerator.  As printed, Eq. score has pc(prof) - pc(cand);
    with the Delta convention of Section 3.4.2 (negative = the counter should
    decrease) that gives a NEGATIVE score to a candidate that lowers a counter
    the expert system wants lowered, against Section 3.5's statement that
    higher scores go to configurations changing the counters in the required
    way and against the normalisation text (positive = preferred, negative =
    "seem worse than c_profile").  The consistent reading, used here, is
    pc(cand) - pc(prof) in the numerator.
  * Counters with Delta = 0 contribute nothing (so skipping them is exact); a
    counter is also left out when the denominator is 0 (possible only for
    signed predictions).
``score_def`` is the float64 definition.  ``score_fp32`` is the float32
decision path: for p ascending, term = delta_p * ((a - A) / (a + A)) with
a = pc_p(cand), A = pc_p(prof), each operation rounded to float32 and no fused
multiply-add; s starts at +0 and adds the term, or +0 when p is unused.
Parity: pinned by antisymmetry, zero for equal predictions, the bound
|s| <= sum |delta|, and hand-computed cases.
"""
from __future__ import annotations

import numpy as np


def score_def(pc_prof, pc_cand, delta) -> np.ndarray:
    A = np.asarray(pc_prof, dtype=np.float64)
    a = np.atleast_2d(np.asarray(pc_cand, dtype=np.float64))
    dl = np.asarray(delta, dtype=np.float64)
    s = np.zeros(a.shape[0], dtype=np.float64)
    with np.errstate(divide="ignore", invalid="ignore"):
        for p in range(a.shape[1]):
            used = (dl[p] != 0.0) & (A[p] != 0.0) & (a[:, p] != 0.0) & (a[:, p] + A[p] != 0.0)
            term = dl[p] * (a[:, p] - A[p]) / (a[:, p] + A[p])
            s += np.where(used, term, 0.0)
    return s


def score_fp32(pc_prof, pc_cand, delta32) -> np.ndarray:
    A = np.asarray(pc_prof, dtype=np.float32)
    a = np.atleast_2d(np.asarray(pc_cand, dtype=np.float32))
    dl = np.asarray(delta32, dtype=np.float32)
    s = np.zeros(a.shape[0], dtype=np.float32)
    with np.errstate(divide="ignore", invalid="ignore"):
        for p in range(a.shape[1]):
            den = a[:, p] + A[p]
            used = (dl[p] != 0) & (A[p] != 0) & (a[:, p] != 0) & (den != 0)
            q = (a[:, p] - A[p]) / den
            term = dl[p] * q
            s = s + np.where(used, term, np.float32(0.0))
    return s.astype(np.float32)
