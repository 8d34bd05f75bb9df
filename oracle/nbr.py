"""Neighbourhood-restricted scoring (oracle).

Test infrastructure only: tests, the package smoke check and the bench's CPU
baseline use it; the library never does.

The paper suggests, for spaces too large to score whole, scoring only a
neighbourhood of c_profile (a footnote of Section 3.5), and lists following
the scores as a local search as future work (Section 3.8.1).  Readings of
this build:
  * the neighbourhood of radius R (1 or 2): the valid configurations whose
    digit vectors differ from c_profile's in 1 .. R parameters (Hamming
    distance on the digits); a step's candidates are its unevaluated members;
  * canonical candidate order: distance 1 first (parameter j ascending, then
    the new digit ascending), then distance 2 (pairs i < j in lexicographic
    order, then the new digit of i ascending, then that of j ascending);
  * a step scores the candidates with Eq. score, normalises over them (s_min
    and s_max of the candidates), and draws k without replacement with the
    full step's integer weights and Philox draws, the prefix sums running in
    the canonical order; or it takes the top k, ties to the lower raw index;
  * with fewer than k candidates the step returns all of them (drawn in the
    same way); with none it returns none.  The step counter advances either
    way.
Parity unpinned beyond the definition: the pins check the neighbourhood
against brute force and its size formula, and the reduction to the full
step's top-k when the neighbourhood covers the whole space.
"""
from __future__ import annotations

from typing import List

import numpy as np

from . import expert, score, select
from .search import OracleSearch


def count(radices: List[int], radius: int) -> int:
    """Size of the radius-R neighbourhood in the raw space."""
    r = [x - 1 for x in radices]
    c = sum(r)
    if radius >= 2:
        c += sum(r[i] * r[j] for i in range(len(r)) for j in range(i + 1, len(r)))
    return c


def neighbour_digits(radices: List[int], cp: np.ndarray, radius: int) -> np.ndarray:
    """Digit vectors of the raw neighbourhood of cp, in the canonical order."""
    cp = np.asarray(cp, dtype=np.int64)
    out = []
    P = len(radices)
    for j in range(P):
        for d in range(radices[j]):
            if d != cp[j]:
                v = cp.copy(); v[j] = d
                out.append(v)
    if radius >= 2:
        for i in range(P):
            for j in range(i + 1, P):
                for di in range(radices[i]):
                    if di == cp[i]:
                        continue
                    for dj in range(radices[j]):
                        if dj == cp[j]:
                            continue
                        v = cp.copy(); v[i] = di; v[j] = dj
                        out.append(v)
    return np.array(out, dtype=np.int64).reshape(-1, P)


class NbrSearch(OracleSearch):
    """Algorithm 1 with each step restricted to c_profile's neighbourhood."""

    def __init__(self, desc, model: dict, radius: int = 1, **kw):
        super().__init__(desc, model, **kw)
        assert radius in (1, 2)
        self.radius = radius
        radices = desc.radices
        self.strides = np.array([int(np.prod(radices[j + 1:])) for j in range(len(radices))],
                                dtype=np.int64)

    def candidates(self) -> np.ndarray:
        """TS positions of the unevaluated valid neighbours, canonical order."""
        nd = neighbour_digits(self.desc.radices, self.digits[self.cprof], self.radius)
        if len(nd) == 0:
            return np.zeros(0, dtype=np.int64)
        raws = nd @ self.strides
        pos = np.searchsorted(self.valid, raws)
        ok = pos < len(self.valid)
        ok[ok] = self.valid[pos[ok]] == raws[ok]
        pos = pos[ok]
        return pos[~self.evaluated[pos]]

    def step(self, counters):
        cand = self.candidates()
        self.last = []
        if len(cand) == 0:
            self.step_no += 1
            return [], []
        d32 = expert.delta_vector(self.roles, counters, self.inst_reaction,
                                  self.cores).astype(np.float32)
        s = score.score_fp32(self.pred[self.cprof], self.pred[cand], d32)
        if self.mode == "topk":
            pick = select.topk(s, self.valid[cand], self.k)
        else:
            sn = select.normalise_fp32(s, s.min(), s.max(), self.gamma)
            pick = select.weighted_draws(select.quantise(sn), self.k, self.seed,
                                         self.search_id, self.step_no)
        chosen = [int(cand[p]) for p in pick]
        self.evaluated[chosen] = True
        self.step_no += 1
        self.last = chosen
        return [int(self.valid[i]) for i in chosen], [float(s[p]) for p in pick]
