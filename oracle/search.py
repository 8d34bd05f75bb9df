"""Algorithm 1 end to end (oracle).

One call of ``step`` is one iteration of Algorithm 1's outer loop after the
profiling run: bottlenecks and Delta from the measured counters of c_profile,
the scores of every configuration not yet evaluated, k draws (or the top k),
and the drawn configurations marked evaluated.  ``report`` takes their
runtimes and makes the fastest of the batch the next c_profile.

Readings: k = n draws per step (the text's "n steps without counters");
t is reset to infinity before the batch, so the next c_profile is the fastest
of the batch even when it is slower than the previous one, and on equal
runtimes the later draw wins (Algorithm 1 tests t' <= t); the initial
c_profile is a uniform draw over TS (Philox domain 1) and counts as evaluated.
Predictions are made once per configuration: the model and the space do not
change during a search.
"""
from __future__ import annotations

from typing import List

import numpy as np

from . import expert, score, select, space, trees


class OracleSearch:
    def __init__(self, desc, model: dict, k: int = 5, inst_reaction: float = 0.7,
                 gamma: float = select.GAMMA, cores: float = 1000.0, seed: int = 0,
                 search_id: int = 0, mode: str = "sample", valid=None, pred=None,
                 uniform: bool = False):
        self.desc = desc
        self.model = model
        self.roles = model["roles"]
        self.k, self.inst_reaction, self.gamma = k, inst_reaction, gamma
        self.cores, self.seed, self.search_id, self.mode = cores, seed, search_id, mode
        self.uniform = uniform            # unweighted random search baseline
        self.valid = space.enumerate_valid(desc) if valid is None else np.asarray(valid)
        self.digits = space.decode(desc.radices, self.valid)
        self.pred = trees.predict(model, self.digits) if pred is None else pred
        self.evaluated = np.zeros(len(self.valid), dtype=bool)
        self.step_no = 0
        n = len(self.valid)
        u = select.uniform_u64(seed, search_id, 0, 0, 1)
        self.cprof = select.scaled_draw(u, n)
        self.evaluated[self.cprof] = True
        self.last = []

    @property
    def cprof_raw(self) -> int:
        return int(self.valid[self.cprof])

    def scores(self, counters):
        """(s fp32 over all TS, delta64) for the measured counters."""
        d64 = expert.delta_vector(self.roles, counters, self.inst_reaction, self.cores)
        d32 = d64.astype(np.float32)
        s = score.score_fp32(self.pred[self.cprof], self.pred, d32)
        return s, d64

    def step(self, counters):
        s, _ = self.scores(counters)
        free = ~self.evaluated
        if self.mode == "topk":
            pos = np.nonzero(free)[0]
            pick = [int(pos[i]) for i in select.topk(s[pos], self.valid[pos], self.k)]
        else:
            if self.uniform:
                w = np.where(free, 1, 0).astype(np.uint64)
            else:
                w = np.zeros(len(s), dtype=np.uint64)
                if free.any():
                    sf = s[free]
                    sn = select.normalise_fp32(sf, sf.min(), sf.max(), self.gamma)
                    w[free] = select.quantise(sn)
            pick = select.weighted_draws(w, self.k, self.seed, self.search_id, self.step_no)
        self.evaluated[pick] = True
        self.step_no += 1
        self.last = pick
        return [int(self.valid[i]) for i in pick], [float(s[i]) for i in pick]

    def report(self, runtimes: List[float]) -> None:
        t = np.inf
        for i, rt in zip(self.last, runtimes):
            if rt <= t:
                t = rt
                self.cprof = i
