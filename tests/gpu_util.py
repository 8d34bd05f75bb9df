"""Helpers for the GPU parity tests (seeded inputs, oracle runs)."""
import numpy as np

import workloads as W
from workloads.synth import SyntheticGPU
from workloads.trees import random_model
from oracle import search as osearch, space as ospace


def run_pair(desc, model, counters_fn, steps, k=5, seed=0, select="sample", valid=None,
             pred=None, runtime_fn=None, kt=None, gamma=-0.25, inst_reaction=0.7, flags=0,
             fused=None):
    """Drive the library and the oracle through the same search; return the
    per-step (gpu_raw, gpu_score, oracle_raw, oracle_score).  fused: the
    search's step shape (ktune_search_set_fused), None for its default."""
    sp = kt.Space.from_desc(desc, flags=flags)
    m = kt.Model(sp, model)
    sel = kt.KTUNE_SELECT_TOPK if select == "topk" else kt.KTUNE_SELECT_SAMPLE
    s = kt.Search(sp, m, k=k, seed=seed, select=sel, gamma=gamma, inst_reaction=inst_reaction)
    if fused is not None:
        s.set_fused(fused)
    o = osearch.OracleSearch(desc, model, k=k, seed=seed, mode=select, valid=valid, pred=pred,
                             gamma=gamma, inst_reaction=inst_reaction)
    assert s.current() == o.cprof_raw
    out = []
    for _ in range(steps):
        c = counters_fn(s.current())
        g_raw, g_sc = s.step(c)
        o_raw, o_sc = o.step(c)
        out.append((list(g_raw), np.asarray(g_sc, np.float32), o_raw, np.float32(o_sc)))
        if not o_raw:
            break
        rts = runtime_fn(g_raw) if runtime_fn else np.arange(len(g_raw), 0, -1, dtype=float)
        s.report(rts)
        o.report(list(rts))
    return out
