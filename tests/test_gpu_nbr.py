"""Neighbourhood-restricted steps (ktune_search_set_neighbourhood) against the
oracle: the candidates, their scores, the draws (or top-k) and the step's
statistics bit for bit, for Hamming radius 1 and 2, on materialised spaces of
1.8k to 491k raw configurations; the graph path; the switch back to
whole-space steps; an exhausted neighbourhood; and the refusals."""
import numpy as np
import pytest

import workloads as W
from workloads.synth import SyntheticGPU
from workloads.trees import random_model
from oracle import nbr as onbr, space as ospace
from oracle.search import OracleSearch

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def kt():
    import torch
    assert torch.cuda.is_available()
    from paper_2102_05297_gb300 import ktune
    return ktune


def load(name):
    return W.space_tiny_block_tile() if name == "tiny" else W.load_space(name)


def drive(kt, desc, model, gpu, radius, select, steps, k=5, seed=0, stream=None):
    sp = kt.Space.from_desc(desc)
    m = kt.Model(sp, model)
    sel = kt.KTUNE_SELECT_TOPK if select == "topk" else kt.KTUNE_SELECT_SAMPLE
    s = kt.Search(sp, m, k=k, seed=seed, select=sel, stream=stream)
    s.set_neighbourhood(radius)
    o = onbr.NbrSearch(desc, model, radius=radius, k=k, seed=seed, mode=select)
    assert s.current() == o.cprof_raw
    n_steps = 0
    for _ in range(steps):
        c = gpu.evaluate(ospace.decode(desc.radices, [s.current()]))[0][0]
        n_cand = len(o.candidates())
        g_raw, g_sc = s.step(c)
        o_raw, o_sc = o.step(c)
        assert list(g_raw) == o_raw
        assert np.array_equal(np.asarray(g_sc, np.float32), np.float32(o_sc))
        st = s.stats()
        assert st.n_scored == n_cand
        if not o_raw:
            break
        rts = list(gpu.evaluate(ospace.decode(desc.radices, o_raw))[1])
        s.report(rts)
        o.report(rts)
        n_steps += 1
    return s, o, n_steps


@pytest.mark.parametrize("name,K,depth,radius,select", [
    ("tiny", 16, 8, 1, "sample"), ("tiny", 16, 8, 2, "sample"), ("tiny", 16, 8, 2, "topk"),
    ("batch_3", 32, 10, 1, "topk"), ("batch_3", 32, 10, 2, "sample"),
    ("batch_4", 40, 12, 1, "sample"), ("batch_4", 40, 12, 2, "topk")])
def test_steps_match_oracle(kt, name, K, depth, radius, select):
    desc = load(name)
    roles = W.layout(K)
    model = random_model(desc.radices, roles, depth=depth, seed=K + radius)
    gpu = SyntheticGPU(desc, roles, seed=radius)
    _, _, n = drive(kt, desc, model, gpu, radius, select, steps=6, seed=radius + 3)
    assert n >= 1


def test_graph_path_and_back_to_whole_space(kt):
    import torch
    desc = load("batch_3")
    roles = W.layout(16)
    model = random_model(desc.radices, roles, depth=8, seed=7)
    gpu = SyntheticGPU(desc, roles, seed=7)
    s, o, n = drive(kt, desc, model, gpu, 2, "sample", steps=4, seed=2, stream=torch.cuda.Stream())
    assert n == 4
    s.set_neighbourhood(0)                      # whole-space steps from here on
    for _ in range(3):
        c = gpu.evaluate(ospace.decode(desc.radices, [s.current()]))[0][0]
        g_raw, g_sc = s.step(c)
        o_raw, o_sc = OracleSearch.step(o, c)
        assert list(g_raw) == o_raw
        assert np.array_equal(np.asarray(g_sc, np.float32), np.float32(o_sc))
        rts = list(gpu.evaluate(ospace.decode(desc.radices, o_raw))[1])
        s.report(rts)
        o.report(rts)


def test_exhausted_neighbourhood(kt):
    desc = W.SpaceDesc("one", ["a", "b"], [[0, 1], [7]], [])
    roles = W.layout(16)
    model = random_model(desc.radices, roles, depth=2, seed=0)
    sp = kt.Space.from_desc(desc)
    s = kt.Search(sp, kt.Model(sp, model), k=3, seed=0)
    s.set_neighbourhood(1)
    c = np.full(16, 10.0, np.float32)
    raw, _ = s.step(c)
    assert len(raw) == 1 and s.stats().n_scored == 1
    raw2, _ = s.step(c)                         # its only neighbour is evaluated
    assert len(raw2) == 0 and s.stats().n_scored == 0
    with pytest.raises(kt.KtuneError):
        kt.Batch([s])


def test_refusals(kt):
    desc = load("batch_3")
    roles = W.layout(16)
    model = random_model(desc.radices, roles, depth=6, seed=1)
    sp = kt.Space.from_desc(desc)
    s = kt.Search(sp, kt.Model(sp, model), k=5)
    for bad in (-1, 3):
        with pytest.raises(kt.KtuneError):
            s.set_neighbourhood(bad)
    otf = kt.Space.from_desc(desc, flags=kt.KTUNE_ON_THE_FLY)
    s2 = kt.Search(otf, kt.Model(otf, model), k=5)
    with pytest.raises(kt.KtuneError):
        s2.set_neighbourhood(1)
