"""Cached predictions (ktune_search_set_cached): steps scored from a cache
filled once give the same selections and scores, bit for bit, as the fused
steps that predict every configuration again -- for tree ensembles (random
trees with early leaves and exact-zero leaves) and for the MLP (an exact
network, whose fused steps match the oracle bit for bit) -- and the cache is
refused where it does not apply."""
import numpy as np
import pytest

import workloads as W
from workloads.synth import SyntheticGPU
from workloads.trees import random_model
from oracle import space as ospace

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def kt():
    import torch
    assert torch.cuda.is_available()
    from paper_2102_05297_gb300 import ktune
    return ktune


def drive(s, gpu, radices, steps, k=None):
    out = []
    for _ in range(steps):
        c = gpu.evaluate(ospace.decode(radices, [s.current()]))[0][0]
        raw, sc = s.step(c, k)
        out.append((list(raw), [float(x) for x in sc]))
        s.report(gpu.evaluate(ospace.decode(radices, raw))[1])
    return out


@pytest.mark.parametrize("name,K,depth,shape", [("batch_4", 32, 12, None), ("batch_3", 40, 10, None),
                                                ("batch_2", 16, 6, None), ("batch_4", 32, 12, 2),
                                                ("batch_3", 40, 10, 2)])
def test_cached_tree_steps_equal_fused(kt, name, K, depth, shape):
    """Cached steps against steps that predict again; shape 2: the steps
    that predict again run as one persistent kernel."""
    d = W.load_space(name)
    roles = W.layout(K)
    model = random_model(d.radices, roles, depth=depth, seed=K + depth)
    gpu = SyntheticGPU(d, roles, seed=1)
    sp = kt.Space.from_desc(d)
    m = kt.Model(sp, model)
    a = kt.Search(sp, m, k=6, seed=9)
    b = kt.Search(sp, m, k=6, seed=9)
    if shape is not None:
        a.set_fused(shape)
        b.set_fused(shape)
    b.set_cached(True)
    assert drive(a, gpu, d.radices, 8) == drive(b, gpu, d.radices, 8)
    st_a, st_b = a.stats(), b.stats()
    assert (st_a.n_active, st_a.s_min, st_a.s_max) == (st_b.n_active, st_b.s_min, st_b.s_max)
    b.set_cached(False)          # back to fused steps, same trajectory
    a.set_cached(False)
    assert drive(a, gpu, d.radices, 2) == drive(b, gpu, d.radices, 2)


def test_cached_graph_path(kt):
    import torch
    d = W.load_space("batch_4")
    roles = W.layout(32)
    sp = kt.Space.from_desc(d)
    m = kt.Model(sp, random_model(d.radices, roles, depth=12, seed=3))
    gpu = SyntheticGPU(d, roles, seed=1)
    stream = torch.cuda.Stream()
    a = kt.Search(sp, m, k=5, seed=4, stream=stream)
    b = kt.Search(sp, m, k=5, seed=4)
    a.set_cached(True)
    assert drive(a, gpu, d.radices, 5) == drive(b, gpu, d.radices, 5)


def test_cached_mlp_steps_equal_fused(kt):
    from test_gpu_mlp import exact_params, tiny_setup
    desc, roles, gpu, valid, dig, C = tiny_setup(seed=2)
    sp = kt.Space.from_desc(desc)
    mlp = kt.Mlp(sp, roles, gpu.counter_ranges(), max_batch=64)
    mlp.set_params(exact_params(desc, mlp.F, len(roles), 2))
    model = kt.Model.from_mlp(mlp)
    a = kt.Search(sp, model, k=5, seed=2)
    b = kt.Search(sp, model, k=5, seed=2)
    b.set_cached(True)
    assert drive(a, gpu, desc.radices, 10) == drive(b, gpu, desc.radices, 10)


def test_cache_refused(kt):
    d = W.load_space("batch_2")
    roles = W.layout(16)
    model = random_model(d.radices, roles, depth=6, seed=1)
    otf = kt.Space.from_desc(d, flags=kt.KTUNE_ON_THE_FLY)
    s1 = kt.Search(otf, kt.Model(otf, model), k=5)
    with pytest.raises(kt.KtuneError):
        s1.set_cached(True)                       # nothing materialised to predict
    sp = kt.Space.from_desc(d)
    s2 = kt.Search(sp, kt.Model(sp, model), k=5, select=kt.KTUNE_SELECT_TOPK)
    with pytest.raises(kt.KtuneError):
        s2.set_cached(True)                       # top-k selection
