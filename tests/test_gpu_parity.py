"""GPU parity against the CPU oracle, through the C ABI.

Bar: bit-exact on enumeration, predictions (tree leaves are stored values)
and selected indices; scores bit-exact against the oracle's float32 decision
path and within (K + 3) 2^-24 sum|delta| of its float64 definition."""
import json
import os

import numpy as np
import pytest

import workloads as W
from workloads.synth import SyntheticGPU, add_noise, sample_indices
from workloads.trees import random_model
from oracle import expert, score as oscore, search as osearch, space as ospace, trees as otrees

from gpu_util import run_pair

pytestmark = pytest.mark.gpu
GOLD = os.path.join(os.path.dirname(__file__), "golden")


@pytest.fixture(scope="module")
def kt():
    import torch
    assert torch.cuda.is_available()
    from paper_2102_05297_gb300 import ktune
    return ktune


def counts():
    with open(os.path.join(GOLD, "space_counts.json")) as f:
        return json.load(f)


# ---- enumeration ---------------------------------------------------------------
def test_enumeration_tiny_exact(kt):
    d = W.space_tiny_block_tile()
    sp = kt.Space.from_desc(d)
    assert sp.count() == (1824, 2304)
    np.testing.assert_array_equal(sp.valid_raw(), ospace.enumerate_valid(d))


@pytest.mark.parametrize("seed", range(8))
def test_enumeration_random_spaces_exact(kt, seed):
    rng = np.random.default_rng(seed)
    P = int(rng.integers(1, 9))
    values = []
    for _ in range(P):
        r = int(rng.integers(1, 17))
        values.append(sorted(int(x) for x in rng.choice(np.arange(-5, 60), size=r, replace=False)))
    code = []
    for _ in range(int(rng.integers(0, 4))):
        a, b = (int(x) for x in rng.integers(0, P, size=2))
        kind = rng.integers(0, 4)
        if kind == 0:
            code += W.c_divides(a, b)
        elif kind == 1:
            code += W.c_product_le([a, b], int(rng.integers(-10, 500)))
        elif kind == 2:
            code += W.c_implies_le(a, values[a][0], b, int(rng.integers(0, 40)))
        else:
            code += W.c_sum_le([a, b], int(rng.integers(0, 80)))
    d = W.SpaceDesc("r", ["p%d" % j for j in range(P)], values, code)
    sp = kt.Space.from_desc(d)
    ref = ospace.enumerate_valid(d)
    assert sp.count() == (len(ref), d.n_raw)
    if len(ref):
        np.testing.assert_array_equal(sp.valid_raw(), ref)


def test_enumeration_edge_cases(kt):
    # a single configuration; an all-invalid space; a ragged last tile
    one = W.SpaceDesc("one", ["a"], [[3]], [])
    assert kt.Space.from_desc(one).count() == (1, 1)
    none = W.SpaceDesc("none", ["a", "b"], [[1, 2], [3, 4]], [W.OP_CONST, 0, W.OP_REQUIRE])
    assert kt.Space.from_desc(none).count() == (0, 4)
    rag = W.SpaceDesc("rag", ["a", "b", "c"], [list(range(16)), list(range(16)), list(range(17 - 1))],
                      W.c_sum_le([0, 1, 2], 20))
    sp = kt.Space.from_desc(rag)
    np.testing.assert_array_equal(sp.valid_raw(), ospace.enumerate_valid(rag))
    odd = W.SpaceDesc("odd", ["a", "b"], [list(range(13)), list(range(7))], W.c_product_le([0, 1], 30))
    np.testing.assert_array_equal(kt.Space.from_desc(odd).valid_raw(), ospace.enumerate_valid(odd))


@pytest.mark.parametrize("name", ["mid_12p", "batch_1", "batch_4"])
def test_enumeration_full_size(kt, name):
    d = W.load_space(name)
    sp = kt.Space.from_desc(d)
    n_valid, n_raw = sp.count()
    assert (n_valid, n_raw) == (counts()[name]["n_valid"], d.n_raw)
    raw = sp.valid_raw()
    assert np.all(np.diff(raw) > 0)
    rng = np.random.default_rng(0)
    pick = rng.choice(len(raw), size=min(len(raw), 200000), replace=False)
    assert ospace.is_valid_raw(d, raw[pick]).all()
    # a contiguous window must equal the oracle's enumeration of that raw range
    lo, hi = int(raw[len(raw) // 3]), int(raw[len(raw) // 3]) + 300000
    window = np.arange(lo, min(hi, d.n_raw))
    ref = window[ospace.is_valid_raw(d, window)]
    got = raw[(raw >= lo) & (raw < min(hi, d.n_raw))]
    np.testing.assert_array_equal(got, ref)


def test_enumeration_large_count(kt):
    d = W.load_space("large_16p")
    sp = kt.Space.from_desc(d)
    assert sp.count() == (counts()["large_16p"]["n_valid"], d.n_raw)


def test_bad_descriptors(kt):
    with pytest.raises(kt.KtuneError):
        kt.Space([[2, 1]], [])                                   # not ascending
    with pytest.raises(kt.KtuneError):
        kt.Space([[1, 2]], [W.OP_VAL, 3, W.OP_REQUIRE])          # parameter out of range
    with pytest.raises(kt.KtuneError):
        kt.Space([[1, 2]], [W.OP_ADD, W.OP_REQUIRE])             # underflow
    with pytest.raises(kt.KtuneError):
        kt.Space([list(range(17))], [])                          # too many values


# ---- predictions ---------------------------------------------------------------
@pytest.mark.parametrize("depth", [1, 3, 8, 12])
def test_predictions_exact(kt, depth):
    import torch
    d = W.load_space("batch_3")
    roles = W.layout(16)
    model = random_model(d.radices, roles, depth=depth, seed=depth)
    sp = kt.Space.from_desc(d)
    m = kt.Model(sp, model)
    n = sp.count()[0]
    out = torch.empty((n, len(roles)), dtype=torch.float32, device="cuda")
    m.predict_device(0, n, out.data_ptr())
    torch.cuda.synchronize()
    valid = ospace.enumerate_valid(d)
    np.testing.assert_array_equal(sp.valid_raw(), valid)
    ref = otrees.predict(model, ospace.decode(d.radices, valid))
    np.testing.assert_array_equal(out.cpu().numpy(), ref)


def test_bad_models(kt):
    d = W.space_tiny_block_tile()
    sp = kt.Space.from_desc(d)
    good = random_model(d.radices, W.layout(16), depth=3, seed=0)
    bad_feat = {"roles": good["roles"], "trees": [dict(t) for t in good["trees"]]}
    f = bad_feat["trees"][0]["feature"].copy(); f[0] = 9
    bad_feat["trees"][0]["feature"] = f
    with pytest.raises(kt.KtuneError) as e:
        kt.Model(sp, bad_feat)
    assert e.value.code == kt.KTUNE_EMODEL
    bad_val = {"roles": good["roles"], "trees": [dict(t) for t in good["trees"]]}
    v = bad_val["trees"][1]["value"].copy(); v[:] = np.nan
    bad_val["trees"][1]["value"] = v
    with pytest.raises(kt.KtuneError):
        kt.Model(sp, bad_val)
    cyc = {"roles": [0], "trees": [{"feature": [0, -1], "threshold": [0, 0], "left": [1, -1],
                                    "right": [1, -1], "value": [0, 1]}]}
    with pytest.raises(kt.KtuneError):
        kt.Model(sp, cyc)


# ---- search steps ----------------------------------------------------------------
def _synthetic(desc, roles, fseed):
    gpu = SyntheticGPU(desc, roles, seed=fseed)
    return gpu, (lambda raw: gpu.evaluate(ospace.decode(desc.radices, [raw]))[0][0]), \
        (lambda raws: gpu.evaluate(ospace.decode(desc.radices, raws))[1])


def _check(out, K_bound=None):
    for g_raw, g_sc, o_raw, o_sc in out:
        assert g_raw == o_raw
        np.testing.assert_array_equal(g_sc, o_sc)


@pytest.mark.parametrize("seed,fused", [(0, None), (1, None), (2, None), (0, 0)])
def test_steps_tiny_fitted_model(kt, seed, fused):
    d = W.space_tiny_block_tile()
    roles = W.layout(16)
    gpu, cnt, rt = _synthetic(d, roles, seed)
    valid = ospace.enumerate_valid(d)
    dig = ospace.decode(d.radices, valid)
    samp = sample_indices(len(valid), 0.10, seed)
    model = otrees.fit_model(dig[samp], gpu.evaluate(dig[samp])[0], 8, d.radices, roles)
    out = run_pair(d, model, cnt, steps=40, seed=seed, valid=valid, runtime_fn=rt, kt=kt,
                   fused=fused)
    _check(out)


@pytest.mark.parametrize("K,depth,fused", [(16, 6, None), (32, 12, None), (40, 12, None),
                                           (40, 12, 0), (32, 1, None), (24, 14, 2)])
def test_steps_random_trees(kt, K, depth, fused):
    d = W.load_space("batch_2")
    roles = W.layout(K) if K in (16, 32, 40) else W.layout(40)[:K]
    model = random_model(d.radices, roles, depth=depth, seed=K)
    gpu, cnt, rt = _synthetic(d, roles, 3)
    out = run_pair(d, model, cnt, steps=12, k=7, seed=11, runtime_fn=rt, kt=kt, fused=fused)
    _check(out)


def test_steps_exhaust_space(kt):
    # 24 valid configurations, k = 5: the fifth step returns the last 3
    d = W.SpaceDesc("small", ["a", "b", "c"], [[1, 2, 4], [1, 2], [1, 2, 3, 4]], [])
    roles = W.layout(16)
    model = random_model(d.radices, roles, depth=2, seed=5)
    gpu, cnt, rt = _synthetic(d, roles, 1)
    out = run_pair(d, model, cnt, steps=6, k=5, seed=2, runtime_fn=rt, kt=kt)
    _check(out)
    sizes = [len(o[0]) for o in out]
    assert sizes[:5] == [5, 5, 5, 5, 3] and sum(sizes) == 23


def test_step_scores_within_fp64_bound(kt):
    d = W.load_space("batch_3")
    roles = W.layout(32)
    model = random_model(d.radices, roles, depth=8, seed=9)
    gpu, cnt, rt = _synthetic(d, roles, 4)
    sp = kt.Space.from_desc(d)
    m = kt.Model(sp, model)
    s = kt.Search(sp, m, k=16, seed=1)
    c = cnt(s.current())
    prof = otrees.predict(model, ospace.decode(d.radices, [s.current()]))[0]
    raw, sc = s.step(c)
    d64 = expert.delta_vector(roles, c)
    cand = otrees.predict(model, ospace.decode(d.radices, raw))
    ref = oscore.score_def(prof, cand, d64)
    bound = (len(roles) + 3) * 2.0 ** -24 * np.abs(d64).sum() + 1e-30
    assert np.all(np.abs(sc.astype(np.float64) - ref) <= bound)


def test_invalid_counters_rejected(kt):
    d = W.space_tiny_block_tile()
    sp = kt.Space.from_desc(d)
    m = kt.Model(sp, random_model(d.radices, W.layout(16), depth=3, seed=0))
    s = kt.Search(sp, m, k=5)
    c = np.ones(16, np.float32)
    c[3] = np.nan
    with pytest.raises(kt.KtuneError) as e:
        s.step(c)
    assert e.value.code == kt.KTUNE_EINVAL


def test_full_size_mid_space_steps(kt):
    """The mid space at full size (2.26M configurations, 32 counters, depth-12
    trees), in the launch configuration the benchmark times; every score of
    the oracle's float32 path is computed for the whole space each step."""
    d = W.load_space("mid_12p")
    roles = W.layout(32)
    model = random_model(d.radices, roles, depth=12, seed=12)
    gpu, cnt, rt = _synthetic(d, roles, 0)
    out = run_pair(d, model, cnt, steps=3, k=5, seed=0, runtime_fn=rt, kt=kt)
    _check(out)


def test_steps_wide_space_general_path(kt):
    """Eleven 5-valued parameters need 33 bits in the one-word layout, so this
    space takes the general (two-word) walk."""
    values = [[1, 2, 3, 4, 5]] * 11
    code = []
    for j in range(0, 10, 2):
        code += W.c_sum_le([j, j + 1], 3)
    d = W.SpaceDesc("wide", ["p%d" % j for j in range(11)], values, code)
    roles = W.layout(16)
    model = random_model(d.radices, roles, depth=9, seed=33)
    gpu, cnt, rt = _synthetic(d, roles, 5)
    out = run_pair(d, model, cnt, steps=4, k=5, seed=3, runtime_fn=rt, kt=kt)
    _check(out)


# ---- top-k select and on-the-fly spaces -------------------------------------------
@pytest.mark.parametrize("name,K,depth,k", [("tiny", 16, 8, 5), ("batch_2", 32, 10, 16),
                                            ("batch_7", 40, 12, 64)])
def test_steps_topk(kt, name, K, depth, k):
    d = W.space_tiny_block_tile() if name == "tiny" else W.load_space(name)
    roles = W.layout(K)
    model = random_model(d.radices, roles, depth=depth, seed=k)
    gpu, cnt, rt = _synthetic(d, roles, 6)
    out = run_pair(d, model, cnt, steps=6, k=k, seed=5, select="topk", runtime_fn=rt, kt=kt)
    _check(out)


# batch_6's constrained parameters have 270,336 value combinations, more than
# the constrained-index table holds: it exercises the window-table check
@pytest.mark.parametrize("name,select,k,fused", [("tiny", "sample", 5, None), ("batch_3", "sample", 7, None),
                                                 ("batch_5", "topk", 16, None), ("batch_0", "topk", 5, None),
                                                 ("batch_6", "sample", 6, None), ("batch_6", "topk", 9, None),
                                                 ("batch_6", "topk", 9, 0), ("tiny", "sample", 5, 0)])
def test_steps_on_the_fly(kt, name, select, k, fused):
    d = W.space_tiny_block_tile() if name == "tiny" else W.load_space(name)
    roles = W.layout(32)
    model = random_model(d.radices, roles, depth=11, seed=7)
    gpu, cnt, rt = _synthetic(d, roles, 7)
    out = run_pair(d, model, cnt, steps=5, k=k, seed=9, select=select, runtime_fn=rt, kt=kt,
                   flags=kt.KTUNE_ON_THE_FLY, fused=fused)
    _check(out)


@pytest.mark.parametrize("fused", [0, 2])
def test_on_the_fly_matches_materialised(kt, fused):
    d = W.load_space("batch_6")
    roles = W.layout(16)
    model = random_model(d.radices, roles, depth=9, seed=2)
    outs = []
    for flags in (kt.KTUNE_MATERIALISE, kt.KTUNE_ON_THE_FLY):
        sp = kt.Space.from_desc(d, flags=flags)
        m = kt.Model(sp, model)
        s = kt.Search(sp, m, k=8, seed=3)
        if flags == kt.KTUNE_ON_THE_FLY:
            s.set_fused(fused)
        gpu, cnt, rt = _synthetic(d, roles, 1)
        seq = []
        for _ in range(4):
            raw, sc = s.step(cnt(s.current()))
            seq.append((list(raw), list(sc)))
            s.report(rt(raw))
        outs.append(seq)
    assert outs[0] == outs[1]


def test_large_on_the_fly_top16_full_size(kt):
    """The large space at full size (113M raw, 19.5M valid, decoded every
    step), K=40 depth-12 trees, top-16.  The oracle checks each selected
    configuration's score exactly, validity, and that no configuration of a
    200k random sample of the space scores higher than the 16th pick."""
    d = W.load_space("large_16p")
    roles = W.layout(40)
    model = random_model(d.radices, roles, depth=12, seed=40)
    gpu, cnt, rt = _synthetic(d, roles, 0)
    sp = kt.Space.from_desc(d, flags=kt.KTUNE_ON_THE_FLY)
    assert sp.count() == (counts()["large_16p"]["n_valid"], d.n_raw)
    m = kt.Model(sp, model)
    s = kt.Search(sp, m, k=16, seed=0, select=kt.KTUNE_SELECT_TOPK)
    rng = np.random.default_rng(0)
    sample = np.unique(rng.integers(0, d.n_raw, size=600000))
    sample = sample[ospace.is_valid_raw(d, sample)][:200000]
    seen = {s.current()}
    for _ in range(2):
        cp = s.current()
        c = cnt(cp)
        raw, sc = s.step(c)
        assert len(raw) == 16 and len(set(raw)) == 16 and not (set(raw) & seen)
        assert ospace.is_valid_raw(d, raw).all()
        assert list(sc) == sorted(sc, reverse=True)
        d32 = expert.delta_vector(roles, c).astype(np.float32)
        prof = otrees.predict(model, ospace.decode(d.radices, [cp]))[0]
        ref = oscore.score_fp32(prof, otrees.predict(model, ospace.decode(d.radices, raw)), d32)
        np.testing.assert_array_equal(sc, ref)
        free = np.array([r not in seen and r not in set(raw) for r in sample])
        ss = oscore.score_fp32(prof, otrees.predict(model, ospace.decode(d.radices, sample[free])), d32)
        assert ss.max() <= sc[-1]
        seen |= set(int(r) for r in raw)
        s.report(rt(raw))


@pytest.mark.parametrize("select", ["sample", "topk"])
def test_graph_path_matches_plain_launches(kt, select):
    """With four kernels per step (ktune_search_set_fused(0)), steps on a
    non-default stream run as a captured CUDA graph whose step parameters are
    replaced each step; they must equal plain launches."""
    import torch
    d = W.load_space("batch_4")
    roles = W.layout(32)
    model = random_model(d.radices, roles, depth=10, seed=8)
    gpu, cnt, rt = _synthetic(d, roles, 2)
    sel = kt.KTUNE_SELECT_TOPK if select == "topk" else kt.KTUNE_SELECT_SAMPLE
    runs = []
    for stream in (None, torch.cuda.Stream()):
        sp = kt.Space.from_desc(d)
        m = kt.Model(sp, model)
        s = kt.Search(sp, m, k=6, seed=4, select=sel, stream=stream)
        s.set_fused(0)
        seq = []
        for i in range(6):
            if i == 3:
                s.set_timing(True)           # re-captures with event nodes
            raw, sc = s.step(cnt(s.current()))
            seq.append((list(raw), list(sc)))
            s.report(rt(raw))
        st = s.stats()
        assert st.n_kernels == 4 and st.kernel_ms[1] > 0
        runs.append(seq)
    assert runs[0] == runs[1]


@pytest.mark.parametrize("select", ["sample", "topk"])
def test_fused_step_matches_four_kernels(kt, select):
    """The whole step as one persistent kernel (every shape, default and
    non-default streams) against the four-kernel chain: the same selections
    and scores, step after step; one timed kernel per fused step."""
    import torch
    d = W.load_space("batch_4")
    roles = W.layout(40)
    model = random_model(d.radices, roles, depth=12, seed=18)
    gpu, cnt, rt = _synthetic(d, roles, 4)
    sel = kt.KTUNE_SELECT_TOPK if select == "topk" else kt.KTUNE_SELECT_SAMPLE
    runs = []
    for shape, stream in [(0, None), (1, None), (2, torch.cuda.Stream()), (3, None)]:
        sp = kt.Space.from_desc(d)
        m = kt.Model(sp, model)
        s = kt.Search(sp, m, k=9, seed=6, select=sel, stream=stream)
        s.set_fused(shape)
        s.set_timing(True)
        seq = []
        for _ in range(5):
            raw, sc = s.step(cnt(s.current()))
            seq.append((list(raw), list(sc)))
            s.report(rt(raw))
        st = s.stats()
        assert st.n_kernels == (4 if shape == 0 else 1) and st.kernel_ms[0] > 0
        runs.append(seq)
    for r in runs[1:]:
        assert r == runs[0]


def test_fused_step_refused_where_it_does_not_apply(kt):
    values = [[1, 2, 3, 4, 5]] * 11           # 33 bits: the two-word walk
    d = W.SpaceDesc("wide", ["p%d" % j for j in range(11)], values, [])
    sp = kt.Space.from_desc(d)
    s = kt.Search(sp, kt.Model(sp, random_model(d.radices, W.layout(16), depth=5, seed=1)), k=5)
    with pytest.raises(kt.KtuneError) as e:
        s.set_fused(1)
    assert e.value.code == kt.KTUNE_ESTATE
    s.set_fused(0)
    d2 = W.load_space("batch_2")
    sp2 = kt.Space.from_desc(d2)
    s2 = kt.Search(sp2, kt.Model(sp2, random_model(d2.radices, W.layout(16), depth=5, seed=1)), k=5)
    with pytest.raises(kt.KtuneError) as e:
        s2.set_fused(7)
    assert e.value.code == kt.KTUNE_EINVAL
    sp3 = kt.Space.from_desc(d2, flags=kt.KTUNE_ON_THE_FLY)
    s3 = kt.Search(sp3, kt.Model(sp3, random_model(d2.radices, W.layout(16), depth=5, seed=1)), k=5)
    for shape in (1, 3):
        with pytest.raises(kt.KtuneError) as e:
            s3.set_fused(shape)
        assert e.value.code == kt.KTUNE_ESTATE
    s3.set_fused(0)
    s3.set_fused(2)
