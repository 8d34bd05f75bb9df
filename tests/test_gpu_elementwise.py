"""Element-wise parity of whole steps against the CPU oracle, through the C ABI.

After each GPU step every score and every integer weight of the step is read
back (ktune_search_scores_device) and compared with the oracle, not only the
k selected configurations:

  * scores (Section 3.5 Eq. score) of every configuration not evaluated before
    the step, bit for bit against the oracle's float32 score;
  * integer weights (Eq. score_normalization, w = round-half-even(s_norm 2^20)),
    bit for bit against the oracle's quantised weights over the same set, with
    the drawn configurations at 0 (Algorithm 1 draws without replacement);
  * s_min / s_max of the step exactly;
  * the selections exactly.

Paths: fused tree steps on the full mid space (2.26M configurations, the
benchmark's launch configuration), the tiny space with fitted trees, top-k,
on-the-fly decode, the general two-word walk, the graph-launched step, cached
predictions (trees, MLP, least squares), the MLP at full size (the persistent
kernel handles about 116 tiles of 128 rows per CTA) and a mixed batch of tree
and MLP searches.  For the MLP and least-squares models the oracle scores the
GPU's own predictions (those models are compared with the oracle's network /
polynomials within their rounding bounds: the MLP here at full size on
sampled tiles, least squares in test_gpu_lsq.py)."""
import numpy as np
import pytest

import workloads as W
from workloads.synth import SyntheticGPU, sample_indices
from workloads.trees import random_model
from oracle import mlp as omlp, search as osearch, select as oselect, space as ospace
from oracle import trees as otrees

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def kt():
    import torch
    assert torch.cuda.is_available()
    from paper_2102_05297_gb300 import ktune
    return ktune


def readback(kt, s, n, weights=True, stream=None):
    import torch
    S = torch.empty(max(n, 1), dtype=torch.float32, device="cuda")
    Wt = torch.empty(max(n, 1), dtype=torch.int32, device="cuda") if weights else None
    s.scores_device(0, n, S.data_ptr(), Wt.data_ptr() if weights else 0, stream=stream)
    torch.cuda.synchronize()
    return S.cpu().numpy()[:n], (Wt.cpu().numpy()[:n].view(np.uint32) if weights else None)


def oracle_weights(s_o, free, picks, gamma):
    """The oracle's integer weights of a step: normalised over the
    configurations not evaluated before it, drawn ones zeroed."""
    w = np.zeros(len(s_o), np.uint64)
    if free.any():
        sf = s_o[free]
        w[free] = oselect.quantise(oselect.normalise_fp32(sf, sf.min(), sf.max(), gamma))
    w[list(picks)] = 0
    return w


def step_and_compare(kt, s, o, c, weights=True, zero_evaluated=True, stream=None):
    """One step of GPU search s and oracle search o on counters c, then the
    whole score and weight vectors compared.  Returns the selected raw indices."""
    free = ~o.evaluated.copy()
    s_o, _ = o.scores(c)
    g_raw, g_sc = s.step(c)
    o_raw, o_sc = o.step(c)
    assert list(g_raw) == o_raw
    np.testing.assert_array_equal(np.asarray(g_sc, np.float32), np.float32(o_sc))
    n = len(s_o)
    S, Wt = readback(kt, s, n, weights, stream)
    bad = np.nonzero(S[free].view(np.uint32) != s_o[free].view(np.uint32))[0]
    assert len(bad) == 0, ("scores differ", len(bad), np.nonzero(free)[0][bad[:5]])
    if zero_evaluated:
        assert not np.any(S[~free])
    if weights:
        ref = oracle_weights(s_o, free, o.last, o.gamma)
        badw = np.nonzero(Wt.astype(np.uint64) != ref)[0]
        assert len(badw) == 0, ("weights differ", len(badw), badw[:5])
    if free.any():
        st = s.stats()
        assert st.s_min == s_o[free].min() and st.s_max == s_o[free].max()
    return g_raw


def synthetic(desc, roles, seed):
    gpu = SyntheticGPU(desc, roles, seed=seed)
    cnt = lambda raw: gpu.evaluate(ospace.decode(desc.radices, [raw]))[0][0]
    rt = lambda raws: gpu.evaluate(ospace.decode(desc.radices, raws))[1]
    return gpu, cnt, rt


def run(kt, desc, model, steps, k=5, seed=0, select="sample", flags=0, fseed=0, cached=False,
        stream=None, valid=None, pred=None, zero_evaluated=True, gpu_model=None, space=None,
        fused=None):
    sel = kt.KTUNE_SELECT_TOPK if select == "topk" else kt.KTUNE_SELECT_SAMPLE
    sp = space or kt.Space.from_desc(desc, flags=flags)
    m = gpu_model or kt.Model(sp, model)
    s = kt.Search(sp, m, k=k, seed=seed, select=sel, stream=stream)
    if fused is not None:
        s.set_fused(fused)
    if cached:
        s.set_cached(True)
    o = osearch.OracleSearch(desc, model, k=k, seed=seed, mode=select, valid=valid, pred=pred)
    assert s.current() == o.cprof_raw
    roles = model["roles"]
    gpu, cnt, rt = synthetic(desc, roles, fseed)
    for _ in range(steps):
        raw = step_and_compare(kt, s, o, cnt(s.current()), weights=select == "sample",
                               zero_evaluated=zero_evaluated, stream=stream)
        if len(raw) == 0:
            break
        r = rt(raw)
        s.report(r)
        o.report(list(r))
    return s, o


# ---- whole-space tree steps ----------------------------------------------------------
@pytest.fixture(scope="module")
def mid_trees():
    d = W.load_space("mid_12p")
    roles = W.layout(32)
    model = random_model(d.radices, roles, depth=12, seed=12)
    valid = ospace.enumerate_valid(d)
    pred = otrees.predict(model, ospace.decode(d.radices, valid))
    return d, model, valid, pred


@pytest.mark.parametrize("fused", [1, 0, 2, 3])
def test_every_score_and_weight_full_mid_space(kt, mid_trees, fused):
    """The headline workload: 2.26M configurations, 32 counters, depth-12
    trees (two groups of active trees in shared memory), k = 5, three steps;
    the whole step as one persistent kernel (each shape) and as four kernels."""
    d, model, valid, pred = mid_trees
    run(kt, d, model, steps=3, valid=valid, pred=pred, fused=fused)


@pytest.mark.parametrize("fused", [0, 1])
def test_every_score_and_weight_stream_path(kt, fused):
    """On a non-default stream: a captured graph of four kernels, or the
    fused kernel launched directly."""
    import torch
    d = W.load_space("batch_4")
    roles = W.layout(40)
    model = random_model(d.radices, roles, depth=12, seed=41)
    run(kt, d, model, steps=4, k=7, seed=2, stream=torch.cuda.Stream(), fseed=3, fused=fused)


@pytest.fixture(scope="module")
def flat_trees():
    values = [list(range(8))] * 6 + [list(range(5)), list(range(4))]
    d = W.SpaceDesc("flat_8p", ["p%d" % j for j in range(8)], values, [])
    model = random_model(d.radices, W.layout(16), depth=8, seed=51)
    valid = ospace.enumerate_valid(d)
    pred = otrees.predict(model, ospace.decode(d.radices, valid))
    return d, model, valid, pred


@pytest.mark.parametrize("fused", [2, 0])
def test_every_score_and_weight_beyond_shared_tile_sums(kt, flat_trees, fused):
    """5.24M configurations (no constraints): more sub-tiles than the fused
    step's draws keep in shared memory, so their super-tile sums are added up
    while the weights are computed and the draws read sub-tile sums from
    global memory."""
    d, model, valid, pred = flat_trees
    assert d.n_raw == 5242880 and d.n_raw // 1024 > 4096
    run(kt, d, model, steps=3, k=9, seed=4, fseed=2, fused=fused, valid=valid, pred=pred)


def test_every_score_and_weight_tiny_fitted(kt):
    d = W.space_tiny_block_tile()
    roles = W.layout(16)
    gpu = SyntheticGPU(d, roles, seed=1)
    valid = ospace.enumerate_valid(d)
    dig = ospace.decode(d.radices, valid)
    samp = sample_indices(len(valid), 0.10, 1)
    model = otrees.fit_model(dig[samp], gpu.evaluate(dig[samp])[0], 8, d.radices, roles)
    run(kt, d, model, steps=40, seed=1, valid=valid, fseed=1)


@pytest.mark.parametrize("name,K,depth,k,fused", [("batch_2", 32, 10, 16, None),
                                                   ("batch_7", 40, 12, 64, None),
                                                   ("batch_7", 40, 12, 64, 0),
                                                   ("mid_12p", 32, 12, 16, 2)])
def test_every_score_topk(kt, name, K, depth, k, fused):
    d = W.load_space(name)
    roles = W.layout(K)
    model = random_model(d.radices, roles, depth=depth, seed=k + 1)
    run(kt, d, model, steps=3, k=k, seed=5, select="topk", fseed=6, fused=fused)


def test_every_score_and_weight_general_walk(kt):
    values = [[1, 2, 3, 4, 5]] * 11
    code = []
    for j in range(0, 10, 2):
        code += W.c_sum_le([j, j + 1], 3)
    d = W.SpaceDesc("wide", ["p%d" % j for j in range(11)], values, code)
    roles = W.layout(32)
    model = random_model(d.radices, roles, depth=9, seed=34)
    run(kt, d, model, steps=4, seed=3, fseed=5)


@pytest.mark.parametrize("name,select,k,fused", [("batch_3", "sample", 7, 0), ("batch_6", "sample", 6, 0),
                                                 ("batch_5", "topk", 16, 0), ("batch_3", "sample", 7, 2),
                                                 ("batch_6", "sample", 6, 2), ("batch_5", "topk", 16, 2),
                                                 ("batch_0", "topk", 5, 2)])
def test_every_score_on_the_fly(kt, name, select, k, fused):
    """On-the-fly spaces score by ordinal without storing TS (the four-kernel
    chain writes no score for configurations evaluated before the step; the
    fused step decodes TS into a per-step list and writes 0 for them)."""
    d = W.load_space(name)
    roles = W.layout(32)
    model = random_model(d.radices, roles, depth=11, seed=7)
    run(kt, d, model, steps=4, k=k, seed=9, select=select, flags=kt.KTUNE_ON_THE_FLY, fseed=7,
        zero_evaluated=bool(fused), fused=fused)


@pytest.mark.parametrize("fused", [2, 0])
def test_every_score_on_the_fly_window_tables(kt, fused):
    """An on-the-fly space whose constrained parameters have too many value
    combinations for one table bit each (validity by window tables and the
    general check) and whose fastest radices are not powers of two (an
    odometer step per raw index): 1.87M raw configurations."""
    values = [list(range(1, r + 1)) for r in (3, 5, 7, 9, 10, 11, 6, 3)]
    code = W.c_sum_le([0, 1, 2, 3], 16) + W.c_sum_le([4, 5, 6, 7], 22) + W.c_product_le([1, 5], 40)
    d = W.SpaceDesc("windows_8p", ["p%d" % j for j in range(8)], values, code)
    assert d.n_raw == 1871100
    roles = W.layout(16)
    model = random_model(d.radices, roles, depth=10, seed=61)
    run(kt, d, model, steps=3, k=6, seed=3, flags=kt.KTUNE_ON_THE_FLY, fseed=4,
        zero_evaluated=bool(fused), fused=fused)


def test_readback_rules(kt):
    import torch
    d = W.load_space("batch_2")
    roles = W.layout(16)
    model = random_model(d.radices, roles, depth=6, seed=1)
    sp = kt.Space.from_desc(d)
    m = kt.Model(sp, model)
    n = sp.count()[0]
    buf = torch.empty(n + 1, dtype=torch.float32, device="cuda")
    s = kt.Search(sp, m, k=5, select=kt.KTUNE_SELECT_TOPK)
    with pytest.raises(kt.KtuneError) as e:
        s.scores_device(0, n, 0, buf.data_ptr())             # top-k: no weights
    assert e.value.code == kt.KTUNE_ESTATE
    with pytest.raises(kt.KtuneError) as e:
        s.scores_device(1, n, buf.data_ptr())                # beyond TS
    assert e.value.code == kt.KTUNE_EINVAL
    with pytest.raises(kt.KtuneError):
        s.scores_device(0, n)                                # nothing to write
    s.scores_device(n, 0, buf.data_ptr())                    # empty range
    s2 = kt.Search(sp, m, k=5)
    s2.set_neighbourhood(1)
    with pytest.raises(kt.KtuneError) as e:
        s2.scores_device(0, n, buf.data_ptr())
    assert e.value.code == kt.KTUNE_ESTATE


# ---- cached predictions ----------------------------------------------------------------
def test_cached_trees_full_mid_space_against_oracle(kt, mid_trees):
    d, model, valid, pred = mid_trees
    run(kt, d, model, steps=3, valid=valid, pred=pred, cached=True, fseed=2)


def device_predictions(kt, predict_device, n, K):
    import torch
    out = torch.empty((n, K), dtype=torch.float32, device="cuda")
    predict_device(0, n, out.data_ptr())
    torch.cuda.synchronize()
    return out.cpu().numpy()


def test_cached_least_squares_against_oracle(kt):
    from test_gpu_lsq import random_coef
    d = W.load_space("mid_12p")
    roles = W.layout(40)[:24]
    coef = random_coef(d.values, 24, seed=5, scale=0.3, offset=2.5)
    sp = kt.Space.from_desc(d)
    m = kt.Model(sp, {"kind": "lsq", "roles": roles, "coef": coef})
    n = sp.count()[0]
    pred = device_predictions(kt, m.predict_device, n, 24)
    valid = sp.valid_raw()
    for cached in (False, True):
        run(kt, d, {"roles": roles}, steps=3, seed=4, valid=valid, pred=pred, cached=cached,
            gpu_model=m, space=sp, fseed=4)


# ---- the MLP at full size -----------------------------------------------------------------
def positive_network(F, K, seed):
    p = omlp.init_params(F, K, seed=seed)
    rng = np.random.default_rng(seed + 100)
    for k in ("b1", "b2", "b3"):
        p[k] = (rng.standard_normal(p[k].shape) * 0.1).astype(np.float32)
    # keep predicted counters well above 0 so that Eq. score stays bounded
    p["W4"] = (p["W4"] * 0.1).astype(np.float32)
    p["b4"] = (np.abs(rng.standard_normal(K)) * 0.1 + 1.0).astype(np.float32)
    return p


@pytest.fixture(scope="module")
def mid_mlp(kt):
    d = W.load_space("mid_12p")
    roles = W.layout(32)
    gpu = SyntheticGPU(d, roles, seed=0)
    ranges = gpu.counter_ranges()
    sp = kt.Space.from_desc(d)
    mlp = kt.Mlp(sp, roles, ranges, max_batch=64)
    p = positive_network(mlp.F, len(roles), 5)
    mlp.set_params(p)
    n = sp.count()[0]
    pred = device_predictions(kt, mlp.predict_device, n, len(roles))
    return d, roles, ranges, sp, mlp, p, pred


def test_mlp_full_size_predictions_against_oracle(kt, mid_mlp):
    """Predictions of every 128-row tile of the full mid space come from the
    persistent tensor-core kernel (about 116 tiles per CTA, both ping-pong
    slots, every ring phase); the oracle network (float64 accumulation,
    bfloat16 activations) is evaluated on 400 random whole tiles plus the
    first and the ragged last tile."""
    d, roles, ranges, sp, mlp, p, pred = mid_mlp
    n = len(pred)
    n_tiles = (n + 127) // 128
    rng = np.random.default_rng(0)
    tiles = np.unique(np.concatenate([[0, n_tiles - 1], rng.choice(n_tiles, 400, replace=False)]))
    rows = np.concatenate([np.arange(t * 128, min(n, t * 128 + 128)) for t in tiles])
    dig = sp.valid_digits()[rows].astype(np.int64)
    ref = omlp.predict(p, d.values, dig, ranges)
    got = pred[rows]
    scale = np.max(np.abs(ref), axis=0) + 1e-6
    err = np.max(np.abs(got - ref), axis=0) / scale
    assert np.all(err <= 5e-3), err
    rms = np.sqrt(np.mean((got - ref) ** 2, axis=0)) / scale
    assert np.all(rms <= 1e-3), rms
    # mlp.predict (host staging, one grid per call) gives the same bits
    np.testing.assert_array_equal(mlp.predict(sp.valid_raw()[rows[:1000]]), got[:1000])


@pytest.mark.parametrize("cached", [False, True])
def test_mlp_full_size_scores_against_oracle(kt, mid_mlp, cached):
    """Fused MLP scoring of all 2.26M configurations (and the cached form):
    every score equals the oracle's float32 Eq. score of the GPU's
    predictions, every weight and every draw equals the oracle's."""
    d, roles, ranges, sp, mlp, p, pred = mid_mlp
    model = kt.Model.from_mlp(mlp)
    run(kt, d, {"roles": roles}, steps=3, seed=6, valid=sp.valid_raw(), pred=pred, cached=cached,
        gpu_model=model, space=sp, zero_evaluated=cached, fseed=0)


# ---- a mixed batch ------------------------------------------------------------------------
def test_mixed_batch_against_oracle(kt):
    """Tree and MLP searches over three spaces in one batched step (one graph
    launch; the three MLP searches of a space share one scoring pass): each
    member's selections, scores and whole weight vector against its own
    oracle search."""
    import torch
    from paper_2102_05297_gb300 import fit
    stream = torch.cuda.Stream()
    members, keep = [], []
    for si, name in enumerate(["batch_2", "batch_3", "batch_6"]):
        d = W.load_space(name)
        K = [16, 32, 40][si]
        roles = W.layout(K)
        gpu = SyntheticGPU(d, roles, seed=si)
        sp = kt.Space.from_desc(d)
        tree = random_model(d.radices, roles, depth=10, seed=200 + si)
        tm = kt.Model(sp, tree)
        mlp = kt.Mlp(sp, roles, gpu.counter_ranges(), max_batch=64)
        p = fit.init_mlp(mlp.F, K, seed=si)
        p["b4"] = np.full(K, 0.5, np.float32)
        mlp.set_params(p)
        mm = kt.Model.from_mlp(mlp)
        valid = sp.valid_raw()
        pred = device_predictions(kt, mlp.predict_device, len(valid), K)
        keep += [sp, tm, mlp, mm]
        for r, kind in enumerate(("tree", "mlp", "mlp", "tree", "mlp")):
            seed = 30 + 10 * si + r
            s = kt.Search(sp, tm if kind == "tree" else mm, k=5, seed=seed, search_id=r,
                          stream=stream)
            o = osearch.OracleSearch(d, tree if kind == "tree" else {"roles": roles}, k=5,
                                     seed=seed, search_id=r, valid=valid,
                                     pred=None if kind == "tree" else pred)
            assert s.current() == o.cprof_raw
            members.append((d, gpu, s, o))
    b = kt.Batch([m[2] for m in members], stream=stream)
    for step in range(3):
        cs = [gpu.evaluate(ospace.decode(d.radices, [s.current()]))[0][0]
              for d, gpu, s, o in members]
        frees = [~m[3].evaluated.copy() for m in members]
        s_os = [m[3].scores(c)[0] for m, c in zip(members, cs)]
        res = b.step(cs, 5)
        for (d, gpu, s, o), c, free, s_o, (g_raw, g_sc) in zip(members, cs, frees, s_os, res):
            o_raw, o_sc = o.step(c)
            assert list(g_raw) == o_raw, step
            np.testing.assert_array_equal(np.asarray(g_sc, np.float32), np.float32(o_sc))
            S, Wt = readback(kt, s, len(s_o), True, stream)
            np.testing.assert_array_equal(S[free].view(np.uint32), s_o[free].view(np.uint32))
            np.testing.assert_array_equal(Wt.astype(np.uint64),
                                          oracle_weights(s_o, free, o.last, o.gamma))
            r = gpu.evaluate(ospace.decode(d.radices, g_raw))[1]
            s.report(r)
            o.report(list(r))
    b.close()
