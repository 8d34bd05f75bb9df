"""The least-squares counter model (Section 3.3.1) on the GPU against the oracle.

The GPU evaluates each counter's polynomial in a float32 Horner form (u
rounded to float32; c_0 + sum_a u_a (g_a + h_aa u_a + sum_{b>a} h_ab u_b), one
fused multiply-add per coefficient), the oracle in float64: the Horner form's
rounding error is at most about (2m + 3) 2^-24 sum_t |c_t x_t|, and the test
allows (T + 8) 2^-23 sum_t |c_t x_t| (T = 1 + 2m + m(m-1)/2 >= 2m + 1).  Eq.
score and the selection are then checked bit for bit against the oracle's
float32 score on the GPU's own predictions (ktune_model_predict_device
evaluates the same Horner form as the fused step), and the cached steps
against the fused ones.  The spaces cover both fused kernels (sorted tiles
for at most 64 subspaces, unsorted beyond) and m from 1 to 11."""
import numpy as np
import pytest

import workloads as W
from workloads.synth import SyntheticGPU, add_noise, sample_indices
from oracle import expert, lsq as olsq, score as oscore, space as ospace

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def kt():
    import torch
    assert torch.cuda.is_available()
    from paper_2102_05297_gb300 import ktune
    return ktune


def load(name):
    """A space of the workloads, or "wide_11": 11 three-valued parameters and
    2 binary ones (m = 11 regressors, T = 78 terms)."""
    if name == "wide_11":
        return W.SpaceDesc("wide_11", ["p%d" % j for j in range(13)],
                           [[1, 2, 4]] * 6 + [[0, 1]] + [[2, 8, 32]] * 5 + [[1, 3]], [])
    return W.load_space(name)


def random_coef(values, K, seed, scale=1.0, offset=0.0):
    d = olsq.design(values)
    rng = np.random.default_rng(seed)
    c = rng.standard_normal((d["n_sub"], K, d["T"])) * scale
    c[:, :, 0] += offset
    return c.astype(np.float32)


def device_predict(model, n, K):
    import torch
    out = torch.empty((n, K), dtype=torch.float32, device="cuda")
    model.predict_device(0, n, out.data_ptr())
    torch.cuda.synchronize()
    return out.cpu().numpy()


def bound(values, coef, dig):
    d = olsq.design(values)
    X = olsq.terms(d, dig)
    C = coef.astype(np.float64)[olsq.subspace(d, dig)]
    return (d["T"] + 8) * 2.0 ** -23 * np.einsum("nkt,nt->nk", np.abs(C), np.abs(X)) + 1e-30


@pytest.mark.parametrize("name,K", [("batch_2", 8), ("batch_3", 12), ("batch_4", 16), ("wide_11", 6)])
def test_predict_matches_oracle(kt, name, K):
    d = load(name)
    roles = W.layout(40)[:K]
    coef = random_coef(d.values, K, seed=K)
    sp = kt.Space.from_desc(d)
    m = kt.Model(sp, {"kind": "lsq", "roles": roles, "coef": coef})
    assert (m.K, m.depth) == (K, 0)
    n = sp.count()[0]
    dig = sp.valid_digits()
    g = device_predict(m, n, K)
    o = olsq.predict(d.values, coef, dig)
    assert np.all(np.abs(g - o) <= bound(d.values, coef, dig))


def test_predict_subrange_and_edges(kt):
    import torch
    d = W.load_space("batch_3")
    roles = W.layout(40)[:5]
    coef = random_coef(d.values, 5, seed=1)
    sp = kt.Space.from_desc(d)
    m = kt.Model(sp, {"kind": "lsq", "roles": roles, "coef": coef})
    n = sp.count()[0]
    full = device_predict(m, n, 5)
    for first, count in [(0, 1), (n - 1, 1), (131, 1000), (7, 0)]:
        out = torch.zeros((max(count, 1), 5), dtype=torch.float32, device="cuda")
        m.predict_device(first, count, out.data_ptr())
        torch.cuda.synchronize()
        np.testing.assert_array_equal(out.cpu().numpy()[:count], full[first:first + count])
    with pytest.raises(kt.KtuneError):
        m.predict_device(n - 1, 2, out.data_ptr())


def drive(s, gpu, radices, steps):
    out = []
    for _ in range(steps):
        c = gpu.evaluate(ospace.decode(radices, [s.current()]))[0][0]
        raw, sc = s.step(c)
        out.append((list(raw), [float(x) for x in sc]))
        s.report(gpu.evaluate(ospace.decode(radices, raw))[1])
    return out


@pytest.mark.parametrize("name,K,seed", [("batch_3", 16, 0), ("batch_4", 24, 1), ("batch_2", 12, 2),
                                         ("mid_12p", 32, 3), ("wide_11", 12, 4)])
def test_search_scores_bit_exact(kt, name, K, seed):
    d = load(name)
    roles = W.layout(40)[:K]
    gpu = SyntheticGPU(d, roles, seed=seed)
    coef = random_coef(d.values, K, seed=seed + 7, scale=0.2, offset=3.0)
    sp = kt.Space.from_desc(d)
    m = kt.Model(sp, {"kind": "lsq", "roles": roles, "coef": coef})
    valid = sp.valid_raw()
    pos = {int(r): i for i, r in enumerate(valid)}
    pred = device_predict(m, len(valid), K)
    s = kt.Search(sp, m, k=7, seed=seed)
    s.set_timing(True)
    free = np.ones(len(valid), bool)
    for step in range(4):
        cp = pos[s.current()]
        free[cp] = False
        c = gpu.evaluate(ospace.decode(d.radices, [s.current()]))[0][0]
        d32 = expert.delta_vector(roles, c, 0.7, 1000.0).astype(np.float32)
        o_s = oscore.score_fp32(pred[cp], pred, d32)
        raw, sc = s.step(c)
        idx = [pos[int(r)] for r in raw]
        assert len(set(idx)) == 7 and all(free[idx])
        assert np.array_equal(np.asarray(sc, np.float32), o_s[idx])
        st = s.stats()
        assert st.s_min == o_s[free].min() and st.s_max == o_s[free].max()
        assert st.n_active == int(np.count_nonzero((d32 != 0) & (pred[cp] != 0)))
        free[idx] = False
        s.report(gpu.evaluate(ospace.decode(d.radices, raw))[1])


@pytest.mark.parametrize("name", ["batch_4", "wide_11"])
def test_cached_and_graph_steps_equal_fused(kt, name):
    import torch
    d = load(name)
    roles = W.layout(40)[:20]
    gpu = SyntheticGPU(d, roles, seed=3)
    coef = random_coef(d.values, 20, seed=5, scale=0.3, offset=2.0)
    sp = kt.Space.from_desc(d)
    m = kt.Model(sp, {"kind": "lsq", "roles": roles, "coef": coef})
    a = kt.Search(sp, m, k=6, seed=9)
    b = kt.Search(sp, m, k=6, seed=9)
    c = kt.Search(sp, m, k=6, seed=9, stream=torch.cuda.Stream())
    b.set_cached(True)
    ta = drive(a, gpu, d.radices, 6)
    assert ta == drive(b, gpu, d.radices, 6)
    assert ta == drive(c, gpu, d.radices, 6)


def test_fitted_model_search_reaches_target(kt):
    """A model fitted by the package's least-squares fitter on a 2 % sample of
    noisy synthetic counters drives a search that reaches a configuration
    within 10 % of the optimum in fewer tests than uniform random draws."""
    from paper_2102_05297_gb300.fit import fit_lsq
    d = W.load_space("batch_3")
    roles = W.layout(16)
    gpu = SyntheticGPU(d, roles, seed=4)
    sp = kt.Space.from_desc(d)
    valid = sp.valid_raw()
    dig = ospace.decode(d.radices, valid)
    C, rt = gpu.evaluate(dig)
    sample = sample_indices(len(valid), 0.02, seed=4)
    model = fit_lsq(d.values, dig[sample], add_noise(C[sample], seed=4), roles)
    m = kt.Model(sp, model)
    target = rt.min() * 1.1
    tests = []
    for seed in range(8):
        s = kt.Search(sp, m, k=5, seed=seed)
        n = 1
        best = rt[np.searchsorted(valid, s.current())]
        while best > target and n < 600:
            c = C[np.searchsorted(valid, s.current())]
            raw, _ = s.step(c)
            r = rt[np.searchsorted(valid, raw)]
            s.report(r)
            n += len(raw)
            best = min(best, r.min())
        tests.append(n)
    good = np.count_nonzero(rt <= target)
    random_expect = (len(valid) + 1) / (good + 1)
    assert np.median(tests) < random_expect, (tests, random_expect)


def test_model_rules(kt):
    d = W.load_space("batch_3")
    roles = W.layout(40)[:6]
    coef = random_coef(d.values, 6, seed=0)
    sp = kt.Space.from_desc(d)
    m = kt.Model(sp, {"kind": "lsq", "roles": roles, "coef": coef})
    with pytest.raises(kt.KtuneError):
        kt.Search(sp, m, k=5, select=kt.KTUNE_SELECT_TOPK)
    s = kt.Search(sp, m, k=5)
    with pytest.raises(kt.KtuneError):
        kt.Batch([s])
    otf = kt.Space.from_desc(d, flags=kt.KTUNE_ON_THE_FLY)
    with pytest.raises(kt.KtuneError):
        kt.Search(otf, kt.Model(otf, {"kind": "lsq", "roles": roles, "coef": coef}), k=5)
    for bad in (coef[:, :, :-1], coef[:-1], np.where(np.arange(coef.size).reshape(coef.shape) == 5,
                                                     np.nan, coef)):
        with pytest.raises(kt.KtuneError):
            kt.Model(sp, {"kind": "lsq", "roles": roles, "coef": bad})
    neg = W.SpaceDesc("neg", ["a", "b"], [[-3, 1, 2], [0, 1]], [])
    sn = kt.Space.from_desc(neg)
    with pytest.raises(kt.KtuneError):
        kt.Model(sn, {"kind": "lsq", "roles": roles[:2], "coef": np.zeros((2, 2, 3), np.float32)})
