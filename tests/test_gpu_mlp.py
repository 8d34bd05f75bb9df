"""The MLP counter model on the tensor cores against the oracle MLP.

The GPU accumulates bfloat16 products in float32 on the tensor cores in its
own order, the oracle in float64 and rounds once, so parity is within a
tolerance: GEMMs within K 2^-22 of sum |a b| per element (float32 accumulation
of K products), predictions, loss and gradients within the bounds written in
each test (they allow rare one-ulp bfloat16 flips of intermediate
activations where the two accumulation orders straddle a rounding boundary)."""
import numpy as np
import pytest

import workloads as W
from workloads.synth import SyntheticGPU, add_noise
from oracle import mlp as omlp, space as ospace

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def kt():
    import torch
    assert torch.cuda.is_available()
    from paper_2102_05297_gb300 import ktune
    return ktune


def bf16_tensor(torch, a):
    return torch.from_numpy(omlp.bf16(a)).to(torch.bfloat16).cuda().contiguous()


@pytest.mark.parametrize("M,N,Kd", [(128, 256, 64), (200, 48, 80), (300, 400, 128), (1, 16, 16),
                                    (513, 272, 208), (64, 256, 4096)])
def test_gemm_matches_float64(kt, M, N, Kd):
    import torch
    rng = np.random.default_rng(M * 7 + N + Kd)
    a = omlp.bf16(rng.standard_normal((M, Kd)).astype(np.float32))
    b = omlp.bf16(rng.standard_normal((N, Kd)).astype(np.float32))
    ta, tb = bf16_tensor(torch, a), bf16_tensor(torch, b)
    tc = torch.full((M, N), float("nan"), dtype=torch.float32, device="cuda")
    kt.gemm_bf16(ta.data_ptr(), Kd, tb.data_ptr(), Kd, tc.data_ptr(), N, M, N, Kd)
    got = tc.cpu().numpy()
    ref = a.astype(np.float64) @ b.astype(np.float64).T
    bound = Kd * 2.0 ** -22 * (np.abs(a).astype(np.float64) @ np.abs(b).astype(np.float64).T)
    assert np.all(np.abs(got - ref) <= bound + 1e-30)


def test_gemm_rejects_bad_shapes(kt):
    with pytest.raises(kt.KtuneError):
        kt.gemm_bf16(16, 24, 16, 24, 16, 16, 16, 16, 24)   # Kd not a multiple of 16
    with pytest.raises(kt.KtuneError):
        kt.gemm_bf16(16, 12, 16, 16, 16, 16, 16, 16, 16)   # lda not a multiple of 8


def tiny_setup(K=16, seed=0):
    desc = W.space_tiny_block_tile()
    roles = W.layout(K)
    gpu = SyntheticGPU(desc, roles, seed=seed)
    valid = ospace.enumerate_valid(desc)
    dig = ospace.decode(desc.radices, valid)
    C, _ = gpu.evaluate(dig)
    return desc, roles, gpu, valid, dig, C


def random_params(F, K, seed):
    p = omlp.init_params(F, K, seed=seed)
    rng = np.random.default_rng(seed + 100)
    for k in ("b1", "b2", "b3", "b4"):
        p[k] = (rng.standard_normal(p[k].shape) * 0.1).astype(np.float32)
    return p


def test_features_width_matches_oracle(kt):
    desc, roles, gpu, valid, dig, C = tiny_setup()
    sp = kt.Space.from_desc(desc)
    m = kt.Mlp(sp, roles, gpu.counter_ranges(), max_batch=256)
    assert m.F == omlp.n_features(desc.radices)
    assert m.n_params == sum(int(np.prod(s)) for s in m.shapes().values())


@pytest.mark.parametrize("seed", [0, 1])
def test_predict_matches_oracle(kt, seed):
    desc, roles, gpu, valid, dig, C = tiny_setup(seed=seed)
    ranges = gpu.counter_ranges()
    sp = kt.Space.from_desc(desc)
    m = kt.Mlp(sp, roles, ranges, max_batch=256)
    p = random_params(m.F, len(roles), seed)
    m.set_params(p)
    back = m.get_params()
    for k in p:
        np.testing.assert_array_equal(back[k], p[k])
    rng = np.random.default_rng(seed)
    pick = np.sort(rng.choice(len(valid), size=300, replace=False))   # 3 tiles, ragged tail
    got = m.predict(valid[pick])
    ref = omlp.predict(p, desc.values, dig[pick], ranges)
    # a one-ulp bfloat16 flip of an activation moves it by 2^-8 relative; a few
    # per row bound the worst element near 5e-3 of the counter's scale
    scale = np.max(np.abs(ref), axis=0) + 1e-6
    err = np.max(np.abs(got - ref), axis=0) / scale
    assert np.all(err <= 5e-3), err
    rms = np.sqrt(np.mean((got - ref) ** 2, axis=0)) / scale
    assert np.all(rms <= 1e-3), rms


def test_predict_device_matches_predict(kt):
    import torch
    desc, roles, gpu, valid, dig, C = tiny_setup()
    sp = kt.Space.from_desc(desc)
    m = kt.Mlp(sp, roles, gpu.counter_ranges(), max_batch=256)
    m.set_params(random_params(m.F, len(roles), 3))
    n = len(valid)
    out = torch.empty((n, len(roles)), dtype=torch.float32, device="cuda")
    m.predict_device(0, n, out.data_ptr())
    torch.cuda.synchronize()
    np.testing.assert_array_equal(out.cpu().numpy(), m.predict(valid))


@pytest.mark.parametrize("B", [64, 272])
def test_grads_match_oracle(kt, B):
    desc, roles, gpu, valid, dig, C = tiny_setup()
    ranges = gpu.counter_ranges()
    sp = kt.Space.from_desc(desc)
    m = kt.Mlp(sp, roles, ranges, max_batch=512)
    p = random_params(m.F, len(roles), 7)
    m.set_params(p)
    rng = np.random.default_rng(B)
    rows = rng.choice(len(valid), size=600, replace=False)
    Cn = add_noise(C[rows], seed=1)
    m.set_data(valid[rows], Cn)
    idx = rng.choice(600, size=B, replace=False).astype(np.int32)
    loss, g = m.grads(idx)
    x = omlp.features(desc.values, dig[rows[idx]])
    t = (Cn[idx] / ranges).astype(np.float32)
    oloss, og = omlp.loss_and_grads(p, x, t)
    assert abs(loss - oloss) <= 1e-3 * oloss
    for k in og:
        scale = float(np.max(np.abs(og[k]))) + 1e-12
        err = float(np.max(np.abs(g[k] - og[k]))) / scale
        assert err <= 2e-2, (k, err)
        # the bulk agrees much more tightly than the worst element
        rel = np.linalg.norm(g[k] - og[k]) / (np.linalg.norm(og[k]) + 1e-12)
        assert rel <= 5e-3, (k, rel)


def test_training_tracks_oracle_and_fits(kt):
    desc, roles, gpu, valid, dig, C = tiny_setup()
    ranges = gpu.counter_ranges()
    sp = kt.Space.from_desc(desc)
    m = kt.Mlp(sp, roles, ranges, max_batch=256)
    p = omlp.init_params(m.F, len(roles), seed=0)
    m.set_params(p)
    m.set_data(valid, C)
    rng = np.random.default_rng(0)
    steps, B = 150, 256
    idx = np.concatenate([rng.choice(len(valid), size=B, replace=False) for _ in range(steps)])
    losses = m.train(idx.astype(np.int32), B)
    assert len(losses) == steps and np.all(np.isfinite(losses))
    # the oracle trained on the same batches
    x = omlp.features(desc.values, dig)
    t = (C / ranges).astype(np.float32)
    op = {k: v.copy() for k, v in p.items()}
    opt = omlp.Adam(op)
    olosses = []
    for s in range(steps):
        b = idx[s * B:(s + 1) * B]
        l, g = omlp.loss_and_grads(op, x[b], t[b])
        olosses.append(l)
        opt.step(op, g)
    olosses = np.array(olosses)
    assert abs(losses[0] - olosses[0]) <= 1e-3 * olosses[0]
    assert np.all(np.abs(losses - olosses) <= 0.1 * olosses + 1e-4), (losses[-5:], olosses[-5:])
    base = float(np.mean((t - t.mean(axis=0)) ** 2))
    final = m.predict(valid) / ranges
    assert float(np.mean((final - t) ** 2)) < 0.5 * base


def test_mlp_bad_arguments(kt):
    desc, roles, gpu, valid, dig, C = tiny_setup()
    sp = kt.Space.from_desc(desc)
    with pytest.raises(kt.KtuneError):
        kt.Mlp(sp, roles, np.zeros(len(roles)))                  # ranges must be > 0
    with pytest.raises(kt.KtuneError):
        kt.Mlp(sp, roles, gpu.counter_ranges(), max_batch=100)   # not a multiple of 16
    m = kt.Mlp(sp, roles, gpu.counter_ranges(), max_batch=64)
    with pytest.raises(kt.KtuneError):
        m.grads(np.zeros(16, np.int32))                          # no training set yet
    m.set_data(valid[:32], C[:32])
    with pytest.raises(kt.KtuneError):
        m.grads(np.zeros(80, np.int32))                          # beyond max_batch
    with pytest.raises(kt.KtuneError):
        m.grads(np.full(16, 32, np.int32))                       # row out of range
    bad = np.array([1], np.int64)
    if not np.isin(1, valid):
        with pytest.raises(kt.KtuneError):
            m.set_data(bad, C[:1])                               # invalid configuration


# ---- searches scored by the MLP ------------------------------------------------------
def exact_params(desc, F, K, seed):
    """A network whose every intermediate value is exact in float32 and bfloat16
    on both sides: integer one-hot weights and a bias of 16 keep every
    pre-activation in [16, 64], where GELU(z) = z exactly (erf rounds to 1 in
    float32 and float64); identity middle layers; output weights in 1/64 steps.
    Predictions, scores and therefore the draws must then match bit for bit."""
    rng = np.random.default_rng(seed)
    H = omlp.HIDDEN
    n_onehot = sum(desc.radices)
    W1 = np.zeros((H, F), np.float32)
    W1[:, :n_onehot] = rng.integers(0, 4, size=(H, n_onehot))
    p = {"W1": W1, "b1": np.full(H, 16.0, np.float32),
         "W2": np.eye(H, dtype=np.float32), "b2": np.zeros(H, np.float32),
         "W3": np.eye(H, dtype=np.float32), "b3": np.zeros(H, np.float32),
         "W4": (rng.integers(-2, 3, size=(K, H)) / 64.0).astype(np.float32),
         "b4": np.full(K, 600.0, np.float32)}
    return p


@pytest.mark.parametrize("seed", [0, 1, 2])
def test_mlp_search_exact_network_matches_oracle(kt, seed):
    from oracle import search as osearch
    desc, roles, gpu, valid, dig, C = tiny_setup(seed=seed)
    ranges = gpu.counter_ranges()
    sp = kt.Space.from_desc(desc)
    m = kt.Mlp(sp, roles, ranges, max_batch=64)
    p = exact_params(desc, m.F, len(roles), seed)
    m.set_params(p)
    pred = omlp.predict(p, desc.values, dig, ranges)
    # the network is exact: the GPU's predictions equal the oracle's bit for bit
    np.testing.assert_array_equal(m.predict(valid), pred)
    model = kt.Model.from_mlp(m)
    s = kt.Search(sp, model, k=5, seed=seed)
    o = osearch.OracleSearch(desc, {"roles": roles}, k=5, seed=seed, valid=valid, pred=pred)
    assert s.current() == o.cprof_raw
    for step in range(12):
        c = gpu.evaluate(ospace.decode(desc.radices, [s.current()]))[0][0]
        g_raw, g_sc = s.step(c)
        o_raw, o_sc = o.step(c)
        assert list(g_raw) == o_raw, step
        np.testing.assert_array_equal(np.asarray(g_sc, np.float32), np.float32(o_sc))
        rts = gpu.evaluate(ospace.decode(desc.radices, g_raw))[1]
        s.report(rts)
        o.report(list(rts))


def test_mlp_search_random_network_scores(kt):
    """A random network: the tensor cores' accumulation order moves
    predictions by a few 1e-3 of a counter's scale, so scores are compared
    within a tolerance (picks of the two sides may then differ)."""
    from oracle import expert, score as oscore
    desc, roles, gpu, valid, dig, C = tiny_setup()
    ranges = gpu.counter_ranges()
    sp = kt.Space.from_desc(desc)
    m = kt.Mlp(sp, roles, ranges, max_batch=64)
    p = random_params(m.F, len(roles), 11)
    # counters are positive: keep the predictions well above 0 (a + A near 0
    # would make Eq. score unbounded and amplify any rounding difference)
    p["W4"] = (p["W4"] * 0.1).astype(np.float32)
    p["b4"] = (np.abs(p["b4"]) + 1.0).astype(np.float32)
    m.set_params(p)
    pred = omlp.predict(p, desc.values, dig, ranges)
    model = kt.Model.from_mlp(m)
    pos = {int(r): i for i, r in enumerate(valid)}
    for seed in range(4):
        s = kt.Search(sp, model, k=8, seed=seed)
        s.set_timing(True)
        cp = pos[s.current()]
        c = gpu.evaluate(dig[cp:cp + 1])[0][0]
        g_raw, g_sc = s.step(c)
        d32 = expert.delta_vector(roles, c, 0.7, 1000.0).astype(np.float32)
        o_s = oscore.score_fp32(pred[cp], pred, d32)
        assert np.all(pred > 0)
        # |d term| <= |delta| * 2 (A |da| + a |dA|) / (a + A)^2 <= |delta| * 4 eps for
        # relative prediction errors eps; eps <= 1e-3 here
        bound = 4e-3 * float(np.sum(np.abs(d32))) + 1e-6
        assert len(set(g_raw)) == 8 and cp not in [pos[r] for r in g_raw]
        for r, sc in zip(g_raw, g_sc):
            assert abs(sc - o_s[pos[r]]) <= bound
        st = s.stats()
        free = np.ones(len(valid), bool)
        free[cp] = False
        assert abs(st.s_min - o_s[free].min()) <= bound
        assert abs(st.s_max - o_s[free].max()) <= bound
        assert st.n_active == int(np.count_nonzero(d32))


def test_mlp_model_rules(kt):
    desc, roles, gpu, valid, dig, C = tiny_setup()
    ranges = gpu.counter_ranges()
    sp = kt.Space.from_desc(desc)
    m = kt.Mlp(sp, roles, ranges, max_batch=64)
    model = kt.Model.from_mlp(m)
    with pytest.raises(kt.KtuneError):
        kt.Search(sp, model, k=5, select=kt.KTUNE_SELECT_TOPK)
    otf = kt.Space.from_desc(desc, flags=kt.KTUNE_ON_THE_FLY)
    m2 = kt.Mlp(otf, roles, ranges, max_batch=64)
    with pytest.raises(kt.KtuneError):
        kt.Search(otf, kt.Model.from_mlp(m2), k=5)
    s = kt.Search(sp, model, k=5)
    with pytest.raises(kt.KtuneError):
        kt.Batch([s, s])                      # the same search twice


def test_bounded_wait_runs_out_and_the_handle_recovers(kt):
    """Fault handling without a fault: with stall set, the forward kernel's
    copy and MMA warps first wait on a barrier that nothing arrives at; with a
    10 ms limit that wait runs out before any copy or MMA is issued, the
    kernel returns and the call reports KTUNE_ETIMEOUT.  The next normal call
    on the same handle gives the same predictions as before."""
    import time
    desc, roles, gpu, valid, dig, C = tiny_setup()
    sp = kt.Space.from_desc(desc)
    m = kt.Mlp(sp, roles, gpu.counter_ranges(), max_batch=64)
    m.set_params(random_params(m.F, len(roles), 3))
    ref = m.predict(valid)
    m.set_wait(10_000_000, stall=True)
    t0 = time.time()
    with pytest.raises(kt.KtuneError) as e:
        m.predict(valid)
    assert e.value.code == kt.KTUNE_ETIMEOUT
    assert time.time() - t0 < 10.0            # every wait gave up and the kernel returned
    m.set_wait(1_000_000_000, stall=False)
    np.testing.assert_array_equal(m.predict(valid), ref)
    with pytest.raises(kt.KtuneError) as e:
        m.set_wait(10, stall=False)           # below the allowed range
    assert e.value.code == kt.KTUNE_EINVAL
