"""What the trained network gains over the method without it.

The MLP counter model is trained on the GPU (the library's forward and
backward tensor-core kernels, Adam) on the same noisy profile sample the tree
model is fitted on.  What it gains: on held-out configurations its counter
predictions are closer to the noise-free synthetic counters (range-normalised
RMSE below 0.8 of the trees'), and the counter-guided search it drives reaches
a configuration within 10% of the space's optimum in fewer empirical tests
than random search.  The tree-guided search's count is printed beside it, not
asserted: on this space the trees guide the search better although their
counter RMSE is higher (the score reacts to ratios of predicted counters, and
the network, trained on range-normalised errors, is least accurate in
relative terms on the counters with small values)."""
import numpy as np
import pytest

import workloads as W
from workloads.synth import SyntheticGPU, add_noise, sample_indices
from oracle import space as ospace

pytestmark = pytest.mark.gpu

SPACE, K, FRAC, DEPTH = "batch_4", 32, 0.03, 10
SEEDS = range(8)
TARGET = 1.10          # within 10% of the best runtime of the whole space
MAX_STEPS = 60


@pytest.fixture(scope="module")
def setup():
    import torch
    assert torch.cuda.is_available()
    from paper_2102_05297_gb300 import fit, ktune as kt
    d = W.load_space(SPACE)
    roles = W.layout(K)
    gpu = SyntheticGPU(d, roles, seed=4)
    sp = kt.Space.from_desc(d)
    valid = sp.valid_raw()
    dig = sp.valid_digits()
    C, T = gpu.evaluate(dig)
    samp = sample_indices(len(valid), FRAC, 1)
    Y = add_noise(C[samp], 1, 0.02)
    trees = fit.fit_model(dig[samp], Y, DEPTH, d.radices, roles)
    tm = kt.Model(sp, trees)
    ranges = gpu.counter_ranges()
    mlp = kt.Mlp(sp, roles, ranges, max_batch=1024)
    mlp.set_params(fit.init_mlp(mlp.F, K, seed=0))
    mlp.set_data(valid[samp], Y)
    rng = np.random.default_rng(2)
    steps, B = 1500, 1024
    losses = mlp.train(rng.integers(0, len(samp), size=steps * B).astype(np.int32), B)
    assert losses[-1] < 0.2 * losses[0]
    mm = kt.Model.from_mlp(mlp)
    return dict(kt=kt, d=d, roles=roles, gpu=gpu, sp=sp, valid=valid, dig=dig, C=C, T=T,
                samp=samp, tm=tm, mlp=mlp, mm=mm, ranges=ranges)


def rmse(pred, truth, ranges):
    e = (np.asarray(pred, np.float64) - truth) / ranges
    return float(np.sqrt(np.mean(e * e)))


def test_network_predicts_counters_better_than_trees(setup):
    import torch
    s = setup
    n = len(s["valid"])
    held = np.setdiff1d(np.arange(n), s["samp"])[::7]
    truth = s["C"][held].astype(np.float64)
    r_mlp = rmse(s["mlp"].predict(s["valid"][held]), truth, s["ranges"])
    out = torch.empty((n, K), dtype=torch.float32, device="cuda")
    s["tm"].predict_device(0, n, out.data_ptr())
    torch.cuda.synchronize()
    r_tree = rmse(out.cpu().numpy()[held], truth, s["ranges"])
    print("held-out counter RMSE: mlp %.4f, trees %.4f" % (r_mlp, r_tree))
    assert r_mlp < 0.8 * r_tree


def _tests_to_target(s, model, seed):
    kt = s["kt"]
    best_t = float(np.min(s["T"]))
    pos = {int(r): i for i, r in enumerate(s["valid"])}
    srch = kt.Search(s["sp"], model, k=5, seed=seed)
    tested = 1
    best = s["T"][pos[srch.current()]]
    for _ in range(MAX_STEPS):
        if best <= TARGET * best_t:
            break
        cp = pos[srch.current()]
        raw, _ = srch.step(s["C"][cp])
        rts = s["T"][[pos[int(r)] for r in raw]]
        tested += len(raw)
        best = min(best, float(np.min(rts)))
        srch.report(rts)
    srch.close()
    return tested


def _random_tests_to_target(s, seed):
    best_t = float(np.min(s["T"]))
    order = np.random.default_rng(1000 + seed).permutation(len(s["T"]))
    hit = np.flatnonzero(s["T"][order] <= TARGET * best_t)
    return int(hit[0]) + 1


def test_network_guided_search_gains(setup):
    s = setup
    mlp_t = [_tests_to_target(s, s["mm"], sd) for sd in SEEDS]
    tree_t = [_tests_to_target(s, s["tm"], sd) for sd in SEEDS]
    rand_t = [_random_tests_to_target(s, sd) for sd in SEEDS]
    print("empirical tests to reach %.0f%% of the optimum: mlp %s (mean %.1f), trees %s (mean %.1f), "
          "random %s (mean %.1f)" % (100 * TARGET, mlp_t, np.mean(mlp_t), tree_t, np.mean(tree_t),
                                     rand_t, np.mean(rand_t)))
    assert np.mean(mlp_t) < np.mean(rand_t)
