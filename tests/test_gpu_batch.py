"""Batched steps: many searches over uneven spaces in one launch per kernel
must reproduce the searches run one at a time (which match the oracle),
before and after the autotuner picks a kernel shape."""
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


SPACES = ["batch_%d" % i for i in range(8)]
KS = [16, 32, 40, 32, 16, 40, 32, 16]
DEPTHS = [8, 12, 10, 12, 6, 11, 12, 9]


def make(kt, select, flags, per_space=2, stream=None, names=SPACES):
    out = []
    for si, name in enumerate(names):
        d = W.load_space(name)
        roles = W.layout(KS[si])
        model = random_model(d.radices, roles, depth=DEPTHS[si], seed=100 + si)
        gpu = SyntheticGPU(d, roles, seed=si)
        sp = kt.Space.from_desc(d, flags=flags)
        m = kt.Model(sp, model)
        for r in range(per_space):
            s = kt.Search(sp, m, k=5, seed=10 * si + r, search_id=r, select=select, stream=stream)
            out.append((d, gpu, sp, m, s))
    return out


def counters(entry):
    d, gpu, sp, m, s = entry
    return gpu.evaluate(ospace.decode(d.radices, [s.current()]))[0][0]


def runtimes(entry, raw):
    d, gpu = entry[0], entry[1]
    return gpu.evaluate(ospace.decode(d.radices, raw))[1]


def run_batch(kt, entries, steps, k, autotune=False, stream=None):
    b = kt.Batch([e[4] for e in entries], stream=stream)
    if autotune:
        choice, ms = b.autotune([counters(e) for e in entries], reps=2)
        assert 0 <= choice < len(ms) and np.all(ms[:1] > 0)
    seq = []
    for _ in range(steps):
        res = b.step([counters(e) for e in entries], k)
        seq.append([(list(r), list(sc)) for r, sc in res])
        for e, (r, sc) in zip(entries, res):
            e[4].report(runtimes(e, r))
    b.close()
    return seq


def run_single(entries, steps, k):
    seq = []
    for _ in range(steps):
        row = []
        for e in entries:
            r, sc = e[4].step(counters(e), k)
            row.append((list(r), list(sc)))
            e[4].report(runtimes(e, r))
        seq.append(row)
    return seq


@pytest.mark.parametrize("select,flags,autotune", [("sample", 0, False), ("sample", 0, True),
                                                   ("topk", 0, False), ("sample", 1, False),
                                                   ("topk", 1, True)])
def test_batch_matches_single_searches(kt, select, flags, autotune):
    import torch
    sel = kt.KTUNE_SELECT_TOPK if select == "topk" else kt.KTUNE_SELECT_SAMPLE
    k = 7
    a = make(kt, sel, flags)
    b = make(kt, sel, flags)
    stream = torch.cuda.Stream() if autotune else None
    got = run_batch(kt, a, 4, k, autotune=autotune, stream=stream)
    ref = run_single(b, 4, k)
    assert got == ref


def test_batch_rejects_mixed_modes(kt):
    e1 = make(kt, kt.KTUNE_SELECT_SAMPLE, 0, per_space=1, names=SPACES[:1])
    e2 = make(kt, kt.KTUNE_SELECT_TOPK, 0, per_space=1, names=SPACES[:1])
    with pytest.raises(kt.KtuneError):
        kt.Batch([e1[0][4], e2[0][4]])


def make_mixed(kt, stream=None):
    """Searches over three spaces, each space searched by two tree-scored and
    three MLP-scored searches (one untrained seeded network per space, whose
    scoring pass the three share in a batch), in one list."""
    from paper_2102_05297_gb300 import fit
    out, keep = [], []
    for si, name in enumerate(["batch_2", "batch_3", "batch_6"]):
        d = W.load_space(name)
        K = [16, 32, 40][si]
        roles = W.layout(K)
        gpu = SyntheticGPU(d, roles, seed=si)
        sp = kt.Space.from_desc(d)
        tm = kt.Model(sp, random_model(d.radices, roles, depth=10, seed=200 + si))
        mlp = kt.Mlp(sp, roles, gpu.counter_ranges(), max_batch=64)
        p = fit.init_mlp(mlp.F, K, seed=si)
        p["b4"] = np.full(K, 0.5, np.float32)        # predictions mostly positive
        mlp.set_params(p)
        mm = kt.Model.from_mlp(mlp)
        keep += [sp, tm, mlp, mm]
        for r, model in enumerate((tm, mm, mm, tm, mm)):   # three MLP searches share one pass
            s = kt.Search(sp, model, k=5, seed=30 + 10 * si + r, search_id=r, stream=stream)
            out.append((d, gpu, sp, model, s))
    return out, keep


def test_mixed_tree_and_mlp_batch_matches_single_searches(kt):
    """Tree-scored and MLP-scored searches in one batch (one CUDA graph per
    step) reproduce the same searches stepped one at a time."""
    import torch
    stream = torch.cuda.Stream()
    a, keep_a = make_mixed(kt, stream=stream)
    b, keep_b = make_mixed(kt)
    got = run_batch(kt, a, 4, 5, stream=stream)
    ref = run_single(b, 4, 5)
    assert got == ref
