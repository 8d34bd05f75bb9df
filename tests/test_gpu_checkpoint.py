"""Search checkpoints (ktune_search_save / ktune_search_load): a search
restored from a checkpoint continues exactly as the original -- the same
draws (the Philox counter includes the step number), the same selections and
scores, in both select modes and on materialised and on-the-fly spaces; a
checkpoint of another space, a truncated one, or one for another model is
rejected."""
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


def drive(kt, s, gpu, radices, steps):
    out = []
    for _ in range(steps):
        c = gpu.evaluate(ospace.decode(radices, [s.current()]))[0][0]
        raw, sc = s.step(c)
        out.append((list(raw), list(sc)))
        s.report(gpu.evaluate(ospace.decode(radices, raw))[1])
    return out


@pytest.mark.parametrize("name,flags,select", [("batch_2", 0, "sample"), ("batch_2", 0, "topk"),
                                                ("batch_0", 1, "sample")])
def test_resume_continues_identically(kt, name, flags, select):
    d = W.load_space(name)
    roles = W.layout(16)
    model = random_model(d.radices, roles, depth=8, seed=5)
    gpu = SyntheticGPU(d, roles, seed=2)
    sp = kt.Space.from_desc(d, flags=flags)
    m = kt.Model(sp, model)
    sel = kt.KTUNE_SELECT_TOPK if select == "topk" else kt.KTUNE_SELECT_SAMPLE
    s = kt.Search(sp, m, k=6, seed=3, select=sel)
    drive(kt, s, gpu, d.radices, 4)
    blob = s.save()
    ref = drive(kt, s, gpu, d.radices, 5)
    r = kt.Search.load(sp, m, blob)
    assert r.evaluated() == 1 + 4 * 6
    got = drive(kt, r, gpu, d.radices, 5)
    assert got == ref
    # a checkpoint taken while a batch awaits its report resumes with the report
    c = gpu.evaluate(ospace.decode(d.radices, [r.current()]))[0][0]
    raw, _ = r.step(c)
    blob2 = r.save()
    r2 = kt.Search.load(sp, m, blob2)
    rts = gpu.evaluate(ospace.decode(d.radices, raw))[1]
    r.report(rts)
    r2.report(rts)
    assert r.current() == r2.current()
    assert drive(kt, r, gpu, d.radices, 2) == drive(kt, r2, gpu, d.radices, 2)


def test_load_rejects_mismatches(kt):
    d = W.load_space("batch_2")
    roles = W.layout(16)
    sp = kt.Space.from_desc(d)
    m = kt.Model(sp, random_model(d.radices, roles, depth=8, seed=5))
    blob = kt.Search(sp, m, k=4, seed=1).save()
    other = kt.Space.from_desc(W.load_space("batch_0"))
    m_other = kt.Model(other, random_model(W.load_space("batch_0").radices, roles, depth=8, seed=5))
    with pytest.raises(kt.KtuneError):
        kt.Search.load(other, m_other, blob)                 # another space
    with pytest.raises(kt.KtuneError):
        kt.Search.load(sp, m, blob[:-4])                      # truncated
    with pytest.raises(kt.KtuneError):
        kt.Search.load(sp, m, b"\\0" * 16)                    # not a checkpoint
    m6 = kt.Model(sp, random_model(d.radices, roles, depth=6, seed=5))
    with pytest.raises(kt.KtuneError) as e:
        kt.Search.load(sp, m6, blob)                          # another model depth
    assert e.value.code == kt.KTUNE_EMODEL
