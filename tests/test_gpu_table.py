"""A measured counter table as the model (model blob kind 2): the exact-counter
experiment of Section 4 (Table "tab:pc_bias"), where the counters measured for
every configuration stand in for a fitted model.

Steps over a table are compared with the oracle search given the same table
as its predictions: selections, scores and every score and integer weight of
each step bit for bit (the oracle's float32 Eq. score and weights), on a
batch space and on the full 2.26M-configuration mid space; the table's rows
read back exactly; the refusals; and the paper's directional claim that
exact counters guide the search to a near-optimal configuration in fewer
tests than uniform random draws."""
import numpy as np
import pytest

import workloads as W
from workloads.synth import SyntheticGPU
from oracle import search as osearch, space as ospace

from test_gpu_elementwise import readback, step_and_compare

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def kt():
    import torch
    assert torch.cuda.is_available()
    from paper_2102_05297_gb300 import ktune
    return ktune


def table_of(desc, roles, seed):
    gpu = SyntheticGPU(desc, roles, seed=seed)
    valid = ospace.enumerate_valid(desc)
    C, rt = gpu.evaluate(ospace.decode(desc.radices, valid))
    return gpu, valid, np.ascontiguousarray(C, np.float32), rt


@pytest.mark.parametrize("name,K,stream", [("batch_4", 32, False), ("batch_2", 16, True),
                                           ("mid_12p", 32, False)])
def test_table_steps_against_oracle(kt, name, K, stream):
    import torch
    d = W.load_space(name)
    roles = W.layout(K)
    gpu, valid, table, rt = table_of(d, roles, 3)
    sp = kt.Space.from_desc(d)
    m = kt.Model(sp, {"kind": "table", "roles": roles, "table": table})
    assert (m.K, m.depth) == (K, 0)
    st = torch.cuda.Stream() if stream else None
    s = kt.Search(sp, m, k=6, seed=5, stream=st)
    o = osearch.OracleSearch(d, {"roles": roles}, k=6, seed=5, valid=valid, pred=table)
    assert s.current() == o.cprof_raw
    pos = {int(r): i for i, r in enumerate(valid)}
    for _ in range(4):
        c = table[pos[s.current()]]
        raw = step_and_compare(kt, s, o, c, stream=st)
        r = rt[[pos[int(x)] for x in raw]]
        s.report(r)
        o.report(list(r))


def test_table_rows_and_rules(kt):
    import torch
    d = W.load_space("batch_3")
    roles = W.layout(16)
    gpu, valid, table, rt = table_of(d, roles, 1)
    sp = kt.Space.from_desc(d)
    m = kt.Model(sp, {"kind": "table", "roles": roles, "table": table})
    n = len(valid)
    out = torch.empty((n, 16), dtype=torch.float32, device="cuda")
    m.predict_device(0, n, out.data_ptr())
    torch.cuda.synchronize()
    np.testing.assert_array_equal(out.cpu().numpy(), table)
    with pytest.raises(kt.KtuneError) as e:
        kt.Model(sp, {"kind": "table", "roles": roles, "table": table[:-1]})   # wrong N
    assert e.value.code == kt.KTUNE_EMODEL
    bad = table.copy()
    bad[7, 3] = np.inf
    with pytest.raises(kt.KtuneError):
        kt.Model(sp, {"kind": "table", "roles": roles, "table": bad})
    otf = kt.Space.from_desc(d, flags=kt.KTUNE_ON_THE_FLY)
    with pytest.raises(kt.KtuneError) as e:
        kt.Model(otf, {"kind": "table", "roles": roles, "table": table})
    assert e.value.code == kt.KTUNE_ESTATE
    with pytest.raises(kt.KtuneError):
        kt.Search(sp, m, k=5, select=kt.KTUNE_SELECT_TOPK)
    s = kt.Search(sp, m, k=5)
    with pytest.raises(kt.KtuneError):
        s.set_cached(True)
    with pytest.raises(kt.KtuneError):
        kt.Batch([s])


def test_exact_counters_beat_random_search(kt):
    """Section 4's exact-counter experiment on a synthetic GPU: with the
    measured counters of every configuration as the model, the median number
    of tests to reach 10% of the optimum over 8 seeds is below the expected
    count of uniform random draws."""
    d = W.load_space("batch_3")
    roles = W.layout(16)
    gpu, valid, table, rt = table_of(d, roles, 4)
    sp = kt.Space.from_desc(d)
    m = kt.Model(sp, {"kind": "table", "roles": roles, "table": table})
    target = rt.min() * 1.1
    pos = {int(r): i for i, r in enumerate(valid)}
    tests = []
    for seed in range(8):
        s = kt.Search(sp, m, k=5, seed=seed)
        n = 1
        best = rt[pos[s.current()]]
        while best > target and n < 800:
            raw, _ = s.step(table[pos[s.current()]])
            r = rt[[pos[int(x)] for x in raw]]
            s.report(r)
            n += len(raw)
            best = min(best, r.min())
        tests.append(n)
    good = np.count_nonzero(rt <= target)
    random_expect = (len(valid) + 1) / (good + 1)
    assert np.median(tests) < random_expect, (tests, random_expect)
