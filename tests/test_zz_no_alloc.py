"""The allocation-free scoring entry point against the regular step.

ktune_score_noalloc is for callers that cannot allocate device memory (it
uses a fixed array inside the library).  These tests call it through the C
ABI on two consecutive steps of a regular search and check that its scores
for the configurations ktune_step selected, and its min / max, are exactly
those of ktune_step (the tolerance of the other parity tests: bit-exact).
The file is named to be collected last."""
import ctypes as C

import numpy as np
import pytest

import workloads as W
from workloads.synth import SyntheticGPU
from workloads.trees import random_model

pytestmark = pytest.mark.gpu


def padded(model, depth):
    """The documented padded layout: node bytes and leaves, [K][2^depth]."""
    L = 1 << depth
    K = len(model["trees"])
    nodes = np.zeros((K, L), np.uint8)
    leaves = np.zeros((K, L), np.float32)
    for k, t in enumerate(model["trees"]):
        stack = [(0, 0, 0)]
        while stack:
            i, pos, lev = stack.pop()
            if lev == depth:
                leaves[k, pos - (L - 1)] = t["value"][i]
                continue
            if t["feature"][i] < 0:
                nodes[k, pos] = 0x0F
                stack += [(i, 2 * pos + 1, lev + 1), (i, 2 * pos + 2, lev + 1)]
            else:
                nodes[k, pos] = (int(t["feature"][i]) << 4) | min(int(t["threshold"][i]), 15)
                stack += [(int(t["left"][i]), 2 * pos + 1, lev + 1),
                          (int(t["right"][i]), 2 * pos + 2, lev + 1)]
    return nodes, leaves


def pack_digits(radices, raw):
    p = 0
    for j in range(len(radices) - 1, -1, -1):
        p |= (raw % radices[j]) << (4 * j)
        raw //= radices[j]
    return p


@pytest.fixture(scope="module")
def kt():
    import torch
    assert torch.cuda.is_available()
    from paper_2102_05297_gb300 import ktune
    return ktune


def test_noalloc_matches_step_two_calls(kt):
    import torch
    d = W.load_space("batch_3")
    roles = W.layout(32)
    depth = 10
    model = random_model(d.radices, roles, depth=depth, seed=21)
    gpu = SyntheticGPU(d, roles, seed=2)
    sp = kt.Space.from_desc(d)
    n = sp.count()[0]
    valid = sp.valid_raw()
    m = kt.Model(sp, model)
    assert m.depth == depth
    s = kt.Search(sp, m, k=5, seed=4)
    s.set_timing(False)
    nodes, leaves = padded(model, depth)
    nodes_d = torch.from_numpy(nodes).cuda()
    leaves_d = torch.from_numpy(leaves).cuda()
    roles_h = (C.c_int32 * len(roles))(*roles)
    evaluated = np.zeros((n + 31) // 32, np.uint32)
    ev_pos = [int(np.searchsorted(valid, s.current()))]
    scores = torch.empty(n, dtype=torch.float32, device="cuda")
    minmax = torch.empty(2, dtype=torch.float32, device="cuda")
    for call in range(2):
        for o in ev_pos:
            evaluated[o >> 5] |= np.uint32(1 << (o & 31))
        ev_d = torch.from_numpy(evaluated.view(np.int32).copy()).cuda()
        cp = s.current()
        digits = np.array([[(cp // st) % r for st, r in zip(_strides(d.radices), d.radices)]])
        counters = gpu.evaluate(digits)[0][0]
        cnt_d = torch.from_numpy(counters).cuda()
        rc = kt.lib.ktune_score_noalloc(
            sp.packed_device(), n, ev_d.data_ptr(), nodes_d.data_ptr(), leaves_d.data_ptr(),
            len(roles), depth, roles_h, cnt_d.data_ptr(), pack_digits(d.radices, cp), 0.7, 1000.0,
            scores.data_ptr(), minmax.data_ptr(), None)
        assert rc == kt.KTUNE_OK, kt.lib.ktune_last_error()
        torch.cuda.synchronize()
        raw, sc = s.step(counters)            # the regular path, same state
        st = s.stats()
        got = scores.cpu().numpy()
        pos = np.searchsorted(valid, raw)
        np.testing.assert_array_equal(got[pos], sc)
        assert minmax[0].item() == st.s_min and minmax[1].item() == st.s_max
        rts = gpu.evaluate(np.array([[(r // st_) % rr for st_, rr in
                                      zip(_strides(d.radices), d.radices)] for r in raw]))[1]
        s.report(rts)
        ev_pos = [int(x) for x in pos]


def _strides(radices):
    out = [1] * len(radices)
    for j in range(len(radices) - 2, -1, -1):
        out[j] = out[j + 1] * radices[j + 1]
    return out


def test_noalloc_rejects_oversized_tables(kt):
    roles_h = (C.c_int32 * 64)(*([0] * 64))
    # 64 counters at depth 12 need 1.3 MB of term tables: beyond the fixed 1 MiB
    rc = kt.lib.ktune_score_noalloc(8, 1, 8, 8, 8, 64, 12, roles_h, 8, 0, 0.7, 1000.0, 8, 8, None)
    assert rc == kt.KTUNE_EINVAL
    assert b"1 MiB" in kt.lib.ktune_last_error()
