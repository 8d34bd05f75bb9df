"""The allocation-free scoring entry point against the oracle and the regular step.

ktune_score_noalloc is for callers that cannot allocate device memory (a
plugin whose host framework owns all device memory, or a loop that cannot
afford the synchronisation of cudaMalloc / cudaFree); it keeps its working
memory in a fixed array inside the library.  These tests call it through the C
ABI and check

  * every one of its n scores against the oracle's float32 score of the same
    configuration (0 for evaluated ones), bit for bit, and its min / max, on
    two consecutive steps of a regular search, whose selected configurations'
    scores and min / max it must also reproduce exactly;
  * a case whose trees do not fit the scoring kernel's shared memory at once
    (depth 13, several groups of active trees staged one after another);
  * its own (device) bottleneck analysis on hand-made counter vectors that
    reach the degenerate branches of Section 3.4 (no memory traffic, no
    instructions, zero warp efficiencies, few threads), through the scores it
    yields against the oracle's float64 expert system.

The file is named to be collected last."""
import ctypes as C

import numpy as np
import pytest

import workloads as W
from workloads.synth import SyntheticGPU
from workloads.trees import random_model
from oracle import expert, score as oscore, space as ospace, trees as otrees

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


class NoAlloc:
    """Device copies of a space's TS and a padded tree ensemble, and one call
    of ktune_score_noalloc over them (the caller's buffers)."""

    def __init__(self, kt, sp, model, depth):
        import torch
        self.kt, self.torch = kt, torch
        self.sp = sp
        self.n = sp.count()[0]
        self.roles = list(model["roles"])
        self.depth = depth
        nodes, leaves = padded(model, depth)
        self.nodes_d = torch.from_numpy(nodes).cuda()
        self.leaves_d = torch.from_numpy(leaves).cuda()
        self.roles_h = (C.c_int32 * len(self.roles))(*self.roles)
        self.scores = torch.empty(self.n, dtype=torch.float32, device="cuda")
        self.minmax = torch.empty(2, dtype=torch.float32, device="cuda")

    def __call__(self, evaluated, counters, cprof_packed):
        torch = self.torch
        ev_d = torch.from_numpy(evaluated.view(np.int32).copy()).cuda()
        cnt_d = torch.from_numpy(np.asarray(counters, np.float32).copy()).cuda()
        rc = self.kt.lib.ktune_score_noalloc(
            self.sp.packed_device(), self.n, ev_d.data_ptr(), self.nodes_d.data_ptr(),
            self.leaves_d.data_ptr(), len(self.roles), self.depth, self.roles_h, cnt_d.data_ptr(),
            cprof_packed, 0.7, 1000.0, self.scores.data_ptr(), self.minmax.data_ptr(), None)
        assert rc == self.kt.KTUNE_OK, self.kt.lib.ktune_last_error()
        torch.cuda.synchronize()
        return self.scores.cpu().numpy(), self.minmax.cpu().numpy()


def oracle_scores(pred, cprof_pos, roles, counters, free):
    d32 = expert.delta_vector(roles, counters, 0.7, 1000.0).astype(np.float32)
    s = oscore.score_fp32(pred[cprof_pos], pred, d32)
    return np.where(free, s, np.float32(0.0)).astype(np.float32), d32


def assert_all_scores(got, mm, ref, free):
    bad = np.nonzero(got.view(np.uint32) != ref.view(np.uint32))[0]
    assert len(bad) == 0, ("scores differ", len(bad), bad[:5])
    assert mm[0] == ref[free].min() and mm[1] == ref[free].max()


def evaluated_bits(n, positions):
    ev = np.zeros((n + 31) // 32, np.uint32)
    for o in positions:
        ev[o >> 5] |= np.uint32(1 << (o & 31))
    return ev


def test_noalloc_matches_oracle_and_step_two_calls(kt):
    d = W.load_space("batch_3")
    roles = W.layout(32)
    depth = 10
    model = random_model(d.radices, roles, depth=depth, seed=21)
    gpu = SyntheticGPU(d, roles, seed=2)
    sp = kt.Space.from_desc(d)
    n = sp.count()[0]
    valid = sp.valid_raw()
    pred = otrees.predict(model, ospace.decode(d.radices, valid))
    m = kt.Model(sp, model)
    assert m.depth == depth
    s = kt.Search(sp, m, k=5, seed=4)
    call = NoAlloc(kt, sp, model, depth)
    free = np.ones(n, bool)
    ev_pos = [int(np.searchsorted(valid, s.current()))]
    for _ in range(2):
        free[ev_pos] = False
        cp = s.current()
        cpos = int(np.searchsorted(valid, cp))
        counters = gpu.evaluate(ospace.decode(d.radices, [cp]))[0][0]
        got, mm = call(evaluated_bits(n, np.nonzero(~free)[0]), counters, pack_digits(d.radices, cp))
        ref, _ = oracle_scores(pred, cpos, roles, counters, free)
        assert_all_scores(got, mm, ref, free)
        raw, sc = s.step(counters)            # the regular path, same state
        st = s.stats()
        pos = np.searchsorted(valid, raw)
        np.testing.assert_array_equal(got[pos], sc)
        assert mm[0] == st.s_min and mm[1] == st.s_max
        s.report(gpu.evaluate(ospace.decode(d.radices, raw))[1])
        ev_pos = [int(x) for x in pos]


def test_noalloc_trees_staged_in_groups(kt):
    """Depth-13 trees take 40 KB each in the scoring kernel's shared memory,
    which holds five at a time: with more active counters the kernel stages
    them group by group."""
    d = W.load_space("batch_2")
    roles = W.layout(16)
    depth = 13
    model = random_model(d.radices, roles, depth=depth, seed=5)
    gpu = SyntheticGPU(d, roles, seed=5)
    sp = kt.Space.from_desc(d)
    n = sp.count()[0]
    valid = sp.valid_raw()
    pred = otrees.predict(model, ospace.decode(d.radices, valid))
    call = NoAlloc(kt, sp, model, depth)
    rng = np.random.default_rng(1)
    for trial in range(3):
        cpos = int(rng.integers(0, n))
        cp = int(valid[cpos])
        counters = gpu.evaluate(ospace.decode(d.radices, [cp]))[0][0]
        free = np.ones(n, bool)
        free[rng.choice(n, size=n // 7, replace=False)] = False
        free[cpos] = False
        ref, d32 = oracle_scores(pred, cpos, roles, counters, free)
        n_active = int(np.count_nonzero((d32 != 0) & (pred[cpos] != 0)))
        assert n_active > 5, n_active        # more than one group of five
        got, mm = call(evaluated_bits(n, np.nonzero(~free)[0]), counters,
                       pack_digits(d.radices, cp))
        assert_all_scores(got, mm, ref, free)


def hand_counters(roles):
    """Counter vectors (by role name) that drive the expert system through its
    degenerate and saturated branches."""
    cases = [
        {},                                                            # all zero
        {"DRAM_RT": 300.0, "DRAM_WT": 100.0, "DRAM_U": 80.0},          # 0.6 / 0.2
        {"DRAM_RT": 0.0, "DRAM_WT": 0.0, "DRAM_U": 90.0, "L2_RT": 5.0, "L2_U": 120.0},
        {"INST_EXE": 100.0, "INST_F32": 2800.0, "INST_ISSUE_U": 60.0, "WARP_E": 0.0,
         "WARP_NP_E": 0.0},                                            # zero efficiencies
        {"INST_EXE": 50.0, "INST_INT": 1500.0, "INST_LDST": 200.0, "INST_ISSUE_U": 25.0,
         "WARP_E": 100.0, "WARP_NP_E": 50.0, "SM_E": 40.0},
        {"GLOBAL": 1200.0, "TEX_U": 75.0, "TEX_RWT": 10.0, "LOC_O": 30.0, "L2_U": 40.0},
        {"SHR_LT": 10.0, "SHR_WT": 30.0, "SHR_U": 100.0, "GLOBAL": 1e7, "SM_E": 100.0},
    ]
    out = []
    for c in cases:
        v = np.zeros(len(roles), np.float32)
        for i, r in enumerate(roles):
            v[i] = c.get(W.ROLE_NAMES[r], 0.0)
        out.append(v)
    return out


def test_noalloc_device_expert_system_hand_cases(kt):
    d = W.load_space("batch_4")
    roles = W.layout(32)
    depth = 9
    model = random_model(d.radices, roles, depth=depth, seed=8)
    sp = kt.Space.from_desc(d)
    n = sp.count()[0]
    valid = sp.valid_raw()
    pred = otrees.predict(model, ospace.decode(d.radices, valid))
    call = NoAlloc(kt, sp, model, depth)
    cpos = n // 3
    free = np.ones(n, bool)
    free[cpos] = False
    ev = evaluated_bits(n, [cpos])
    seen_active = 0
    for counters in hand_counters(roles):
        ref, d32 = oracle_scores(pred, cpos, roles, counters, free)
        seen_active += int(np.count_nonzero(d32))
        got, mm = call(ev, counters, pack_digits(d.radices, int(valid[cpos])))
        assert_all_scores(got, mm, ref, free)
    assert seen_active > 0


def test_noalloc_rejects_oversized_tables(kt):
    roles_h = (C.c_int32 * 64)(*([0] * 64))
    # 64 counters at depth 12 need 1.3 MB of term tables: beyond the fixed 1 MiB
    rc = kt.lib.ktune_score_noalloc(8, 1, 8, 8, 8, 64, 12, roles_h, 8, 0, 0.7, 1000.0, 8, 8, None)
    assert rc == kt.KTUNE_EINVAL
    assert b"1 MiB" in kt.lib.ktune_last_error()
