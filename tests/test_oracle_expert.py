"""Pins of the expert system: hand-computed cases of each equation of
Sections 3.4.1 and 3.4.2."""
import math

import numpy as np
import pytest

import workloads as W
from oracle import expert

R = W.ROLE


def pc(**kw):
    return {k: float(v) for k, v in kw.items()}


def test_memory_read_write_split():
    B = expert.bottlenecks(pc(DRAM_RT=3, DRAM_WT=1, DRAM_U=80), cores=1000)
    assert B["dram_read"] == pytest.approx(0.6, abs=1e-15)
    assert B["dram_write"] == pytest.approx(0.2, abs=1e-15)
    D = expert.delta_by_name(B, 0.7)
    assert D["DRAM_RT"] == pytest.approx(-0.6) and D["DRAM_WT"] == pytest.approx(-0.2)
    # the same form for L2 and shared memory
    B = expert.bottlenecks(pc(L2_RT=1, L2_WT=4, L2_U=50, SHR_LT=2, SHR_WT=2, SHR_U=30), 1000)
    assert B["l2_read"] == pytest.approx(0.1) and B["l2_write"] == pytest.approx(0.4)
    assert B["shr_read"] == pytest.approx(0.15) and B["shr_write"] == pytest.approx(0.15)


def test_no_transactions_no_bottleneck():
    B = expert.bottlenecks(pc(DRAM_RT=0, DRAM_WT=0, DRAM_U=90), 1000)
    assert B["dram_read"] == 0.0 and B["dram_write"] == 0.0


def test_tex_and_local():
    B = expert.bottlenecks(pc(TEX_U=45, LOC_O=50, DRAM_U=40, L2_U=60), 1000)
    assert B["tex"] == pytest.approx(0.45)
    assert B["local"] == pytest.approx(0.5 * 0.6)


def test_instruction_bottlenecks_and_reaction():
    # ins_fitted = 32 * 10 * (100/50) * (100/100) = 640; ins_util = min(1, 40/50) = 0.8
    p = pc(INST_EXE=10, WARP_E=50, WARP_NP_E=100, INST_ISSUE_U=40, INST_F32=576, INST_INT=64)
    B = expert.bottlenecks(p, 1000)
    assert B["INST_F32"] == pytest.approx(0.9 * 0.8)
    assert B["INST_INT"] == pytest.approx(0.1 * 0.8)
    # Eq. maxutil / issue: 0.9 * (100 - 40) / 100
    assert B["issue"] == pytest.approx(0.54)
    D = expert.delta_by_name(B, 0.7)
    assert D["INST_F32"] == pytest.approx(-(0.72 - 0.7) / 0.3)
    assert D["INST_INT"] == 0.0 and D["INST_ISSUE_U"] == 0.0
    D = expert.delta_by_name(B, 0.5)
    assert D["INST_F32"] == pytest.approx(-(0.72 - 0.5) / 0.5)
    assert D["INST_ISSUE_U"] == pytest.approx(-(0.54 - 0.5) / 0.5)


def test_issue_util_caps_at_one():
    B = expert.bottlenecks(pc(INST_EXE=1, INST_ISSUE_U=90, INST_LDST=32), 1000)
    assert B["INST_LDST"] == pytest.approx(1.0)


@pytest.mark.parametrize("b,r,expect", [(0.7, 0.7, 0.0), (0.85, 0.7, -0.5), (1.0, 0.7, -1.0),
                                        (0.3, 0.5, 0.0), (0.75, 0.5, -0.5)])
def test_reaction_cases(b, r, expect):
    assert expert.reaction(b, r) == pytest.approx(expect)


def test_parallelism():
    B = expert.bottlenecks(pc(SM_E=70, GLOBAL=2000), cores=1000)
    assert B["sm"] == pytest.approx(0.3)
    assert B["paral"] == pytest.approx(0.6)
    D = expert.delta_by_name(B, 0.7)
    assert D["SM_E"] == pytest.approx(0.3) and D["GLOBAL"] == pytest.approx(0.6)
    assert expert.bottlenecks(pc(GLOBAL=6000), 1000)["paral"] == 0.0
    assert expert.bottlenecks(pc(), 1000)["paral"] == 0.0


def test_layout_mapping_and_defaults():
    roles = W.layout(16)
    c = np.zeros(16)
    c[roles.index(R["DRAM_RT"])] = 3
    c[roles.index(R["DRAM_WT"])] = 1
    c[roles.index(R["DRAM_U"])] = 80
    d = expert.delta_vector(roles, c)
    assert d[roles.index(R["DRAM_RT"])] == pytest.approx(-0.6)
    assert d[roles.index(R["DRAM_U"])] == 0.0              # stress counters get no Delta
    # K=32: inert counters never get a Delta
    roles32 = W.layout(32)
    c32 = np.full(32, 50.0)
    d32 = expert.delta_vector(roles32, c32)
    assert all(d32[k] == 0.0 for k, r in enumerate(roles32) if r == R["INERT"])
    assert np.all(np.abs(d32) <= 1.0)


def test_clamping():
    B = expert.bottlenecks(pc(DRAM_RT=1, DRAM_WT=0, DRAM_U=250, SM_E=-50), 1000)
    assert B["dram_read"] == 1.0 and B["sm"] == 1.0
