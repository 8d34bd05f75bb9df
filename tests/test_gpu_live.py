"""The search on real profiles (paper_2102_05297_gb300.live): the tunable
kernel computes the same potential in every configuration (the same
summation order, so the same bits), the ncu counters of one launch convert to
a plausible counter vector that ktune_step accepts, and a short search on
real profiles runs end to end.  Each profile is one launch of a small
kernel, captured after the same program has run without ncu."""
import shutil

import numpy as np
import pytest

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def live():
    import torch
    assert torch.cuda.is_available()
    if shutil.which("ncu") is None:
        pytest.skip("ncu is not on PATH")
    from paper_2102_05297_gb300 import live
    return live


def test_every_configuration_computes_the_same_grid(live):
    sp = live.space()
    n, n_raw = sp.count()
    assert (n, n_raw) == (242, 288)
    rows = live.rows_of(sp.valid_digits())
    ms, checks = live.time_configs(rows[::11], reps=3)
    assert np.all(ms > 0) and np.all(checks == checks[0])


def test_profile_counters_and_a_short_search(live):
    from paper_2102_05297_gb300 import ktune as kt
    sp = live.space()
    rows = live.rows_of(sp.valid_digits())
    C = live.profile(rows[[0, 57, 241]])
    assert C.shape == (3, 25) and np.all(np.isfinite(C))
    names = live.nc.ROLE_NAMES
    f32, exe, glob = names.index("INST_F32"), names.index("INST_EXE"), names.index("GLOBAL")
    assert np.all(C[:, f32] > 0) and np.all(C[:, exe] > 0)
    for i, r in enumerate([0, 57, 241]):
        bx, by, out = rows[r][:3]
        assert C[i, glob] == 512 * 512 // out         # threads launched
    for u in ("INST_ISSUE_U", "DRAM_U", "L2_U", "SM_E"):
        assert np.all((C[:, names.index(u)] >= 0) & (C[:, names.index(u)] <= 100.5))
    rec = live.run(seeds=[0], k=5, sample_frac=0.1, depth=6, max_tests=16, log=lambda *a: None)
    s = rec["searches"][0]
    assert s["steps"] >= 1 and s["tests"] >= 6 and rec["checksums_equal"]
