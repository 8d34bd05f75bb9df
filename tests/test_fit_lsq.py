"""The package's least-squares fitter (Section 3.3.1) and its model blob,
checked against the oracle on the CPU: the same coefficients on samples that
determine them, the same fallback for a subspace without samples, and the
blob layout of include/ktune.h."""
import struct

import numpy as np

import workloads as W
from workloads.synth import SyntheticGPU, add_noise, sample_indices
from oracle import lsq as olsq, space as ospace
from paper_2102_05297_gb300.fit import fit_lsq, lsq_shape


def test_shape_matches_oracle_design():
    d = W.load_space("mid_12p")
    binary, regs, u = lsq_shape(d.values)
    o = olsq.design(d.values)
    assert binary == o["binary"] and regs == o["regs"]
    for j in regs:
        np.testing.assert_allclose(u[j], o["u"][j], rtol=0, atol=1e-15)


def test_fit_matches_oracle_on_sampled_counters():
    d = W.load_space("batch_3")
    roles = W.layout(16)
    gpu = SyntheticGPU(d, roles, seed=1)
    valid = ospace.enumerate_valid(d)
    dig = ospace.decode(d.radices, valid)
    idx = sample_indices(len(valid), 0.05, seed=1)
    Y = add_noise(gpu.evaluate(dig[idx])[0], seed=1)
    model = fit_lsq(d.values, dig[idx], Y, roles)
    ref = olsq.fit(d.values, dig[idx], Y)
    assert model["coef"].dtype == np.float32 and model["coef"].shape == ref.shape
    scale = np.abs(ref).max(axis=2, keepdims=True) + 1e-30
    assert np.all(np.abs(model["coef"] - ref) <= 1e-6 * scale)


def test_fit_fallback_and_blob_layout():
    from paper_2102_05297_gb300 import ktune
    values = [[0, 1], [1, 2, 4, 8], [3, 6, 9], [0, 1]]
    dig = np.array([[a, b, c, e] for a in range(2) for b in range(4) for c in range(3) for e in range(2)
                    if not (a == 1 and e == 1)])
    Y = (dig[:, 1] * 1.5 - dig[:, 2] + 0.25 * dig[:, 0])[:, None]
    model = fit_lsq(values, dig, Y, [3])
    ref = olsq.fit(values, dig, Y)
    np.testing.assert_allclose(model["coef"], ref, rtol=0, atol=1e-5)
    blob = ktune.model_blob(model)
    magic, ver, kind, K, role, n_sub, T = struct.unpack_from("<4Ii2I", blob)
    assert (magic, ver, kind, K, role, n_sub, T) == (0x314D544B, 1, 3, 1, 3, 4, 6)
    assert len(blob) == 28 + 4 * 4 * 6
    np.testing.assert_array_equal(np.frombuffer(blob[28:], "<f4").reshape(4, 1, 6), model["coef"])
