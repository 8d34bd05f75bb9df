"""Least-squares non-linear regression counter model (oracle).

Test infrastructure only: tests, the package smoke check and the bench's CPU
baseline use it; the library never does.

Section 3.3.1 of the paper: the tuning space is split into subspaces by the
values of its binary tuning parameters (b binary parameters give 2^b
subspaces); within each subspace, each counter is modelled from the
non-binary parameters with main effects, quadratic terms and interactions,
and the coefficients are computed by least squares.

Readings of this build where the paper is silent:
  * regressor of a non-binary parameter j: its value mapped to [-1, 1] on a
    log scale, u = 2 (log2(1 + v) - lo) / (hi - lo) - 1 over j's value list;
    parameters with one value are constant and take no part;
  * terms, in this order: 1; u_j for each non-binary j (ascending j); u_j^2;
    u_i u_j for i < j (lexicographic) -- interactions up to order two;
    T = 1 + 2m + m(m - 1)/2 for m non-binary parameters;
  * subspace index: the binary parameters' digits as bits, the first binary
    parameter the most significant;
  * training points: the profiled sample, whatever it is (the paper chooses
    2-3 values per parameter and subspace; here the sample is given);
  * least squares per subspace and counter: the minimum-norm solution
    (numpy.linalg.lstsq); a subspace without samples takes the fit over all
    samples.
Predictions are float64 here.  Parity unpinned beyond the definition: the
pins below check the definition (exact recovery, normal equations, subspace
split), not agreement with the paper's own models.
"""
from __future__ import annotations

from typing import Dict, List

import numpy as np


def design(values: List[List[int]]) -> Dict:
    """Which parameters split subspaces, which are regressors, and the u table."""
    binary = [j for j, v in enumerate(values) if len(v) == 2]
    regs = [j for j, v in enumerate(values) if len(v) >= 3]
    u = {}
    for j in regs:
        lv = np.log2(1.0 + np.asarray(values[j], dtype=np.float64))
        lo, hi = lv.min(), lv.max()
        u[j] = 2.0 * (lv - lo) / (hi - lo) - 1.0
    m = len(regs)
    return {"binary": binary, "regs": regs, "u": u, "n_sub": 1 << len(binary),
            "T": 1 + 2 * m + m * (m - 1) // 2}


def terms(d: Dict, digits: np.ndarray) -> np.ndarray:
    """Design matrix rows [n, T] of configurations given by digits [n, P]."""
    digits = np.atleast_2d(np.asarray(digits, dtype=np.int64))
    n = digits.shape[0]
    U = np.stack([d["u"][j][digits[:, j]] for j in d["regs"]], axis=1) if d["regs"] else np.zeros((n, 0))
    cols = [np.ones(n)]
    cols += [U[:, a] for a in range(U.shape[1])]
    cols += [U[:, a] ** 2 for a in range(U.shape[1])]
    for a in range(U.shape[1]):
        for b in range(a + 1, U.shape[1]):
            cols.append(U[:, a] * U[:, b])
    return np.stack(cols, axis=1)


def subspace(d: Dict, digits: np.ndarray) -> np.ndarray:
    digits = np.atleast_2d(np.asarray(digits, dtype=np.int64))
    idx = np.zeros(digits.shape[0], dtype=np.int64)
    for j in d["binary"]:
        idx = idx * 2 + digits[:, j]
    return idx


def fit(values: List[List[int]], digits: np.ndarray, Y: np.ndarray) -> np.ndarray:
    """Coefficients [n_sub, K, T] (float64) by least squares per subspace."""
    d = design(values)
    X = terms(d, digits)
    Y = np.asarray(Y, dtype=np.float64).reshape(X.shape[0], -1)
    sub = subspace(d, digits)
    glob = np.linalg.lstsq(X, Y, rcond=None)[0].T if len(X) else np.zeros((Y.shape[1], d["T"]))
    C = np.empty((d["n_sub"], Y.shape[1], d["T"]))
    for g in range(d["n_sub"]):
        rows = sub == g
        C[g] = np.linalg.lstsq(X[rows], Y[rows], rcond=None)[0].T if rows.any() else glob
    return C


def predict(values: List[List[int]], coef: np.ndarray, digits: np.ndarray) -> np.ndarray:
    """Predicted counters [n, K] (float64): the subspace's coefficients times the terms."""
    d = design(values)
    X = terms(d, digits)
    C = np.asarray(coef, dtype=np.float64)[subspace(d, digits)]      # [n, K, T]
    return np.einsum("nkt,nt->nk", C, X)
