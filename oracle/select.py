"""Score normalisation, weighted draws, top-k (oracle).

Section 3.5 Eq. "score_normalization", Section 3.6 and Algorithm 1.

Readings:
  * Normalisation covers the configurations not yet evaluated; s_min and s_max
    are taken over them.  s > 0 -> (1 + s/s_max)^8; gamma < s <= 0 ->
    max(1e-4, (1 - s/s_min)^8), with s = 0 giving 1 (also when s_min = 0);
    s <= gamma -> 1e-4; gamma = -0.25.  x^8 is ((x^2)^2)^2.  Computed in
    float32 (the kernels' precision), each operation rounded, no fusion.
  * The garbled sampling lines of Algorithm 1 are read as: draw r uniformly
    in [0, W), W = sum of weights, and take the first l whose inclusive prefix
    sum exceeds r.  To make prefix sums exact the weights are integers,
    w = round-half-even(s_norm * 2^20) (so w is in [105, 2^28]), and
    r = floor(u * W / 2^64) for a 64-bit uniform u.  Evaluated configurations
    have weight 0 (Algorithm 1), and a drawn one is set to 0 before the next
    draw (draws without replacement).
  * u comes from Philox4x32-10 (Salmon et al., SC'11) with key = (seed low
    32 bits, seed high 32 bits) and counter = (draw, step, search id, domain);
    u = x0 + 2^32 x1.  Domain 0 = the step's draws, domain 1 = the initial
    c_profile draw.
  * Top-k (the alternative select): the k highest raw scores, ties to the
    lower raw index.
Parity: Philox pinned by the published known-answer vectors; normalisation
by its end points; draws by a chi-square test against w / W.
"""
from __future__ import annotations

from typing import List, Tuple

import numpy as np

GAMMA = -0.25
W_SCALE = 1 << 20
M32 = 0xFFFFFFFF


def normalise_fp32(s, s_min, s_max, gamma: float = GAMMA) -> np.ndarray:
    s = np.asarray(s, dtype=np.float32)
    smin = np.float32(s_min); smax = np.float32(s_max)
    g = np.float32(gamma)
    one = np.float32(1.0); floor_ = np.float32(1e-4)
    out = np.empty_like(s)
    with np.errstate(divide="ignore", invalid="ignore"):
        for i, v in enumerate(s):
            if v > 0:
                x = one + v / smax
                x2 = x * x; x4 = x2 * x2; out[i] = x4 * x4
            elif v > g:
                if v == 0:
                    out[i] = one
                else:
                    y = one - v / smin
                    y2 = y * y; y4 = y2 * y2; y8 = y4 * y4
                    out[i] = max(floor_, y8)
            else:
                out[i] = floor_
    return out


def normalise_def(s, s_min, s_max, gamma: float = GAMMA) -> np.ndarray:
    """Float64 form of Eq. score_normalization (for checking the fp32 path)."""
    out = []
    for v in np.asarray(s, dtype=np.float64):
        if v > 0:
            out.append((1.0 + v / s_max) ** 8)
        elif v > gamma:
            out.append(1.0 if v == 0 else max(1e-4, (1.0 - v / s_min) ** 8))
        else:
            out.append(1e-4)
    return np.asarray(out)


def quantise(s_norm) -> np.ndarray:
    """w = round-half-even(s_norm * 2^20) as uint64."""
    x = np.asarray(s_norm, dtype=np.float32) * np.float32(W_SCALE)
    return np.rint(x).astype(np.uint64)


# -- Philox4x32-10 ------------------------------------------------------------
_M0, _M1 = 0xD2511F53, 0xCD9E8D57
_W0, _W1 = 0x9E3779B9, 0xBB67AE85


def philox4x32_10(ctr: Tuple[int, int, int, int], key: Tuple[int, int]) -> List[int]:
    """Ten rounds of the Philox 4x32 bijection; the key is bumped by the Weyl
    constants before every round after the first."""
    c0, c1, c2, c3 = (x & M32 for x in ctr)
    k0, k1 = key[0] & M32, key[1] & M32
    for rnd in range(10):
        if rnd:
            k0 = (k0 + _W0) & M32
            k1 = (k1 + _W1) & M32
        p0 = _M0 * c0
        p1 = _M1 * c2
        hi0, lo0 = p0 >> 32, p0 & M32
        hi1, lo1 = p1 >> 32, p1 & M32
        c0, c1, c2, c3 = hi1 ^ c1 ^ k0, lo1, hi0 ^ c3 ^ k1, lo0
    return [c0, c1, c2, c3]


def uniform_u64(seed: int, search_id: int, step: int, draw: int, domain: int) -> int:
    x = philox4x32_10((draw, step, search_id, domain), (seed & M32, (seed >> 32) & M32))
    return x[0] | (x[1] << 32)


def scaled_draw(u: int, total: int) -> int:
    """floor(u * total / 2^64), in [0, total)."""
    return (u * total) >> 64


def weighted_draws(w, k: int, seed: int, search_id: int, step: int) -> List[int]:
    """Up to k positions drawn without replacement with probability w / W,
    in draw order (Algorithm 1's inner loop)."""
    w = np.array(w, dtype=np.uint64)
    out = []
    for j in range(k):
        total = int(w.sum(dtype=np.uint64))
        if total == 0:
            break
        r = scaled_draw(uniform_u64(seed, search_id, step, j, 0), total)
        csum = np.cumsum(w, dtype=np.uint64)
        l = int(np.searchsorted(csum, np.uint64(r), side="right"))
        out.append(l)
        w[l] = 0
    return out


def topk(s, raw, k: int) -> List[int]:
    """Positions of the k highest scores, ties to the lower raw index."""
    s = np.asarray(s, dtype=np.float64)
    order = np.lexsort((np.asarray(raw), -s))
    return [int(i) for i in order[:k]]
