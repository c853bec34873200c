"""Counter-based random numbers for the method's own draws (oracle side).

Philox4x64-10 follows its published definition (Salmon, Moraes, Dror & Shaw,
"Parallel random numbers: as easy as 1, 2, 3", SC'11): a 4x64-bit counter, a
2x64-bit key, ten rounds of

    (hi0, lo0) = M0 * x0,  (hi1, lo1) = M1 * x2         (128-bit products)
    x <- (hi1 ^ x1 ^ k0, lo1, hi0 ^ x3 ^ k1, lo0)

with the key bumped by the Weyl constants (W0, W1) between rounds.

Draw layout (shared contract with the CUDA side, each side its own code):
counter = (p, block, stream, 0), key = (seed, 0), p = the caller's point index.

* Rademacher probe r[p, j]  (Section 3, Eq. def_SLQ with Rademacher vectors):
  block = j // 256, bit = j % 256 of the 256 output bits (word bit // 64,
  position bit % 64); r = 1 - 2 * bit_value.
* Gaussian z[p, j]  (Algorithm simAlgo): block = j // 4; output words
  (2q, 2q + 1) with q = (j % 4) // 2 give u1 = ((w >> 11) + 1) 2^-53 in (0, 1]
  and u2 = (w >> 11) 2^-53; Box-Muller: sqrt(-2 ln u1) * (cos, sin)(2 pi u2),
  cos for even j, sin for odd j.
"""
from __future__ import annotations

import numpy as np

M0 = 0xD2E7470EE14C6C93
M1 = 0xCA5A826395121157
W0 = 0x9E3779B97F4A7C15
W1 = 0xBB67AE8584CAA73B
_MASK = (1 << 64) - 1

STREAM_PROBE = 0      # SLQ probes (n part)
STREAM_SIM1 = 1       # simAlgo z1
STREAM_SIM2 = 2       # simAlgo z2
STREAM_PROBE_K = 3    # LRAC probes, rank-k part


def philox4x64_10_scalar(ctr, key):
    """Reference scalar Philox4x64-10 in Python integers."""
    x0, x1, x2, x3 = (int(c) & _MASK for c in ctr)
    k0, k1 = (int(k) & _MASK for k in key)
    for r in range(10):
        if r:
            k0 = (k0 + W0) & _MASK
            k1 = (k1 + W1) & _MASK
        p0 = M0 * x0
        p1 = M1 * x2
        x0, x1, x2, x3 = ((p1 >> 64) ^ x1 ^ k0, p1 & _MASK, (p0 >> 64) ^ x3 ^ k1, p0 & _MASK)
    return x0, x1, x2, x3


def _mulhilo64(a: int, x: np.ndarray):
    """128-bit product of the constant a and uint64 array x, from 32-bit halves."""
    m32 = np.uint64(0xFFFFFFFF)
    s32 = np.uint64(32)
    a_lo, a_hi = np.uint64(a & 0xFFFFFFFF), np.uint64(a >> 32)
    x_lo, x_hi = x & m32, x >> s32
    ll = a_lo * x_lo
    lh = a_lo * x_hi
    hl = a_hi * x_lo
    hh = a_hi * x_hi
    mid = (ll >> s32) + (lh & m32) + (hl & m32)
    hi = hh + (lh >> s32) + (hl >> s32) + (mid >> s32)
    lo = (ll & m32) | ((mid & m32) << s32)
    return hi, lo


def philox4x64_10(c0, c1, c2, c3, k0: int, k1: int):
    """Vectorised Philox4x64-10 over uint64 counter arrays (broadcastable)."""
    x0, x1, x2, x3 = (np.asarray(c, dtype=np.uint64) for c in (c0, c1, c2, c3))
    x0, x1, x2, x3 = np.broadcast_arrays(x0, x1, x2, x3)
    x0, x1, x2, x3 = (a.copy() for a in (x0, x1, x2, x3))
    ka, kb = k0 & _MASK, k1 & _MASK
    with np.errstate(over="ignore"):
        for r in range(10):
            if r:
                ka = (ka + W0) & _MASK
                kb = (kb + W1) & _MASK
            hi0, lo0 = _mulhilo64(M0, x0)
            hi1, lo1 = _mulhilo64(M1, x2)
            x0, x1, x2, x3 = hi1 ^ x1 ^ np.uint64(ka), lo1, hi0 ^ x3 ^ np.uint64(kb), lo0
    return x0, x1, x2, x3


def rademacher(points: np.ndarray, ncols: int, seed: int, stream: int = STREAM_PROBE) -> np.ndarray:
    """r[a, j] in {-1, +1} for the caller point indices ``points[a]``; float64."""
    points = np.asarray(points, dtype=np.uint64)
    out = np.empty((len(points), ncols))
    for blk in range((ncols + 255) // 256):
        w = philox4x64_10(points, np.uint64(blk), np.uint64(stream), np.uint64(0), seed, 0)
        for j in range(blk * 256, min(ncols, blk * 256 + 256)):
            bit = j - blk * 256
            v = (w[bit // 64] >> np.uint64(bit % 64)) & np.uint64(1)
            out[:, j] = 1.0 - 2.0 * v.astype(np.float64)
    return out


def gaussian(points: np.ndarray, ncols: int, seed: int, stream: int) -> np.ndarray:
    """z[a, j] ~ N(0, 1) by Box-Muller on Philox words; float64."""
    points = np.asarray(points, dtype=np.uint64)
    out = np.empty((len(points), ncols))
    two_m53 = 2.0 ** -53
    for blk in range((ncols + 3) // 4):
        w = philox4x64_10(points, np.uint64(blk), np.uint64(stream), np.uint64(0), seed, 0)
        for q in range(2):
            u1 = ((w[2 * q] >> np.uint64(11)).astype(np.float64) + 1.0) * two_m53
            u2 = (w[2 * q + 1] >> np.uint64(11)).astype(np.float64) * two_m53
            rad = np.sqrt(-2.0 * np.log(u1))
            ang = 2.0 * np.pi * u2
            for par, fn in ((0, np.cos), (1, np.sin)):
                j = blk * 4 + 2 * q + par
                if j < ncols:
                    out[:, j] = rad * fn(ang)
    return out
