"""Philox4x32-10 counter-based generator (Salmon, Moraes, Dror, Shaw, SC'11, "Parallel random
numbers: as easy as 1, 2, 3") and the sketch entry draws of Sec. 3.2.

Sec. 3.2 considers Gaussian entries ("N(mu=0, sigma=1/S)") and Rademacher entries (+-1 with
p = 0.5).  Reading adopted (unit-variance normalisation, the default): Gaussian entries with
variance 1/S and Rademacher entries +-1/sqrt(S), so that E[S~_S^T S~_S] = I; at the paper's
chosen S = 1 this equals its literal values.  The literal reading (Gaussian with standard
deviation 1/S, Rademacher +-1) is the second normalisation option.

Entry e = s*(C-V) + j (row-major in S~_S of outer iteration t) uses counter (e, t, 0, 0) and
key (seed mod 2^32, seed >> 32).  Of the four output words o0..o3:
  u1 = ((o0 >> 8) + 0.5) 2^-24,  u2 = ((o1 >> 8) + 0.5) 2^-24,
  Gaussian   = sqrt(-2 ln u1) cos(2 pi u2) (Box-Muller, float64),
  Rademacher = +1 if (o2 >> 31) == 0 else -1,
then scaled, rounded to float32 and finally to the nearest bfloat16 value (ties to even) so
the entries are exact tensor-core operands.
"""
from __future__ import annotations

import numpy as np

M0 = 0xD2511F53
M1 = 0xCD9E8D57
W0 = 0x9E3779B9
W1 = 0xBB67AE85
MASK = 0xFFFFFFFF

GAUSSIAN = 0
RADEMACHER = 1
NORM_UNIT_VAR = 0
NORM_PAPER_LITERAL = 1


def philox4x32_10(ctr, key):
    """One Philox4x32 block with 10 rounds. ctr: 4 ints, key: 2 ints -> 4 ints."""
    c0, c1, c2, c3 = [int(v) & MASK for v in ctr]
    k0, k1 = [int(v) & MASK for v in key]
    for r in range(10):
        if r:
            k0 = (k0 + W0) & MASK
            k1 = (k1 + W1) & MASK
        p0 = M0 * c0
        p1 = M1 * c2
        hi0, lo0 = p0 >> 32, p0 & MASK
        hi1, lo1 = p1 >> 32, p1 & MASK
        c0, c1, c2, c3 = (hi1 ^ c1 ^ k0) & MASK, lo1, (hi0 ^ c3 ^ k1) & MASK, lo0
    return c0, c1, c2, c3


def round_to_bf16(x):
    """Round float32 values to the nearest bfloat16 (ties to even), returned as float32."""
    f = np.asarray(x, dtype=np.float32).copy()
    b = f.view(np.uint32).astype(np.uint64)
    lsb = (b >> 16) & 1
    b = (b + 0x7FFF + lsb) & 0xFFFF0000
    return b.astype(np.uint32).view(np.float32)


def sketch_draw(seed, t0, T, C, V, S, dist=GAUSSIAN, norm=NORM_UNIT_VAR):
    """Random blocks S~_S^t for t = t0 .. t0+T-1, float32 [T, S, C-V]."""
    K = C - V
    out = np.zeros((T, S, K), dtype=np.float32)
    key = (seed & MASK, (seed >> 32) & MASK)
    if dist == GAUSSIAN:
        scale = (1.0 / np.sqrt(S)) if norm == NORM_UNIT_VAR else (1.0 / S)
    else:
        scale = (1.0 / np.sqrt(S)) if norm == NORM_UNIT_VAR else 1.0
    for ti in range(T):
        t = t0 + ti
        for e in range(S * K):
            o = philox4x32_10((e, t, 0, 0), key)
            if dist == GAUSSIAN:
                u1 = ((o[0] >> 8) + 0.5) * 2.0 ** -24
                u2 = ((o[1] >> 8) + 0.5) * 2.0 ** -24
                v = np.sqrt(-2.0 * np.log(u1)) * np.cos(2.0 * np.pi * u2)
            else:
                v = 1.0 if (o[2] >> 31) == 0 else -1.0
            out[ti, e // K, e % K] = np.float32(v * scale)
    return round_to_bf16(out)
