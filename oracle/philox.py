"""Counter-based normal deviates for the band-power simulations, CPU side.

TEST INFRASTRUCTURE ONLY (same rule as wf_oracle.py: only the tests, the smoke
check and the benchmark's CPU legs use it).  The GPU library draws the same
numbers with its own implementation; the two share nothing but the published
definitions below.

Generator: Philox4x32-10 of Salmon, Moraes, Dror and Shaw, "Parallel random
numbers: as easy as 1, 2, 3", SC'11 (2011).  A round maps the counter
(c0, c1, c2, c3) with key (k0, k1) to
    (hi(M1 c2) ^ c1 ^ k0,  lo(M1 c2),  hi(M0 c0) ^ c3 ^ k1,  lo(M0 c0)),
M0 = 0xD2511F53, M1 = 0xCD9E8D57 (32 x 32 -> 64-bit products); between rounds
the key is bumped by the Weyl constants (0x9E3779B9, 0xBB67AE85); ten rounds.

Normal deviates (the library's convention, stated here and in include/wf.h):
for seed S, stream t and deviate index i, the block j = i // 2 is
x = Philox(counter = (j mod 2^32, j div 2^32, t, 0), key = (S mod 2^32, S div 2^32)),
two uniforms u1 = (2^26 (x0 >> 5) + (x1 >> 6) + 1/2) 2^-53 and
u2 = (2^26 (x2 >> 5) + (x3 >> 6) + 1/2) 2^-53 in (0, 1), and the Box-Muller pair
(r cos 2 pi u2, r sin 2 pi u2), r = sqrt(-2 ln u1) (Box & Muller, Ann. Math.
Stat. 29, 1958): deviate 2j is the cosine, 2j + 1 the sine.
"""
from __future__ import annotations

import numpy as np

M0, M1 = 0xD2511F53, 0xCD9E8D57
W0, W1 = 0x9E3779B9, 0xBB67AE85
MASK32 = 0xFFFFFFFF


def _mulhilo(a: int, b: np.ndarray):
    p = np.uint64(a) * b.astype(np.uint64)
    return (p >> np.uint64(32)).astype(np.uint64), (p & np.uint64(MASK32)).astype(np.uint64)


def philox4x32_10(ctr, key):
    """Philox4x32 with ten rounds.  ctr: four arrays (or ints) of 32-bit words,
    key: two ints.  Returns the four output words as uint64 arrays."""
    c = [np.asarray(v, dtype=np.uint64) & np.uint64(MASK32) for v in ctr]
    k0, k1 = int(key[0]) & MASK32, int(key[1]) & MASK32
    for r in range(10):
        if r > 0:
            k0 = (k0 + W0) & MASK32
            k1 = (k1 + W1) & MASK32
        hi0, lo0 = _mulhilo(M0, c[0])
        hi1, lo1 = _mulhilo(M1, c[2])
        c = [hi1 ^ c[1] ^ np.uint64(k0), lo1, hi0 ^ c[3] ^ np.uint64(k1), lo0]
    return c


def normals(seed: int, stream: int, count: int, offset: int = 0) -> np.ndarray:
    """Deviates offset .. offset + count - 1 of (seed, stream), FP64."""
    if count <= 0:
        return np.zeros(0)
    i = np.arange(offset, offset + count, dtype=np.uint64)
    j = i >> np.uint64(1)
    x = philox4x32_10((j & np.uint64(MASK32), j >> np.uint64(32), np.full_like(j, stream), np.zeros_like(j)),
                      (seed & MASK32, (seed >> 32) & MASK32))
    two53 = 2.0 ** -53
    u1 = ((x[0] >> np.uint64(5)).astype(np.float64) * 67108864.0 + (x[1] >> np.uint64(6)).astype(np.float64)
          + 0.5) * two53
    u2 = ((x[2] >> np.uint64(5)).astype(np.float64) * 67108864.0 + (x[3] >> np.uint64(6)).astype(np.float64)
          + 0.5) * two53
    r = np.sqrt(-2.0 * np.log(u1))
    th = 2.0 * np.pi * u2
    return np.where((i & np.uint64(1)) == 0, r * np.cos(th), r * np.sin(th))


# Streams of bandpower_estimate's own draws.
STREAM_Z, STREAM_NOISE, STREAM_U = 0, 1, 2
