"""Philox4x32-10 counter-based generator, from its published definition
(J. K. Salmon, M. A. Moraes, R. O. Dror, D. E. Shaw, "Parallel random numbers:
as easy as 1, 2, 3", SC'11, Sec. 4.2 and Table 2).

State: a 128-bit counter (c0, c1, c2, c3) and a 64-bit key (k0, k1).  One round:
    (hi0, lo0) = mulhilo32(0xD2511F53, c0)
    (hi1, lo1) = mulhilo32(0xCD9E8D57, c2)
    c' = (hi1 ^ c1 ^ k0, lo1, hi0 ^ c3 ^ k1, lo0)
then the key is bumped by the Weyl constants (0x9E3779B9, 0xBB67AE85).
Ten rounds, the first with the unbumped key.

The paper does not name its generator (its experiments used MATLAB); the draws
the sketch needs (Sec. 3, the matrices D, P and B) are defined on top of this
generator in ``oracle.sketch``.  Vectorised over counters with numpy uint64
arithmetic; all values are exact integers.
"""
import numpy as np

M0 = np.uint64(0xD2511F53)
M1 = np.uint64(0xCD9E8D57)
W0 = np.uint64(0x9E3779B9)
W1 = np.uint64(0xBB67AE85)
MASK = np.uint64(0xFFFFFFFF)
S32 = np.uint64(32)


def philox4x32_10(c0, c1, c2, c3, k0, k1):
    """Return the four 32-bit output words (as uint64 arrays holding values < 2^32)."""
    c0, c1, c2, c3 = (np.asarray(c, dtype=np.uint64) & MASK for c in (c0, c1, c2, c3))
    k0 = np.uint64(int(k0) & 0xFFFFFFFF)
    k1 = np.uint64(int(k1) & 0xFFFFFFFF)
    for rnd in range(10):
        if rnd > 0:
            k0 = (k0 + W0) & MASK
            k1 = (k1 + W1) & MASK
        p0 = M0 * c0          # < 2^64: exact in uint64
        p1 = M1 * c2
        hi0, lo0 = p0 >> S32, p0 & MASK
        hi1, lo1 = p1 >> S32, p1 & MASK
        c0, c1, c2, c3 = hi1 ^ c1 ^ k0, lo1, hi0 ^ c3 ^ k1, lo0
    return c0, c1, c2, c3


def stream_words(seed: int, stream: int, n: int):
    """Output words for counters i = 0..n-1 of one stream.

    Counter layout: (i mod 2^32, i div 2^32, stream, 0); key: (seed mod 2^32,
    seed div 2^32).  Returns (w0, w1, w2, w3) uint64 arrays of length n.
    """
    i = np.arange(n, dtype=np.uint64)
    seed = int(seed) & 0xFFFFFFFFFFFFFFFF
    return philox4x32_10(i & MASK, i >> S32, np.full(n, stream, np.uint64), np.zeros(n, np.uint64),
                         seed & 0xFFFFFFFF, seed >> 32)
