"""FP8 (E4M3) block-scaled storage of a sketch, in FP64 arithmetic.

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__.py``).

The paper stores its sketches in double precision; the FP8 form is an extension (a
lower-precision sketch for the 1st-stage subproblems, whose exact values matter only
through the subspace embedding).  Definitions written from the OCP 8-bit floating-point
and microscaling (MX) specifications:

* E4M3: sign, 4 exponent bits (bias 7), 3 mantissa bits; no infinities; the all-ones
  exponent with mantissa 111 is NaN, so the largest finite value is 1.75 * 2^8 = 448.
  Normal values 1.m * 2^(e-7) for e = 1..15, subnormal values m/8 * 2^-6 (e = 0).
  Conversion rounds to nearest, ties to even, and saturates at +-448.
* Block scaling: each run of 32 consecutive elements of a row shares one power-of-two
  scale 2^k (an E8M0 byte, k in [-127, 127]).  Reading taken here: k is the smallest
  integer with amax <= 448 * 2^k (amax = largest magnitude in the block), so no element
  saturates; an all-zero block uses k = -127.  Stored value q = E4M3(x / 2^k); the
  element reads back as q * 2^k.
"""
import math

import numpy as np

E4M3_MAX = 448.0
BLOCK = 32


def e4m3_values() -> np.ndarray:
    """The 253 distinct finite E4M3 values (both signs), from the bit-field definition."""
    vals = []
    for code in range(256):
        s = -1.0 if code & 0x80 else 1.0
        e = (code >> 3) & 0xF
        m = code & 0x7
        if e == 0xF and m == 0x7:
            continue  # NaN
        if e == 0:
            v = m / 8.0 * 2.0 ** -6
        else:
            v = (1.0 + m / 8.0) * 2.0 ** (e - 7)
        vals.append(s * v)
    return np.array(sorted(set(vals)))


_GRID = e4m3_values()
_POS = _GRID[_GRID >= 0]


def round_e4m3(x) -> np.ndarray:
    """Round to the nearest E4M3 value, ties to the even mantissa, saturating at +-448."""
    x = np.asarray(x, np.float64)
    a = np.minimum(np.abs(x), E4M3_MAX)
    i = np.searchsorted(_POS, a)            # _POS[i-1] < a <= _POS[i]
    i = np.clip(i, 1, len(_POS) - 1)
    lo, hi = _POS[i - 1], _POS[i]
    below = a - lo
    above = hi - a
    # ties: the even code; positive values are consecutive codes 0..126, code index = i
    even_hi = (i % 2) == 0
    pick_hi = (above < below) | ((above == below) & even_hi)
    r = np.where(a <= lo, lo, np.where(pick_hi, hi, lo))
    r = np.where(a == 0, 0.0, r)
    return np.copysign(r, x)


def block_exponent(amax: float) -> int:
    """Smallest k with amax <= 448 * 2^k, clamped to the E8M0 range; -127 for amax = 0."""
    if amax == 0.0:
        return -127
    m, e = math.frexp(amax / E4M3_MAX)      # amax/448 = m 2^e, m in [0.5, 1)
    k = e if m > 0.5 else e - 1
    return max(-127, min(127, k))


def quantize_rows(A) -> tuple:
    """(Q, K): E4M3 values of A / 2^k per 32-column block of each row, and the exponents k
    (rows x ceil(cols/32))."""
    A = np.asarray(A, np.float64)
    rows, cols = A.shape
    nb = (cols + BLOCK - 1) // BLOCK
    Q = np.zeros_like(A)
    K = np.zeros((rows, nb), np.int64)
    for b in range(nb):
        blk = A[:, b * BLOCK:(b + 1) * BLOCK]
        amax = np.abs(blk).max(axis=1)
        k = np.array([block_exponent(float(v)) for v in amax])
        K[:, b] = k
        Q[:, b * BLOCK:(b + 1) * BLOCK] = round_e4m3(blk / np.ldexp(1.0, k)[:, None])
    return Q, K


def dequantize_rows(Q, K) -> np.ndarray:
    Q = np.asarray(Q, np.float64)
    out = np.empty_like(Q)
    for b in range(K.shape[1]):
        out[:, b * BLOCK:(b + 1) * BLOCK] = Q[:, b * BLOCK:(b + 1) * BLOCK] * np.ldexp(1.0, K[:, b])[:, None]
    return out


def decode_e4m3(codes) -> np.ndarray:
    """Values of E4M3 codes (uint8), from the bit-field definition (NaN codes -> nan)."""
    table = np.empty(256)
    for code in range(256):
        s = -1.0 if code & 0x80 else 1.0
        e = (code >> 3) & 0xF
        m = code & 0x7
        if e == 0xF and m == 0x7:
            table[code] = np.nan
        elif e == 0:
            table[code] = s * m / 8.0 * 2.0 ** -6
        else:
            table[code] = s * (1.0 + m / 8.0) * 2.0 ** (e - 7)
    return table[np.asarray(codes, np.int64)]
