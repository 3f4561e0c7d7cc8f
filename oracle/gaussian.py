"""Gaussian sketch (Sec. 2: a sketching matrix S in R^{m x N} with i.i.d. N(0, 1/m)
entries), used as the Hessian sketch S-hat of SLSE-FRS in place of the sampled SRHT
rows (Sec. 2 lists it among the classical sketches; forming S X costs O(m N d)).
Test infrastructure: only the tests, the smoke check and the benchmark's CPU legs use it.

Definition of the draws (the paper does not say how its Gaussian entries are made):
S = G / sqrt(m) with G[i, k] ~ N(0, 1) taken from Philox4x32-10 (``oracle.philox``) at
counter (q mod 2^32, q div 2^32, 5, i), q = k div 8, key = seed: one call gives the
eight entries G[i, 8q .. 8q + 7].  Output word j (0..3) feeds the Box-Muller transform
(G. E. P. Box and M. E. Muller, Ann. Math. Statist. 29 (1958) 610-611) with two 16-bit
uniforms, u1 = (w mod 2^16 + 1/2) / 2^16 and u2 = (w div 2^16 + 1/2) / 2^16:
    G[i, 8q + 2j]     = sqrt(-2 ln u1) cos(2 pi u2)
    G[i, 8q + 2j + 1] = sqrt(-2 ln u1) sin(2 pi u2).
The 16-bit uniforms make G a discretised normal with |G| <= sqrt(34 ln 2) = 4.85
(P(|N(0,1)| > 4.85) = 1.2e-6); entries used in BF16 carry only 8 significant bits.
Rows beyond N of a padded problem are never touched: S X only reads the N rows of X.
"""
import math

import numpy as np

from .philox import MASK, S32, philox4x32_10

STREAM_G = 5


def normals_from_words(w):
    """Box-Muller pair of each 32-bit word: returns (even, odd) float64 arrays."""
    w = np.asarray(w, np.uint64)
    u1 = ((w & np.uint64(0xFFFF)).astype(np.float64) + 0.5) / 65536.0
    u2 = ((w >> np.uint64(16)).astype(np.float64) + 0.5) / 65536.0
    rad = np.sqrt(-2.0 * np.log(u1))
    ang = 2.0 * math.pi * u2
    return rad * np.cos(ang), rad * np.sin(ang)


def gaussian_rows(seed: int, i0: int, i1: int, N: int) -> np.ndarray:
    """G[i0:i1, 0:N] (unscaled standard normals), float64."""
    seed = int(seed) & 0xFFFFFFFFFFFFFFFF
    nq = (N + 7) // 8
    q = np.arange(nq, dtype=np.uint64)
    rows = np.arange(i0, i1, dtype=np.uint64)
    c0 = np.broadcast_to(q & MASK, (i1 - i0, nq))
    c1 = np.broadcast_to(q >> S32, (i1 - i0, nq))
    c2 = np.full((i1 - i0, nq), STREAM_G, np.uint64)
    c3 = np.broadcast_to(rows[:, None], (i1 - i0, nq))
    words = philox4x32_10(c0, c1, c2, c3, seed & 0xFFFFFFFF, seed >> 32)
    G = np.empty((i1 - i0, nq, 8))
    for j, w in enumerate(words):
        G[:, :, 2 * j], G[:, :, 2 * j + 1] = normals_from_words(w)
    return G.reshape(i1 - i0, 8 * nq)[:, :N]


def gaussian_matrix_dense(N: int, m: int, seed: int) -> np.ndarray:
    """S = G / sqrt(m), m x N (small sizes only)."""
    return gaussian_rows(seed, 0, m, N) / math.sqrt(m)


def gaussian_sketch(X, Y, m: int, seed: int, block_rows: int = 64):
    """(S X, S Y) = (G X, G Y) / sqrt(m), G drawn in blocks of rows to bound memory."""
    X = np.asarray(X, np.float64)
    Y = np.asarray(Y, np.float64)
    N, d = X.shape
    SX = np.empty((m, d))
    SY = np.empty(m)
    for i0 in range(0, m, block_rows):
        i1 = min(m, i0 + block_rows)
        G = gaussian_rows(seed, i0, i1, N)
        SX[i0:i1] = G @ X
        SY[i0:i1] = G @ Y
    s = 1.0 / math.sqrt(m)
    return SX * s, SY * s
