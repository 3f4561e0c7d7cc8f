"""SRHT sketch of the tall data [X | Y], written from Sec. 3 of the paper.

Sec. 3 (SRHT definition): for N = 2^p, S = sqrt(N/m) B H D P, with P a uniformly
random permutation matrix, D a diagonal of i.i.d. Rademacher signs, H the
normalised Hadamard matrix and B a row sampler; the non-zero rows of S are kept.
Sec. 3 (construction of the nested sketches, Algorithm 2): the full transform
(S_0 X, S_0 Y) = (H D P X, H D P Y) is formed once, and the i-th sketch keeps m_i
of its rows, scaled by sqrt(N/m_i); the rows of S_i are a subset of those of
S_{i+1}.

Readings taken where the paper leaves freedom:
* N is padded with zero rows to N' = 2^ceil(log2 N); all scales use N'.
* H is the Sylvester (natural-order) matrix H[k, j] = (-1)^popcount(k & j), and
  the 1/sqrt(N') normalisation is applied once, after the transform.
* B keeps exactly m_i rows: the first m_i entries of a second uniform random
  permutation sigma of [0, N').  The nested property holds by construction.
* The Hessian sketch S-hat uses the disjoint rows sigma[m_K : m_K + r]; if
  m_K + r > N' it falls back to sigma[0 : r].
* Random draws, from ``oracle.philox`` with key = seed:
    stream 0 -> D_j = -1 if bit 0 of word 0 is set, else +1;
    stream 1 -> P   = stable argsort of the 64-bit keys (w1 << 32) | w0;
    stream 2 -> sigma, the same construction.
  Stable argsort breaks (vanishingly rare) key ties by the smaller index.
"""
import math

import numpy as np

from .philox import stream_words

STREAM_D, STREAM_P, STREAM_SIGMA = 0, 1, 2


def padded_size(N: int) -> int:
    """N' = 2^ceil(log2 N) (N >= 1)."""
    return 1 << max(0, int(N - 1).bit_length())


def rademacher(Np: int, seed: int) -> np.ndarray:
    w0, _, _, _ = stream_words(seed, STREAM_D, Np)
    return np.where((w0 & np.uint64(1)) == 1, -1.0, 1.0)


def uniform_permutation(Np: int, seed: int, stream: int) -> np.ndarray:
    w0, w1, _, _ = stream_words(seed, stream, Np)
    keys = (w1 << np.uint64(32)) | w0
    return np.argsort(keys, kind="stable").astype(np.int64)


def draws(Np: int, seed: int):
    """(D, P, sigma) for a padded size Np: signs (float64 +-1), permutation, sampling order."""
    return (rademacher(Np, seed), uniform_permutation(Np, seed, STREAM_P),
            uniform_permutation(Np, seed, STREAM_SIGMA))


def fwht(A: np.ndarray) -> np.ndarray:
    """Unnormalised Walsh-Hadamard transform along axis 0 in Sylvester order:
    out[k] = sum_j (-1)^popcount(k & j) A[j].  In-place butterfly on a copy; one
    level per bit of the row index (the recursive structure of H noted in Sec. 1.1)."""
    out = np.array(A, dtype=np.float64, copy=True)
    n = out.shape[0]
    assert n & (n - 1) == 0, "length must be a power of two"
    tail = out.shape[1:]
    h = 1
    while h < n:
        v = out.reshape((n // (2 * h), 2, h) + tail)
        a = v[:, 0].copy()
        b = v[:, 1]
        v[:, 0] = a + b
        v[:, 1] = a - b
        h *= 2
    return out


def hadamard_dense(n: int) -> np.ndarray:
    """Dense H[k, j] = (-1)^popcount(k & j) (unnormalised), for brute-force checks."""
    k = np.arange(n)[:, None]
    j = np.arange(n)[None, :]
    pc = np.vectorize(lambda v: bin(int(v)).count("1"))(k & j)
    return np.where(pc % 2 == 0, 1.0, -1.0)


def hdp(X: np.ndarray, D: np.ndarray, P: np.ndarray) -> np.ndarray:
    """Z = H D P X_pad / sqrt(N'): the full transformed data S_0 X of Sec. 3.
    Row j of P X_pad is X_pad[P[j]] (zero when P[j] >= N)."""
    Np = D.shape[0]
    X = np.asarray(X, dtype=np.float64)
    squeeze = X.ndim == 1
    if squeeze:
        X = X[:, None]
    N = X.shape[0]
    Xt = np.zeros((Np, X.shape[1]))
    live = P < N
    Xt[live] = X[P[live]]
    Xt *= D[:, None]
    Z = fwht(Xt) * (1.0 / math.sqrt(Np))
    return Z[:, 0] if squeeze else Z


def hessian_rows(Np: int, m_K: int, r: int):
    """Positions in sigma used for the Hessian sketch: sigma[m_K : m_K + r], or
    sigma[0 : r] when the disjoint block does not fit."""
    if m_K + r <= Np:
        return m_K, m_K + r
    return 0, r


def sketch(X, Y, m: int, seed: int):
    """(S X, S Y) for one sketch of size m: sqrt(N'/m) * rows sigma[0:m] of H D P [X|Y]/sqrt(N')."""
    N = np.shape(X)[0]
    Np = padded_size(N)
    D, P, sigma = draws(Np, seed)
    ZX = hdp(X, D, P)
    ZY = hdp(Y, D, P)
    s = math.sqrt(Np / m)
    return s * ZX[sigma[:m]], s * ZY[sigma[:m]]


def sketch_matrix_dense(N: int, m: int, seed: int) -> np.ndarray:
    """The m x N sketch matrix S = sqrt(N'/m) B H D P restricted to the N real
    columns, built entry by entry from the definition (brute force, N' <= 256)."""
    Np = padded_size(N)
    D, P, sigma = draws(Np, seed)
    H = hadamard_dense(Np) / math.sqrt(Np)
    Pm = np.zeros((Np, Np))
    Pm[np.arange(Np), P] = 1.0               # (P x)[j] = x[P[j]]
    B = np.zeros((m, Np))
    B[np.arange(m), sigma[:m]] = 1.0
    S = math.sqrt(Np / m) * B @ H @ np.diag(D) @ Pm
    return S[:, :N]


def sketch_entries(X, Y, D, P, sigma, m: int, rows, cols) -> np.ndarray:
    """Single entries of the sketch S [X | Y] computed one by one from the definition of Sec. 3
    (for sampled checks at sizes where the full transform is too large): entry (s, c) is
    sqrt(N'/m) * (H D P [X | Y]_pad)[sigma[s], c] / sqrt(N') = sum_j (-1)^popcount(k & j) D_j
    [X | Y][P_j, c] / sqrt(m) with k = sigma[s], over the j with P_j < N (the padding rows are
    zero).  Column c = d is Y.  Returns a len(rows) x len(cols) array."""
    X = np.asarray(X)
    N, d = X.shape
    Np = D.shape[0]
    j = np.arange(Np, dtype=np.int64)
    live = P < N
    src = P[live]
    cols_data = [np.asarray(Y if c == d else X[:, c], np.float64)[src] for c in cols]
    out = np.empty((len(rows), len(cols)))
    for a, s in enumerate(rows):
        k = int(sigma[s])
        sgn = np.where(np.bitwise_count(j & k) % 2 == 0, 1.0, -1.0) * D
        w = sgn[live]
        for b, col in enumerate(cols_data):
            out[a, b] = float(np.dot(w, col)) / math.sqrt(m)
    return out
