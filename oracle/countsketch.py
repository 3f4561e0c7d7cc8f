"""CountSketch variant of the sketch (the sparse projection of Sec. 2, used in place of the
SRHT in the SLSE-FRS-CS experiment of Sec. 5), in FP64.

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__.py``).

Definition (Sec. 2, CountSketch): S in R^{m x N} has independent columns, and column k
holds a single non-zero entry, a random sign, in a uniformly random row.  S X then
costs O(N d): row k of X is added, with its sign, to row h(k) of S X.  Because every
column of S has unit norm and distinct columns are orthogonal in expectation,
E[S^T S] = I_N, so no scale factor is applied (unlike the sqrt(N/m) of the SRHT).

Readings taken where the paper is silent:
* Rows are not padded: k ranges over [0, N).
* Hash and sign of row k from Philox4x32-10 (``oracle.philox``) stream 3, counter k:
  h(k) = w0 (a uniform 32-bit word), s(k) = -1 if bit 0 of w1 is set, else +1.
* Nested sketches: a sketch with m rows (m a power of two) puts row k in bucket
  h(k) mod m.  Sketch sizes m_1 < ... < m_K that double share the same h, so
  S_i = F_i S_K where F_i adds the rows of S_K X that agree modulo m_i ("folding"):
  every S_i is itself a CountSketch, and one pass over X serves all of them.
* Hessian sketch S-hat (r rows, any r): an independent hash from stream 4:
  h-hat(k) = floor(w0 * r / 2^32) (multiply-shift onto [0, r)), s-hat(k) from bit 0 of w1.
"""
import numpy as np

from .philox import stream_words

STREAM_CS, STREAM_CS_HAT = 3, 4


def is_pow2(m: int) -> bool:
    return m >= 1 and (m & (m - 1)) == 0


def cs_hash(N: int, seed: int):
    """(h, s): 32-bit hash words (uint64 array) and signs (float64 +-1) of rows 0..N-1."""
    w0, w1, _, _ = stream_words(seed, STREAM_CS, N)
    return w0, np.where((w1 & np.uint64(1)) == 1, -1.0, 1.0)


def cs_buckets(h: np.ndarray, m: int) -> np.ndarray:
    """Bucket of every row in the m-row sketch of the nested family: h mod m (m = 2^l)."""
    if not is_pow2(m):
        raise ValueError("CountSketch sizes of the nested family are powers of two")
    return (h & np.uint64(m - 1)).astype(np.int64)


def hat_hash(N: int, seed: int, r: int):
    """(b, s): bucket in [0, r) and sign of every row for the Hessian sketch S-hat."""
    w0, w1, _, _ = stream_words(seed, STREAM_CS_HAT, N)
    b = ((w0 * np.uint64(r)) >> np.uint64(32)).astype(np.int64)
    return b, np.where((w1 & np.uint64(1)) == 1, -1.0, 1.0)


def _scatter_add(A, b, s, m, block_rows=1 << 16):
    """out[b_k] += s_k A[k] for every row k (row blocks keep the FP64 copy of A small)."""
    A = np.asarray(A)
    out = np.zeros((m,) + A.shape[1:])
    for lo in range(0, A.shape[0], block_rows):
        blk = np.asarray(A[lo:lo + block_rows], np.float64)
        sb = s[lo:lo + block_rows]
        np.add.at(out, b[lo:lo + block_rows], blk * (sb[:, None] if blk.ndim == 2 else sb))
    return out


def countsketch(X, Y, m: int, seed: int):
    """(S X, S Y) for the m-row sketch of the nested family (bucket order 0..m-1)."""
    N = np.asarray(X).shape[0]
    h, s = cs_hash(N, seed)
    b = cs_buckets(h, m)
    return _scatter_add(X, b, s, m), _scatter_add(Y, b, s, m)


def countsketch_hat(X, Y, r: int, seed: int):
    """(S-hat X, S-hat Y) for the r-row Hessian sketch."""
    N = np.asarray(X).shape[0]
    b, s = hat_hash(N, seed, r)
    return _scatter_add(X, b, s, r), _scatter_add(Y, b, s, r)


def countsketch_matrix_dense(N: int, m: int, seed: int) -> np.ndarray:
    """The m x N matrix S of the definition: S[h(k) mod m, k] = s(k), zero elsewhere."""
    h, s = cs_hash(N, seed)
    S = np.zeros((m, N))
    S[cs_buckets(h, m), np.arange(N)] = s
    return S


def countsketch_hat_matrix_dense(N: int, r: int, seed: int) -> np.ndarray:
    b, s = hat_hash(N, seed, r)
    S = np.zeros((r, N))
    S[b, np.arange(N)] = s
    return S


def fold(SX: np.ndarray, m: int) -> np.ndarray:
    """F S X: the m-row sketch from a larger one of the same family (m divides its rows):
    row b is the sum of the rows b, b + m, b + 2m, ...; rows are added in that order."""
    M = SX.shape[0]
    if M % m:
        raise ValueError("m must divide the number of rows")
    out = np.zeros((m,) + SX.shape[1:])
    for q in range(M // m):
        out += SX[q * m:(q + 1) * m]
    return out
