"""Dense linear algebra for the oracle, in FP64.

* ``householder_r``: textbook Householder QR (Golub & Van Loan, Alg. 5.2.1), the
  factorisation the paper uses to apply the inverse sketched Hessian (Appendix,
  implementation details: H-hat^{-1} v = R^{-1} R^{-T} v from S-hat X = Q R).
  R is returned with a non-negative diagonal (rows of R multiplied by -1 where
  needed), which makes it unique for a full-column-rank input.
* ``ols``: the OLS estimator of Sec. 1, beta-hat = argmin 1/2 ||Y - X beta||^2,
  computed as R^{-1} (Q^T Y) from a Householder QR of [X | Y].  For tall inputs the
  QR is taken by row blocks and the stacked R factors are factorised again (TSQR);
  each block QR is LAPACK's Householder QR (numpy.linalg.qr, a library primitive).
* ``solve_upper`` / ``solve_lower``: plain substitution loops.
"""
import numpy as np


def householder_r(A: np.ndarray) -> np.ndarray:
    """R factor (min(r,d) x d, non-negative diagonal) of the r x d matrix A."""
    A = np.array(A, dtype=np.float64, copy=True)
    r, d = A.shape
    k = min(r, d)
    for j in range(k):
        x = A[j:, j]
        nrm = np.sqrt(np.dot(x, x))
        if nrm == 0.0:
            continue
        alpha = -nrm if x[0] >= 0.0 else nrm
        v = x.copy()
        v[0] -= alpha
        vtv = np.dot(v, v)
        w = v @ A[j:, j:]
        A[j:, j:] -= np.outer(v, (2.0 / vtv) * w)
    R = np.triu(A[:k, :])
    sgn = np.where(np.diag(R) < 0.0, -1.0, 1.0)
    return R * sgn[:, None]


def solve_upper(R: np.ndarray, b: np.ndarray) -> np.ndarray:
    """x with R x = b, R upper triangular (back substitution)."""
    d = R.shape[0]
    x = np.zeros(d)
    for i in range(d - 1, -1, -1):
        x[i] = (b[i] - np.dot(R[i, i + 1:], x[i + 1:])) / R[i, i]
    return x


def solve_lower(L: np.ndarray, b: np.ndarray) -> np.ndarray:
    """x with L x = b, L lower triangular (forward substitution)."""
    d = L.shape[0]
    x = np.zeros(d)
    for i in range(d):
        x[i] = (b[i] - np.dot(L[i, :i], x[:i])) / L[i, i]
    return x


def _qr_r_lapack(A: np.ndarray) -> np.ndarray:
    return np.linalg.qr(A, mode="r")


def ols(X: np.ndarray, Y: np.ndarray, block_rows: int = 1 << 16, textbook: bool = False) -> np.ndarray:
    """OLS beta-hat = (X^T X)^{-1} X^T Y (Sec. 1), via Householder QR of [X | Y].

    With QR [X|Y] = Q [[R, z], [0, rho]], beta-hat solves R beta = z.
    ``textbook=True`` uses ``householder_r`` on the whole matrix (small inputs).
    """
    N, d = X.shape
    if textbook:
        Rf = householder_r(np.column_stack([np.asarray(X, np.float64), np.asarray(Y, np.float64)]))
    else:
        Rs = []
        for lo in range(0, N, block_rows):
            hi = min(N, lo + block_rows)
            blk = np.empty((hi - lo, d + 1))
            blk[:, :d] = X[lo:hi]
            blk[:, d] = Y[lo:hi]
            if hi - lo >= d + 1:
                Rs.append(_qr_r_lapack(blk))
            else:
                Rs.append(blk)
        Rf = _qr_r_lapack(np.vstack(Rs)) if len(Rs) > 1 else Rs[0] if Rs[0].shape[0] == d + 1 else _qr_r_lapack(Rs[0])
    return solve_upper(Rf[:d, :d], Rf[:d, d])


def ols_normal(X: np.ndarray, Y: np.ndarray, block_rows: int = 1 << 16) -> np.ndarray:
    """beta-hat = (X^T X)^{-1} X^T Y written out (Sec. 1): the Gram matrix and X^T Y are
    accumulated in FP64 over row blocks (numpy matmul as the library primitive) and the
    d x d system is solved by Cholesky.  Its error grows like cond(X)^2 * u, so it serves
    only well-conditioned inputs (cond(X) ~ 3 for the AR(1) workload: ~1e-15); the QR
    route ``ols`` is the general oracle."""
    N, d = X.shape
    G = np.zeros((d, d))
    b = np.zeros(d)
    for lo in range(0, N, block_rows):
        Xb = np.asarray(X[lo:lo + block_rows], np.float64)
        G += Xb.T @ Xb
        b += Xb.T @ np.asarray(Y[lo:lo + block_rows], np.float64)
    L = np.linalg.cholesky(G)
    return solve_upper(L.T, solve_lower(L, b))


def ols_normal_longdouble(X: np.ndarray, Y: np.ndarray) -> np.ndarray:
    """Brute-force OLS from the normal equations X^T X beta = X^T Y, formed and solved
    by Gaussian elimination with partial pivoting in extended precision (np.longdouble).
    For small cross-checks only."""
    X = np.asarray(X, dtype=np.longdouble)
    Y = np.asarray(Y, dtype=np.longdouble)
    A = X.T @ X
    b = X.T @ Y
    d = A.shape[0]
    M = np.column_stack([A, b])
    for k in range(d):
        p = k + int(np.argmax(np.abs(M[k:, k])))
        if p != k:
            M[[k, p]] = M[[p, k]]
        for i in range(k + 1, d):
            M[i, k:] -= (M[i, k] / M[k, k]) * M[k, k:]
    x = np.zeros(d, dtype=np.longdouble)
    for i in range(d - 1, -1, -1):
        x[i] = (M[i, d] - np.dot(M[i, i + 1:d], x[i + 1:])) / M[i, i]
    return x.astype(np.float64)
