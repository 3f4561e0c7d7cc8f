"""Gradients through the least-squares estimate, in FP64 (dense formulas).

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__.py``).

SLSE-FRS converges to the OLS estimate beta-hat = (X^T X)^{-1} X^T Y (Sec. 1 problem
statement; the 2nd stage's fixed point solves the normal equations, Sec. 3).  For a loss
L(beta-hat) with v = dL/d(beta-hat), differentiating X^T X beta-hat = X^T Y gives

    X^T X d(beta-hat) = dX^T (Y - X beta-hat) - X^T dX beta-hat + X^T dY,

so with w = (X^T X)^{-1} v and r = Y - X beta-hat:

    dL/dY = X w,        dL/dX = r w^T - (X w) beta-hat^T.

The paper does not differentiate its estimator; this is an extension for training through
it, checked here against finite differences of ``linalg.ols``.
"""
import numpy as np

from .linalg import ols


def normal_solve(X, v):
    """w = (X^T X)^{-1} v by a Cholesky factorisation of the FP64 Gram matrix."""
    X = np.asarray(X, np.float64)
    G = X.T @ X
    L = np.linalg.cholesky(G)
    return np.linalg.solve(L.T, np.linalg.solve(L, np.asarray(v, np.float64)))


def ols_vjp(X, Y, beta_hat, v):
    """(w, dL/dX, dL/dY) for the loss gradient v = dL/d(beta-hat)."""
    X = np.asarray(X, np.float64)
    Y = np.asarray(Y, np.float64)
    w = normal_solve(X, v)
    Xw = X @ w
    r = Y - X @ beta_hat
    return w, np.outer(r, w) - np.outer(Xw, beta_hat), Xw


def loss_to_truth(beta_hat, beta_star):
    """L = 1/2 ||beta-hat - beta*||^2 and its gradient v = beta-hat - beta*."""
    e = np.asarray(beta_hat, np.float64) - np.asarray(beta_star, np.float64)
    return 0.5 * float(e @ e), e


def fd_gradients(X, Y, beta_star, entries_x, entries_y, h=1e-6):
    """Central differences of L(ols(X, Y)) for chosen entries of X ((i, j) pairs) and Y."""
    X = np.array(X, np.float64, copy=True)
    Y = np.array(Y, np.float64, copy=True)

    def L(Xa, Ya):
        return loss_to_truth(ols(Xa, Ya), beta_star)[0]

    gx = []
    for i, j in entries_x:
        x0 = X[i, j]
        X[i, j] = x0 + h
        lp = L(X, Y)
        X[i, j] = x0 - h
        lm = L(X, Y)
        X[i, j] = x0
        gx.append((lp - lm) / (2 * h))
    gy = []
    for i in entries_y:
        y0 = Y[i]
        Y[i] = y0 + h
        lp = L(X, Y)
        Y[i] = y0 - h
        lm = L(X, Y)
        Y[i] = y0
        gy.append((lp - lm) / (2 * h))
    return np.array(gx), np.array(gy)
