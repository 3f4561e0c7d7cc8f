"""Pins of the gradient formulas through the least-squares estimate (oracle/adjoint.py):
central finite differences of the oracle's OLS solve (N = 2000, d = 10, h = 1e-6), the
square-system closed form, and linearity/adjoint identities."""
import numpy as np
import pytest

from oracle import adjoint as adj
from oracle import linalg


def _problem(N, d, seed):
    rng = np.random.default_rng(seed)
    X = rng.standard_normal((N, d))
    beta_star = rng.standard_normal(d)
    Y = X @ beta_star + 0.05 * rng.standard_normal(N)
    return X, Y, beta_star


def test_formula_matches_central_differences():
    X, Y, bs = _problem(2000, 10, 0)
    bh = linalg.ols(X, Y)
    _, v = adj.loss_to_truth(bh, bs)
    _, dX, dY = adj.ols_vjp(X, Y, bh, v)
    rng = np.random.default_rng(1)
    ex = [(int(i), int(j)) for i, j in zip(rng.integers(0, 2000, 12), rng.integers(0, 10, 12))]
    ey = [int(i) for i in rng.integers(0, 2000, 12)]
    gx, gy = adj.fd_gradients(X, Y, bs, ex, ey, h=1e-6)
    ax = np.array([dX[i, j] for i, j in ex])
    ay = dY[ey]
    scale = np.abs(dX).max()
    assert np.all(np.abs(ax - gx) <= 1e-6 * scale + 1e-5 * np.abs(gx))
    assert np.all(np.abs(ay - gy) <= 1e-6 * np.abs(dY).max() + 1e-5 * np.abs(gy))


def test_square_system_closed_form():
    # X square and invertible: beta-hat = X^{-1} Y, r = 0, so dL/dY = X^{-T} v and
    # dL/dX = -X^{-T} v beta-hat^T
    rng = np.random.default_rng(2)
    X = rng.standard_normal((6, 6)) + 5 * np.eye(6)
    Y = rng.standard_normal(6)
    bh = np.linalg.solve(X, Y)
    v = rng.standard_normal(6)
    w, dX, dY = adj.ols_vjp(X, Y, bh, v)
    u = np.linalg.solve(X.T, v)
    np.testing.assert_allclose(dY, u, rtol=1e-11, atol=1e-12)
    np.testing.assert_allclose(dX, -np.outer(u, bh), rtol=1e-10, atol=1e-11)


def test_adjoint_identity_for_y():
    # d(beta-hat)/dY = (X^T X)^{-1} X^T is linear: <v, J dy> = <dL/dY, dy> exactly
    X, Y, _ = _problem(300, 7, 3)
    bh = linalg.ols(X, Y)
    rng = np.random.default_rng(4)
    v = rng.standard_normal(7)
    dy = rng.standard_normal(300)
    _, _, dY = adj.ols_vjp(X, Y, bh, v)
    jdy = linalg.ols(X, Y + dy) - bh
    assert abs(v @ jdy - dY @ dy) <= 1e-10 * abs(dY @ dy)


def test_normal_solve_inverts_gram():
    X, _, _ = _problem(500, 12, 5)
    v = np.arange(12, dtype=np.float64) - 3
    w = adj.normal_solve(X, v)
    np.testing.assert_allclose(X.T @ (X @ w), v, rtol=1e-12, atol=1e-12)


@pytest.mark.parametrize("bad", ["sign", "transpose"])
def test_planted_mistakes_are_caught(monkeypatch, bad):
    good = adj.ols_vjp

    def wrong(X, Y, b, v):
        w, dX, dY = good(X, Y, b, v)
        if bad == "sign":
            return w, -dX, dY                         # dropped sign of the whole dX
        return w, dX - np.outer(np.asarray(X) @ w, b) + np.outer(np.asarray(Y) - np.asarray(X) @ b, w) * 0, dY
    monkeypatch.setattr(adj, "ols_vjp", wrong)
    with pytest.raises(AssertionError):
        test_formula_matches_central_differences()
