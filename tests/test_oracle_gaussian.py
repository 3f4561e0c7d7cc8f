"""Pins of the Gaussian-sketch oracle (Sec. 2: S with i.i.d. N(0, 1/m) entries) against
what the Box-Muller transform and the mathematics fix: closed-form values of the
transform, the normal law (moments and Kolmogorov-Smirnov distance), independence of
rows and columns, E[S^T S] = I, the Marchenko-Pastur edge of the embedding error, the
exact finite-sample prediction efficiency of sketch-and-solve with a Gaussian sketch,
and the SLSE-FRS fit with a Gaussian Hessian sketch converging to OLS."""
import math

import numpy as np
import pytest

from oracle import gaussian as gs
from oracle import linalg, slse


def _word(lo, hi):
    return np.array([(hi << 16) | lo], np.uint64)


def test_box_muller_closed_form_values():
    # u1 = 1/2 - 2^-17, u2 = 1/4 + 2^-17: radius sqrt(2 ln 2) (to 2e-5), angle pi/2 + 2 pi 2^-17,
    # so the cosine entry is about -R 2 pi 2^-17 and the sine entry about R
    e, o = gs.normals_from_words(_word(32767, 16384))
    assert abs(o[0] - math.sqrt(2 * math.log(2))) < 1e-4
    assert abs(e[0] + math.sqrt(2 * math.log(2)) * 2 * math.pi * 2.0 ** -17) < 1e-6
    # u1 = 1 - 2^-17: -2 ln u1 = 2^-16 (1 + O(2^-17)), radius 2^-8; u2 = 2^-17: angle ~ 0
    e, o = gs.normals_from_words(_word(0xFFFF, 0))
    assert abs(e[0] - 2.0 ** -8) < 1e-7 and abs(o[0]) < 1e-6
    # u1 = 2^-17: radius sqrt(34 ln 2), the largest magnitude; u2 = 1/2 - 2^-17: angle ~ pi
    e, o = gs.normals_from_words(_word(0, 32767))
    assert abs(e[0] + math.sqrt(34 * math.log(2))) < 1e-6 and abs(o[0]) < 1e-3


def test_normal_law_moments_and_ks():
    G = gs.gaussian_rows(7, 0, 16, 1 << 16).ravel()
    n = G.size
    assert abs(G.mean()) < 6 / math.sqrt(n)
    assert abs((G ** 2).mean() - 1.0) < 6 * math.sqrt(2.0 / n)
    assert abs((G ** 4).mean() - 3.0) < 6 * math.sqrt(96.0 / n)
    assert np.abs(G).max() <= math.sqrt(34 * math.log(2)) + 1e-12
    # Kolmogorov-Smirnov distance to the standard normal CDF (the 16-bit uniforms move
    # the CDF by at most ~2^-16)
    x = np.sort(G)
    cdf = 0.5 * (1.0 + np.vectorize(math.erf)(x / math.sqrt(2.0)))
    i = np.arange(1, n + 1) / n
    D = max(np.abs(i - cdf).max(), np.abs(i - 1.0 / n - cdf).max())
    assert D < 1.63 / math.sqrt(n) + 2.0 ** -15, D


def test_rows_and_columns_are_independent():
    # distinct counters for every (row, 8-column block): no two rows or columns repeat or
    # correlate; the even/odd (cosine/sine) entries of one word are uncorrelated
    G = gs.gaussian_rows(3, 0, 64, 4096)
    C = np.corrcoef(G)
    off = C[~np.eye(64, dtype=bool)]
    assert np.abs(off).max() < 6 / math.sqrt(4096)
    Gc = np.corrcoef(gs.gaussian_rows(4, 0, 2048, 64).T)
    assert np.abs(Gc[~np.eye(64, dtype=bool)]).max() < 6 / math.sqrt(2048)
    ev, od = G[:, 0::2].ravel(), G[:, 1::2].ravel()
    assert abs(np.mean(ev * od)) < 6 / math.sqrt(ev.size)
    # seeds give different matrices; the same seed the same one
    assert np.array_equal(G, gs.gaussian_rows(3, 0, 64, 4096))
    assert not np.allclose(G, gs.gaussian_rows(4, 0, 64, 4096))
    # a row block is the same whatever block it is drawn in
    assert np.array_equal(G[10:20], gs.gaussian_rows(3, 10, 20, 4096))


@pytest.mark.parametrize("N,m,seed", [(1, 1, 0), (13, 5, 1), (100, 37, 2)])
def test_sketch_equals_dense_product(N, m, seed):
    S = gs.gaussian_matrix_dense(N, m, seed)
    rng = np.random.default_rng(seed)
    X = rng.standard_normal((N, 4))
    Y = rng.standard_normal(N)
    SX, SY = gs.gaussian_sketch(X, Y, m, seed, block_rows=3)
    np.testing.assert_allclose(SX, S @ X, rtol=1e-13, atol=1e-13)
    np.testing.assert_allclose(SY, S @ Y, rtol=1e-13, atol=1e-13)


def test_expectation_of_sts_is_identity():
    # (S^T S)_{kl} = (1/m) sum_i G_ik G_il: mean delta_kl; variance 2/m on the diagonal and
    # 1/m off it, so the average over T seeds has standard deviation sqrt(2/(mT)) at most
    N, m, T = 16, 8, 400
    acc = np.zeros((N, N))
    for seed in range(T):
        S = gs.gaussian_matrix_dense(N, m, seed)
        acc += S.T @ S
    acc /= T
    assert np.abs(acc - np.eye(N)).max() < 6 * math.sqrt(2.0 / (m * T))


def test_embedding_error_at_the_marchenko_pastur_edge():
    # S U for orthonormal U (N x d) is m x d with i.i.d. N(0, 1/m) entries, so the extreme
    # eigenvalues of (SU)^T SU approach (1 +- sqrt(d/m))^2 and ||(SU)^T SU - I|| -> 2 sqrt(d/m) + d/m
    rng = np.random.default_rng(0)
    N, d, m = 4096, 8, 512
    U, _ = np.linalg.qr(rng.standard_normal((N, d)))
    errs = []
    for seed in range(6):
        SU = gs.gaussian_sketch(U, U[:, 0], m, seed)[0]
        errs.append(np.linalg.norm(SU.T @ SU - np.eye(d), 2))
    edge = 2 * math.sqrt(d / m) + d / m
    assert 0.6 * edge < np.mean(errs) < 1.2 * edge, (np.mean(errs), edge)


def test_prediction_efficiency_exact_gaussian_value():
    # Sketch-and-solve b~ = (SX)^+ S Y.  Writing the noise as X a + e_perp, SX and S e_perp
    # are independent for Gaussian S, and E[(A^T A)^{-1}] = I/(m - d - 1) for an m x d
    # standard normal A (inverse Wishart mean), so
    #   PE = E||X(b~ - b)||^2 / E||X(b^ - b)||^2 = 1 + (N - d)/(m - d - 1)
    # exactly, for any full-rank X.  Given S the noise expectation is sigma^2 ||X (SX)^+ S||_F^2.
    rng = np.random.default_rng(1)
    N, d, m = 512, 8, 64
    X = rng.standard_normal((N, d)) * np.logspace(0, -1, d)
    acc = 0.0
    T = 300
    for seed in range(T):
        S = gs.gaussian_matrix_dense(N, m, seed)
        P = X @ np.linalg.pinv(S @ X) @ S
        acc += np.sum(P * P)
    pe = acc / T / d
    expect = 1.0 + (N - d) / (m - d - 1)
    assert abs(pe / expect - 1.0) < 0.05, (pe, expect)


def test_gaussian_hessian_sketch_fit_converges_to_ols():
    rng = np.random.default_rng(4)
    N, d = 4096, 16
    X = rng.standard_normal((N, d)) * np.logspace(0, -2, d)
    beta = rng.standard_normal(d)
    Y = X @ beta + 0.01 * rng.standard_normal(N)
    sched = slse.default_schedule(N, d, tol=1e-13, kind="gaussian")
    res = slse.slse_fit(X, Y, sched, seed=2)
    ols = linalg.ols(X, Y)
    assert res.converged
    assert np.linalg.norm(res.beta - ols) <= 1e-11 * np.linalg.norm(ols)
    # the preconditioner is R of G X / sqrt(r): R^T R equals (G X)^T (G X) / r
    G = gs.gaussian_rows(2, 0, sched.r, N)
    H = (G @ X).T @ (G @ X) / sched.r
    np.testing.assert_allclose(res.R.T @ res.R, H, rtol=1e-10, atol=1e-12 * np.abs(H).max())
