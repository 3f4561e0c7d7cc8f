"""Pins for the oracle's Hadamard transform and SRHT (Sec. 3 of the paper)."""
import math

import numpy as np
import pytest

from oracle import linalg, sketch as sk


def _kron_hadamard(n):
    # Sylvester construction by Kronecker products, independent of the popcount formula
    H = np.array([[1.0]])
    while H.shape[0] < n:
        H = np.kron(np.array([[1.0, 1.0], [1.0, -1.0]]), H)
    return H


@pytest.mark.parametrize("n", [1, 2, 4, 8, 32, 64])
def test_dense_hadamard_matches_sylvester(n):
    assert np.array_equal(sk.hadamard_dense(n), _kron_hadamard(n))


@pytest.mark.parametrize("n", [1, 2, 16, 64])
def test_fwht_matches_dense(n):
    rng = np.random.default_rng(n)
    A = rng.standard_normal((n, 3))
    np.testing.assert_allclose(sk.fwht(A), _kron_hadamard(n) @ A, rtol=0, atol=1e-12)


def test_fwht_involution_and_parseval():
    rng = np.random.default_rng(1)
    n = 1 << 12
    x = rng.standard_normal((n, 2))
    Hx = sk.fwht(x)
    np.testing.assert_allclose(sk.fwht(Hx) / n, x, atol=1e-12)           # H H = n I
    np.testing.assert_allclose((Hx ** 2).sum(0), n * (x ** 2).sum(0), rtol=1e-12)  # Parseval


@pytest.mark.parametrize("N,m,seed", [(16, 5, 0), (37, 11, 3), (64, 64, 1), (50, 20, 7)])
def test_fast_sketch_equals_dense_definition(N, m, seed):
    rng = np.random.default_rng(N)
    X = rng.standard_normal((N, 4))
    Y = rng.standard_normal(N)
    S = sk.sketch_matrix_dense(N, m, seed)
    SX, SY = sk.sketch(X, Y, m, seed)
    np.testing.assert_allclose(SX, S @ X, atol=1e-12)
    np.testing.assert_allclose(SY, S @ Y, atol=1e-12)


def test_sketch_rows_orthogonal():
    # rows of B H D P are orthonormal, so S S^T = (N'/m) I when N = N'
    S = sk.sketch_matrix_dense(64, 24, 2)
    np.testing.assert_allclose(S @ S.T, (64 / 24) * np.eye(24), atol=1e-12)


def test_full_sketch_is_orthogonal_so_sketched_ls_is_ols():
    # m = N = N': S is square orthogonal, the sketched LS estimator equals OLS exactly
    rng = np.random.default_rng(4)
    N, d = 256, 6
    X = rng.standard_normal((N, d))
    Y = X @ rng.standard_normal(d) + 0.1 * rng.standard_normal(N)
    SX, SY = sk.sketch(X, Y, N, seed=8)
    np.testing.assert_allclose(SX.T @ SX, X.T @ X, rtol=1e-12, atol=1e-10)
    np.testing.assert_allclose(linalg.ols(SX, SY, textbook=True), linalg.ols(X, Y, textbook=True),
                               rtol=1e-11, atol=1e-12)


def test_padding_rows_are_zero_contributions():
    # N not a power of two: the padded rows of X carry zeros, so the sketch of
    # X equals the sketch of X_pad (explicit zero rows appended)
    rng = np.random.default_rng(5)
    X = rng.standard_normal((37, 3))
    Y = rng.standard_normal(37)
    Xp = np.vstack([X, np.zeros((27, 3))])
    Yp = np.concatenate([Y, np.zeros(27)])
    a = sk.sketch(X, Y, 17, 6)
    b = sk.sketch(Xp, Yp, 17, 6)
    np.testing.assert_allclose(a[0], b[0], atol=1e-13)
    np.testing.assert_allclose(a[1], b[1], atol=1e-13)


def test_nested_sketches_share_rows():
    # Sec. 3: S_i is a row subset of S_{i+1}; rows scale by sqrt(N/m_i)
    rng = np.random.default_rng(6)
    X = rng.standard_normal((128, 3))
    Y = rng.standard_normal(128)
    a, _ = sk.sketch(X, Y, 16, 1)
    b, _ = sk.sketch(X, Y, 32, 1)
    np.testing.assert_allclose(a / math.sqrt(128 / 16), b[:16] / math.sqrt(128 / 32), atol=1e-13)


def test_subspace_embedding_improves_with_m():
    # Def. 3.1: ||U^T S^T S U - I|| shrinks as m grows (averaged over seeds)
    rng = np.random.default_rng(7)
    N, d = 1 << 11, 8
    U, _ = np.linalg.qr(rng.standard_normal((N, d)))
    eps = []
    for m in (64, 256, 1024):
        e = []
        for s in range(6):
            SU, _ = sk.sketch(U, np.zeros(N), m, s)
            e.append(np.linalg.norm(SU.T @ SU - np.eye(d), 2))
        eps.append(np.mean(e))
    assert eps[0] > eps[1] > eps[2]
    assert eps[2] < 0.3


@pytest.mark.slow
def test_prediction_efficiency_matches_srht_limit():
    # Lemma A.6 (Dobriban & Liu): PE = E||X(b~ - b)||^2 / E||X(b^ - b)||^2 -> (1-g)/(xi-g)
    # with g = d/N, xi = m/N, i.e. (N - d)/(m - d).  Monte Carlo over noise and sketch seeds.
    rng = np.random.default_rng(8)
    N, d, m = 1 << 12, 16, 512
    X = rng.standard_normal((N, d))
    beta = rng.standard_normal(d)
    num = den = 0.0
    for s in range(200):
        Y = X @ beta + rng.standard_normal(N)
        SX, SY = sk.sketch(X, Y, m, s)
        bt = np.linalg.lstsq(SX, SY, rcond=None)[0]
        bh = np.linalg.lstsq(X, Y, rcond=None)[0]
        num += np.sum((X @ (bt - beta)) ** 2)
        den += np.sum((X @ (bh - beta)) ** 2)
    pe = num / den
    assert abs(pe / ((N - d) / (m - d)) - 1.0) < 0.15, pe


def test_hessian_rows_disjoint_block_or_prefix():
    # reading of Sec. 4 / Thm 4.4: S-hat takes the r sampled rows after the largest nested
    # sketch (disjoint from every S_i), or the prefix when that block does not fit in N'
    assert sk.hessian_rows(4096, 3000, 1000) == (3000, 4000)
    assert sk.hessian_rows(4096, 3096, 1000) == (3096, 4096)
    assert sk.hessian_rows(4096, 3840, 400) == (0, 400)
    for Np, mK, r in [(1 << 12, 1 << 11, 300), (1 << 10, 1000, 24)]:
        h0, h1 = sk.hessian_rows(Np, mK, r)
        assert h1 - h0 == r and 0 <= h0 and h1 <= Np
        assert h0 >= mK or h0 == 0


@pytest.mark.parametrize("N,m,seed", [(40, 12, 2), (64, 64, 5), (300, 100, 9)])
def test_sketch_entries_equal_dense_definition(N, m, seed):
    # single entries from the definition against the dense matrix S built entry by entry
    # (N' <= 512, padding included), so a sign, index or scale slip in either shows up
    rng = np.random.default_rng(seed)
    d = 5
    X = rng.standard_normal((N, d))
    Y = rng.standard_normal(N)
    Np = sk.padded_size(N)
    D, P, sigma = sk.draws(Np, seed)
    rows = [0, m // 2, m - 1]
    cols = [0, 2, d - 1, d]
    got = sk.sketch_entries(X, Y, D, P, sigma, m, rows, cols)
    S = sk.sketch_matrix_dense(N, m, seed) if Np <= 256 else None
    if S is not None:
        ref = (S @ np.column_stack([X, Y]))[np.ix_(rows, cols)]
    else:
        SX, SY = sk.sketch(X, Y, m, seed)
        ref = np.column_stack([SX, SY])[np.ix_(rows, cols)]
    np.testing.assert_allclose(got, ref, rtol=1e-12, atol=1e-12)
