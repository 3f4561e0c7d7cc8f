"""Pins of the CountSketch oracle (Sec. 2 definition; SLSE-FRS-CS of Sec. 5) against
what the definition and the mathematics fix: the matrix structure, E[S^T S] = I, the
folding identity of the nested family, uniform buckets, the embedding improving with m,
and the fit converging to OLS."""
import math

import numpy as np
import pytest

from oracle import countsketch as cs
from oracle import linalg, slse


@pytest.mark.parametrize("N,m,seed", [(1, 1, 0), (13, 4, 1), (64, 16, 2), (100, 32, 7)])
def test_dense_matrix_structure_and_product(N, m, seed):
    S = cs.countsketch_matrix_dense(N, m, seed)
    # one non-zero per column, equal to +-1
    nz = (S != 0).sum(axis=0)
    assert np.all(nz == 1)
    assert set(np.unique(S[S != 0]).tolist()) <= {-1.0, 1.0}
    # the fast scatter-add equals the dense product S X (integer data: exact)
    rng = np.random.default_rng(seed)
    X = rng.integers(-50, 50, size=(N, 3)).astype(np.float64)
    Y = rng.integers(-50, 50, size=N).astype(np.float64)
    SX, SY = cs.countsketch(X, Y, m, seed)
    assert np.array_equal(SX, S @ X)
    assert np.array_equal(SY, S @ Y)


def test_hat_matrix_structure_and_range():
    N, r = 5000, 96
    S = cs.countsketch_hat_matrix_dense(N, r, 3)
    assert np.all((S != 0).sum(axis=0) == 1)
    b, s = cs.hat_hash(N, 3, r)
    assert b.min() >= 0 and b.max() < r
    # every bucket is hit (5000 rows into 96 buckets)
    assert np.bincount(b, minlength=r).min() > 0
    X = np.arange(N, dtype=np.float64)[:, None] % 7
    assert np.array_equal(cs.countsketch_hat(X, X[:, 0], r, 3)[0], S @ X)


def test_expectation_of_sts_is_identity():
    # E[S^T S] = I_N: average over seeds; off-diagonal entries are s_k s_l [h(k) = h(l)],
    # mean 0 with variance 1/m per seed; diagonal entries are exactly 1.
    N, m, T = 24, 8, 600
    acc = np.zeros((N, N))
    for seed in range(T):
        S = cs.countsketch_matrix_dense(N, m, seed)
        G = S.T @ S
        assert np.allclose(np.diag(G), 1.0)
        acc += G
    acc /= T
    off = acc - np.eye(N)
    sd = math.sqrt(1.0 / m / T)
    assert np.abs(off).max() < 6 * sd


@pytest.mark.parametrize("m", [1, 2, 8, 64])
def test_folding_identity(m):
    # S_m = F S_{4m}: rows agreeing modulo m are added (exact on integer data)
    rng = np.random.default_rng(m)
    N = 777
    X = rng.integers(-9, 9, size=(N, 4)).astype(np.float64)
    Y = rng.integers(-9, 9, size=N).astype(np.float64)
    big = cs.countsketch(X, Y, 4 * m, 5)
    small = cs.countsketch(X, Y, m, 5)
    assert np.array_equal(cs.fold(big[0], m), small[0])
    assert np.array_equal(cs.fold(big[1], m), small[1])


def test_bucket_and_sign_uniformity():
    N, m = 1 << 16, 64
    h, s = cs.cs_hash(N, 11)
    counts = np.bincount(cs.cs_buckets(h, m), minlength=m)
    chi2 = ((counts - N / m) ** 2 / (N / m)).sum()
    assert chi2 < m + 6 * math.sqrt(2 * m)   # chi-square with m-1 dof, generous bound
    assert abs(s.mean()) < 6 / math.sqrt(N)
    # independent streams: the Hessian-sketch signs are uncorrelated with the nested ones
    _, s_hat = cs.hat_hash(N, 11, 96)
    assert abs((s * s_hat).mean()) < 6 / math.sqrt(N)


def test_non_power_of_two_sizes_are_rejected():
    with pytest.raises(ValueError):
        cs.countsketch(np.ones((4, 1)), np.ones(4), 3, 0)


def test_embedding_error_shrinks_with_m():
    # subspace embedding (Def. 3.1) of an orthonormal basis: ||(S U)^T (S U) - I|| falls
    # as m grows (CountSketch needs m ~ d^2, Sec. 3)
    rng = np.random.default_rng(0)
    N, d = 1 << 13, 4
    U, _ = np.linalg.qr(rng.standard_normal((N, d)))
    errs = []
    for m in (16, 256, 4096):
        e = []
        for seed in range(8):
            SU = cs.countsketch(U, U[:, 0], m, seed)[0]
            e.append(np.linalg.norm(SU.T @ SU - np.eye(d), 2))
        errs.append(np.mean(e))
    assert errs[0] > errs[1] > errs[2]
    assert errs[2] < 0.15


def test_countsketch_fit_converges_to_ols():
    rng = np.random.default_rng(4)
    N, d = 4096, 16
    X = rng.standard_normal((N, d)) * np.logspace(0, -2, d)
    beta = rng.standard_normal(d)
    Y = X @ beta + 0.01 * rng.standard_normal(N)
    sched = slse.default_schedule(N, d, tol=1e-13, kind="countsketch")
    assert all(cs.is_pow2(m) for m in sched.m)
    res = slse.slse_fit(X, Y, sched, seed=2)
    ols = linalg.ols(X, Y)
    assert res.converged
    assert np.linalg.norm(res.beta - ols) <= 1e-11 * np.linalg.norm(ols)


def test_countsketch_stage_iterates_solve_the_sketched_problem():
    # with many inner steps, each stage's iterate reaches the LS solution of its own
    # sketched problem (S_i X, S_i Y) (the fixed point used in the proof of Thm 4.1)
    rng = np.random.default_rng(5)
    N, d = 2048, 8
    X = rng.standard_normal((N, d))
    Y = X @ rng.standard_normal(d) + 0.1 * rng.standard_normal(N)
    sched = slse.default_schedule(N, d, kind="countsketch")
    sched.m = sched.m[:2]
    sched.a = [60, 60]
    sched.T = 120
    res = slse.slse_fit(X, Y, sched, seed=9, trace=True)
    SX, SY = cs.countsketch(X, Y, sched.m[1], 9)
    tilde = np.linalg.lstsq(SX, SY, rcond=None)[0]
    assert np.linalg.norm(res.trace[119] - tilde) <= 1e-9 * np.linalg.norm(tilde)
