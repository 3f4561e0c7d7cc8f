"""Pins for the oracle's OLS, QR, M-IHS and SLSE-FRS (Sec. 1, 3, 4, 5 of the paper)."""
import math
import os

import numpy as np
import pytest

import workloads
from oracle import linalg, sketch as sk, slse

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _paper_values():
    vals = {}
    for line in open(os.path.join(GOLDEN, "paper_values.txt")):
        line = line.split("#")[0].strip()
        if line:
            name, value = line.split()[:2]
            vals[name] = float(value)
    return vals


# ---------------------------------------------------------------- QR / OLS

@pytest.mark.parametrize("r,d", [(8, 8), (30, 5), (300, 50)])
def test_householder_r_properties(r, d):
    rng = np.random.default_rng(r)
    A = rng.standard_normal((r, d))
    R = linalg.householder_r(A)
    assert np.allclose(R, np.triu(R))
    assert (np.diag(R) >= 0).all()
    np.testing.assert_allclose(R.T @ R, A.T @ A, rtol=1e-12, atol=1e-10)
    # unique R with positive diagonal = Cholesky factor of A^T A
    np.testing.assert_allclose(R, np.linalg.cholesky(A.T @ A).T, rtol=1e-9, atol=1e-10)


def test_ols_brute_force_longdouble():
    rng = np.random.default_rng(1)
    for N, d in ((10, 3), (64, 7), (40, 40)):
        X = rng.standard_normal((N, d))
        Y = rng.standard_normal(N)
        ref = linalg.ols_normal_longdouble(X, Y)
        np.testing.assert_allclose(linalg.ols(X, Y), ref, rtol=1e-10, atol=1e-12)
        np.testing.assert_allclose(linalg.ols(X, Y, textbook=True), ref, rtol=1e-10, atol=1e-12)


def test_ols_normal_equations_and_noiseless_recovery():
    p = workloads.cfg2(N=1 << 14, d=32, seed=3)
    X, Y = p["X"], p["Y"]
    bh = linalg.ols(X, Y, block_rows=1000)
    g = X.T @ (Y - X @ bh)
    u = np.finfo(float).eps
    assert np.linalg.norm(g) <= 100 * u * np.linalg.norm(X, 2) ** 2 * np.linalg.norm(bh) + 1e-12
    # noiseless: Y = X beta gives beta back to ~cond * u
    b = p["beta_true"]
    rec = linalg.ols(X, X @ b, block_rows=1000)
    assert np.linalg.norm(rec - b) / np.linalg.norm(b) < 1e4 * 1e4 * u


def test_ols_normal_equations_route_on_well_conditioned_data():
    # the written-out definition (X^T X)^{-1} X^T Y agrees with the QR route to cond^2 * u
    p = workloads.cfg3(N=20000, d=64, seed=2)
    X, Y = p["X"].astype(np.float64), p["Y"].astype(np.float64)
    a = linalg.ols_normal(X, Y, block_rows=3000)
    b = linalg.ols(X, Y)
    np.testing.assert_allclose(a, b, rtol=1e-12, atol=1e-13)
    q = workloads.gaussian(40, 5, seed=3)
    np.testing.assert_allclose(linalg.ols_normal(q["X"], q["Y"]), linalg.ols_normal_longdouble(q["X"], q["Y"]),
                               rtol=1e-12)


def test_ols_square_orthogonal():
    Q = workloads.haar_orthogonal(20, 4)
    y = np.random.default_rng(2).standard_normal(20)
    np.testing.assert_allclose(linalg.ols(Q, y, textbook=True), Q.T @ y, atol=1e-13)


def test_tsqr_blocks_agree():
    p = workloads.gaussian(5000, 12, seed=9)
    a = linalg.ols(p["X"], p["Y"], block_rows=64)
    b = linalg.ols(p["X"], p["Y"], block_rows=1 << 16)
    c = linalg.ols(p["X"], p["Y"], textbook=True)
    np.testing.assert_allclose(a, b, rtol=1e-12)
    np.testing.assert_allclose(a, c, rtol=1e-12)


def test_triangular_solves():
    rng = np.random.default_rng(3)
    R = np.triu(rng.standard_normal((9, 9))) + 4 * np.eye(9)
    b = rng.standard_normal(9)
    np.testing.assert_allclose(R @ linalg.solve_upper(R, b), b, atol=1e-12)
    np.testing.assert_allclose(R.T @ linalg.solve_lower(R.T, b), b, atol=1e-12)


# ---------------------------------------------------------------- schedule / a_i

def test_default_schedule_paper_settings():
    s = slse.default_schedule(1 << 20, 64)
    assert s.r == 6 * 64 and s.m[0] == 8 * 64 and s.m[-1] == (1 << 19)
    assert all(b == 2 * a for a, b in zip(s.m, s.m[1:]))
    assert s.K == int(math.log2((1 << 20) / s.m[0]))       # K = log2(N/m_1)
    assert s.eta == pytest.approx(64 / 384) and s.mu == pytest.approx((1 - 64 / 384) ** 2)
    assert all(a == 2 for a in s.a) and s.T == 100


def test_ai_bound_closed_forms():
    v = _paper_values()
    big = 1 << 40
    # r(i-1,i) -> sqrt(2) for doubling sketch sizes far above d
    a16 = slse.ai_bound(1 / 16, big, 2 * big, 64)
    assert a16 == pytest.approx(math.log(((17 / 16) * math.sqrt(2) + 1) * 16, 3), rel=1e-9)
    assert a16 == pytest.approx(3.3587, abs=1e-4)
    assert round(a16) == v["ai_max_over_omega"]             # Sec. 5.1: largest a_i ~ 3
    assert slse.ai_bound(1.0, big, 2 * big, 64) == pytest.approx(math.log(2 * math.sqrt(2) + 1, 3), rel=1e-9)
    # Theorem 4.3 as stated: r(i-1,i) = sqrt((m_i - d)/(m_{i-1} - d)) > 1, so for
    # doubling sizes the bound decreases in i toward the r -> sqrt(2) value.  The
    # proof of Thm 4.4 uses the reciprocal ratio (a_i increasing, below alpha);
    # both readings give a_i ~ 3 at omega = 1/16, as Sec. 5.1 reports.
    N, d, K, om = 1 << 22, 64, 8, 0.25
    m = [N >> (K + 1 - i) for i in range(1, K + 1)]
    a = [slse.ai_bound(om, m[i - 1], m[i], d) for i in range(1, K)]
    assert all(x > y for x, y in zip(a, a[1:]))
    lim = math.log(((1 + om) * math.sqrt(2) + 1) / om, 3)
    assert all(x > lim for x in a) and a[-1] == pytest.approx(lim, rel=1e-3)
    recip = math.log(((17 / 16) / math.sqrt(2) + 1) * 16, 3)
    assert round(recip) == v["ai_max_over_omega"]
    assert math.log(16, 3) < recip < slse.ai_bound_limit(1 / 16) + 1e-12


def test_theory_eta_value():
    assert 53 / 36 - math.sqrt(17) / 3 == pytest.approx(_paper_values()["eta_theory"], abs=1e-4)


# ---------------------------------------------------------------- M-IHS / SLSE-FRS

def test_gradient_sign_and_value():
    rng = np.random.default_rng(5)
    X = rng.standard_normal((100, 4))
    Y = rng.standard_normal(100)
    b = rng.standard_normal(4)
    g = slse.grad(X, Y, b, block_rows=7)
    # g = X^T (Y - X b) is minus the gradient of f(b) = 1/2 ||Y - X b||^2
    f = lambda v: 0.5 * np.sum((Y - X @ v) ** 2)
    num = np.array([(f(b + 1e-6 * e) - f(b - 1e-6 * e)) / 2e-6 for e in np.eye(4)])
    np.testing.assert_allclose(g, -num, rtol=1e-6)


def test_hinv_apply_inverts_sketched_hessian():
    # H-hat = (S-hat X)^T (S-hat X); H-hat^{-1} v computed through the R factor (Appendix)
    p = workloads.cfg2(N=1 << 12, d=24, seed=5)
    A, _ = sk.sketch(p["X"], p["Y"], 6 * 24, 3)
    R = linalg.householder_r(A)
    v = np.random.default_rng(1).standard_normal(24)
    x = slse.hinv_apply(R, v)
    np.testing.assert_allclose((A.T @ A) @ x, v, rtol=1e-6, atol=1e-9 * np.abs(v).max())


def test_stage_iterates_reach_sketched_ls_with_many_inner_iterations():
    # Thm 4.1 (proof): within subproblem i the M-IHS iterates converge to the
    # sketched LS estimator beta~^i = argmin ||S_i Y - S_i X beta||
    p = workloads.gaussian(4096, 8, seed=11)
    X, Y = p["X"], p["Y"]
    sched = slse.Schedule(m=[128, 256, 512], a=[60, 60, 60], r=48, mu=(1 - 8 / 48) ** 2, eta=8 / 48,
                          T=180, tol=0.0)
    res = slse.slse_fit(X, Y, sched, seed=2, trace=True)
    for i, m in enumerate(sched.m):
        SX, SY = sk.sketch(X, Y, m, 2)
        bt = linalg.ols(SX, SY, textbook=True)
        bi = res.trace[60 * (i + 1) - 1]
        assert np.linalg.norm(bi - bt) <= 1e-10 * np.linalg.norm(bt)


def test_stage2_limit_is_ols_and_rate_near_sqrt_d_over_r():
    p = workloads.paper(1 << 14, 16, kappa=1e4, sigma2=1e-8, seed=3)
    X, Y = p["X"], p["Y"]
    bh = linalg.ols(X, Y)
    sched = slse.default_schedule(X.shape[0], 16, T=100)
    res = slse.slse_fit(X, Y, sched, seed=1, trace=True)
    assert np.linalg.norm(res.beta - bh) <= 1e-12 * np.linalg.norm(bh)
    e = np.array([np.linalg.norm(b - bh) for b in res.trace])
    t1 = res.iters_stage1
    seg = e[t1 + 2:t1 + 16]
    rate = (seg[-1] / seg[0]) ** (1.0 / (len(seg) - 1))
    assert 0.2 < rate < 0.6, rate            # M-IHS rate sqrt(d/r) = 0.408 (Sec. 1)


def test_theory_parameters_contract_by_one_third():
    # Thm 4.1/4.2: with eps < 1/10, |mu - 1| <= 1/4 and eta = 53/36 - sqrt(17)/3 the
    # error contracts by at most 1/3 per iteration; a large Hessian sketch keeps eps small
    v = _paper_values()
    p = workloads.gaussian(1 << 13, 4, seed=12, noise_sd=1.0)
    X, Y = p["X"], p["Y"]
    bh = linalg.ols(X, Y)
    eta = 53 / 36 - math.sqrt(17) / 3
    sched = slse.Schedule(m=[], a=[], r=4096, mu=1.0, eta=eta, T=12, tol=0.0)
    res = slse.slse_fit(X, Y, sched, seed=3, trace=True)
    e = [np.linalg.norm(X @ (b - bh)) for b in res.trace]
    e0 = np.linalg.norm(X @ bh)
    # two-step scheme: bound the average contraction over 10 steps
    assert (e[10] / e0) ** (1 / 11) <= v["rate_theory"]


def test_final_prediction_error_reaches_ls_error():
    # Sec. 5.2: Delta_T = ||X(beta_T - beta)||^2 reaches the LS error Delta ~ sigma^2 d
    p = workloads.paper(1 << 14, 64, kappa=1e4, sigma2=1e-8, seed=4)
    X, Y, b = p["X"], p["Y"], p["beta_true"]
    bh = linalg.ols(X, Y)
    res = slse.slse_fit(X, Y, slse.default_schedule(X.shape[0], 64, T=100), seed=5)
    delta = np.sum((X @ (bh - b)) ** 2)
    delta_T = np.sum((X @ (res.beta - b)) ** 2)
    assert delta_T == pytest.approx(delta, rel=1e-6)
    # E[Delta] = sigma^2 d exactly (projection of the noise onto range(X)); chi^2_64 spread
    assert 0.5 < delta / (1e-8 * 64) < 1.6
    assert 1e-8 * 64 == pytest.approx(_paper_values()["ls_error_d64_s2_1e-8"])


def test_noiseless_fit_recovers_beta():
    p = workloads.paper(1 << 12, 8, kappa=10.0, sigma2=0.0, seed=6)
    res = slse.slse_fit(p["X"], p["Y"], slse.default_schedule(1 << 12, 8, T=100), seed=1)
    np.testing.assert_allclose(res.beta, p["beta_true"], rtol=1e-12, atol=1e-12)


def test_tolerance_stop_and_momentum_reset_option():
    p = workloads.cfg1()
    s = slse.Schedule(m=[200 * 2 ** t for t in range(6)], a=[2] * 6, r=300, mu=(1 - 1 / 6) ** 2,
                      eta=1 / 6, T=100, tol=1e-10)
    res = slse.slse_fit(p["X"], p["Y"], s, seed=0)
    bh = linalg.ols(p["X"], p["Y"])
    assert res.converged and res.iters_stage1 + res.iters_stage2 < 100
    assert np.linalg.norm(res.beta - bh) <= 1e-9 * np.linalg.norm(bh)
    s.momentum_reset = True   # the proof's reading (Thm 4.1): restart momentum per subproblem
    s.tol = 0.0
    res2 = slse.slse_fit(p["X"], p["Y"], s, seed=0)
    assert np.linalg.norm(res2.beta - bh) <= 1e-12 * np.linalg.norm(bh)
