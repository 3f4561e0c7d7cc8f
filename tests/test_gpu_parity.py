"""GPU parity: each step of the CUDA path, called through the C ABI, against the CPU
oracle on the same seeded inputs.  Sizes span several tiles, clusters and ragged tails."""
import math

import numpy as np
import pytest

import workloads
from oracle import linalg, sketch as osk, slse as osl
from tests.gpu_helpers import dev, host, padded, torch_cuda

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def slse():
    torch_cuda()
    import paper_2509_06856_gb300 as m
    return m


# ------------------------------------------------------------------ a1: random draws (bit-exact)
@pytest.mark.parametrize("N,seed", [(1, 0), (2, 1), (37, 2), (1000, 3), (1 << 15, 4), ((1 << 20) + 5, 5),
                                    (1 << 22, 7)])
def test_draws_bit_exact(slse, N, seed):
    P, sigma, D = slse.draws(N, seed)
    Do, Po, so = osk.draws(padded(N), seed)
    assert np.array_equal(host(P).astype(np.int64), Po)
    assert np.array_equal(host(sigma).astype(np.int64), so)
    assert np.array_equal(host(D).astype(np.float64), Do)


# ------------------------------------------------------------------ a2-a4: SRHT sketch
SKETCH_CASES = [
    (1, 1, 1), (37, 3, 11), (64, 5, 64), (500, 7, 300),          # single pass (N' <= 512)
    (1000, 9, 700),                                               # two passes 5+5 (direct register path)
    (20000, 50, 6400),                                            # 8+7 split, ragged d and N
    ((1 << 16) + 123, 100, 4096),                                 # 9+9
    ((1 << 19) + 1, 33, 1 << 15),                                 # N' = 2^20: 10+10, 2-CTA clusters
]


@pytest.mark.parametrize("N,d,m", SKETCH_CASES)
def test_sketch_fp64_matches_oracle(slse, N, d, m):
    p = workloads.gaussian(N, d, seed=N % 97)
    X, Y = p["X"], p["Y"]
    SX, SY = slse.sketch(dev(X), dev(Y), m, seed=3, prec="fp64")
    ox, oy = osk.sketch(X, Y, m, 3)
    scale = np.sqrt((X ** 2).sum(0).max() * padded(N) / m / padded(N)) + 1e-300
    np.testing.assert_allclose(host(SX), ox, rtol=0, atol=1e-12 * max(1.0, scale))
    np.testing.assert_allclose(host(SY), oy, rtol=0, atol=1e-12 * max(1.0, np.sqrt((Y ** 2).sum() / m)))


def test_sketch_fp64_from_fp32_storage(slse):
    p = workloads.cfg3(N=5000, d=40, seed=2)
    X, Y = p["X"], p["Y"]  # float32
    SX, SY = slse.sketch(dev(X), dev(Y), 2000, seed=9, prec="fp64")
    ox, oy = osk.sketch(X.astype(np.float64), Y.astype(np.float64), 2000, 9)
    np.testing.assert_allclose(host(SX), ox, rtol=0, atol=1e-11)
    np.testing.assert_allclose(host(SY), oy, rtol=0, atol=1e-11)


def test_sketch_fp64_from_fp32_storage_clustered_special_values(slse):
    # a size whose pass-1 groups span a cluster (N' = 2^18: groups of 2^9 rows on 2 CTAs), FP32
    # storage with signed zeros, denormals and the exponent limits scattered through X; then an
    # infinity and a NaN, which must leave the sketch non-finite exactly where the oracle's is
    rng = np.random.default_rng(11)
    N, d, m = (1 << 17) + 5, 24, 4096
    X = rng.standard_normal((N, d)).astype(np.float32)
    Y = rng.standard_normal(N).astype(np.float32)
    specials = np.array([0.0, -0.0, 1e-40, -3e-45, 1.1754944e-38, -1.1754942e-38, 2.0 ** -126, 3.0e30,
                         -2.5e30, 1.0], np.float32)
    X.reshape(-1)[rng.integers(0, N * d, size=5 * len(specials))] = np.tile(specials, 5)
    SX, SY = slse.sketch(dev(X), dev(Y), m, seed=6, prec="fp64")
    ox, oy = osk.sketch(X.astype(np.float64), Y.astype(np.float64), m, 6)
    scale = np.sqrt((X.astype(np.float64) ** 2).sum(0).max() / m)
    np.testing.assert_allclose(host(SX), ox, rtol=0, atol=1e-12 * scale)
    for bad in (np.float32(np.inf), np.float32(np.nan)):
        Xb = X.copy()
        Xb[N // 2, d // 3] = bad
        SXb, _ = slse.sketch(dev(Xb), dev(Y), m, seed=6, prec="fp64")
        oxb, _ = osk.sketch(Xb.astype(np.float64), Y.astype(np.float64), m, 6)
        g = host(SXb)
        assert np.array_equal(np.isfinite(g), np.isfinite(oxb))
        assert np.array_equal(np.isnan(g), np.isnan(oxb))


@pytest.mark.parametrize("N,d,m", [(37, 3, 11), (20000, 50, 6400), ((1 << 17) + 9, 64, 8192), ((1 << 20), 31, 1 << 14)])
def test_sketch_bf16_matches_oracle_within_bf16_rounding(slse, N, d, m):
    # BF16 storage of the intermediate and of the output: relative rounding 2^-9 at
    # each of the two stores, FP32 arithmetic in between.
    p = workloads.cfg3(N=N, d=d, seed=5)
    X, Y = p["X"], p["Y"]
    SX, SY = slse.sketch(dev(X), dev(Y), m, seed=4, prec="mixed_bf16")
    ox, oy = osk.sketch(X.astype(np.float64), Y.astype(np.float64), m, 4)
    gx = host(SX)
    rms = np.sqrt((ox ** 2).mean(0))
    err = np.abs(gx - ox) / rms
    assert err.max() < 2.0 ** -5, err.max()
    assert err.mean() < 2.0 ** -7, err.mean()
    ey = np.abs(host(SY) - oy) / np.sqrt((oy ** 2).mean())
    assert ey.max() < 2.0 ** -5


# ------------------------------------------------------------------ a6: residual-gradient
GRAD_CASES = [(1, 1), (100, 3), (5000, 50), (20000, 64), ((1 << 16) + 7, 256), (3000, 512), (777, 511)]


def _grad_bound(X, Y, beta):
    X = np.asarray(X, np.float64)
    Y = np.asarray(Y, np.float64)
    return np.abs(X).T @ (np.abs(Y) + np.abs(X) @ np.abs(beta))


@pytest.mark.parametrize("N,d", GRAD_CASES)
def test_grad_fp64_matches_oracle(slse, N, d):
    p = workloads.gaussian(N, d, seed=d)
    X, Y = p["X"], p["Y"]
    beta = p["beta_true"] + 0.01 * np.random.default_rng(1).standard_normal(d)
    g = host(slse.grad(dev(X), dev(Y), beta, prec="fp64"))
    go = osl.grad(X, Y, beta)
    np.testing.assert_array_less(np.abs(g - go), 1e-13 * _grad_bound(X, Y, beta) + 1e-300)


@pytest.mark.parametrize("N,d", [(100, 3), (20000, 64), ((1 << 16) + 7, 256), (3000, 512), (4097, 50)])
def test_grad_fp64_on_fp32_storage(slse, N, d):
    p = workloads.cfg3(N=N, d=d, seed=3)
    X, Y = p["X"], p["Y"]
    beta = p["beta_true"] * 1.001
    g = host(slse.grad(dev(X), dev(Y), beta, prec="fp64"))
    go = osl.grad(X.astype(np.float64), Y.astype(np.float64), beta)
    np.testing.assert_array_less(np.abs(g - go), 1e-13 * _grad_bound(X, Y, beta) + 1e-300)


@pytest.mark.parametrize("d", [7, 256, 512])
def test_grad_fp64_on_fp32_storage_special_values(slse, d):
    # FP32 storage widened to FP64: signed zeros, denormals, the largest and smallest normals and
    # powers of two exactly at the exponent limits, in scattered rows and columns, then a row with
    # an infinity and one with a NaN (the gradient is then non-finite exactly where the oracle's is)
    rng = np.random.default_rng(d)
    N = 3000
    X = rng.standard_normal((N, d)).astype(np.float32)
    Y = rng.standard_normal(N).astype(np.float32)
    specials = np.array([0.0, -0.0, 1e-40, -3e-45, 1.1754944e-38, -1.1754942e-38, 2.0 ** -126, 2.0 ** 127,
                         -3.4e38, 1.0, -1.0, 0.5], np.float32)
    idx = rng.integers(0, N * d, size=4 * len(specials))
    X.reshape(-1)[idx] = np.tile(specials, 4)
    Y[rng.integers(0, N, size=6)] = np.array([0.0, -0.0, 1e-40, -1e-42, 2.0 ** -126, 3e38], np.float32)
    beta = 1e-3 * rng.standard_normal(d)
    go = osl.grad(X.astype(np.float64), Y.astype(np.float64), beta)
    g = host(slse.grad(dev(X), dev(Y), beta, prec="fp64"))
    np.testing.assert_array_less(np.abs(g - go), 1e-13 * _grad_bound(X, Y, beta) + 1e-300)
    for bad in (np.float32(np.inf), np.float32(np.nan)):
        Xb = X.copy()
        Xb[N // 3, d // 2] = bad
        gob = osl.grad(Xb.astype(np.float64), Y.astype(np.float64), beta)
        gb = host(slse.grad(dev(Xb), dev(Y), beta, prec="fp64"))
        assert np.array_equal(np.isfinite(gb), np.isfinite(gob))
        assert np.array_equal(np.isnan(gb), np.isnan(gob))


@pytest.mark.parametrize("N,d", [(100, 3), (20000, 64), ((1 << 16) + 7, 256), (3000, 512), (4097, 50), (999, 7)])
def test_grad_mixed_matches_oracle(slse, N, d):
    # FP32 arithmetic with error-free residuals: the residual is exact to ~2^-48
    # relative, then rounded to FP32 (2^-24 |r|); accumulation is two-sum compensated.
    p = workloads.cfg3(N=N, d=d, seed=4)
    X, Y = p["X"], p["Y"]
    beta = p["beta_true"] * (1.0 + 1e-4)
    g = host(slse.grad(dev(X), dev(Y), beta, prec="mixed_bf16"))
    X64, Y64 = X.astype(np.float64), Y.astype(np.float64)
    go = osl.grad(X64, Y64, beta)
    r = Y64 - X64 @ beta
    bound = np.abs(X64).T @ np.abs(r)
    np.testing.assert_array_less(np.abs(g - go), 4e-7 * bound + 1e-300)


# ------------------------------------------------------------------ a5: QR of the Hessian sketch
@pytest.mark.parametrize("r,d", [(1, 1), (8, 8), (300, 50), (1536, 256), (3072, 512), (600, 77)])
def test_qr_matches_oracle(slse, r, d):
    torch = torch_cuda()
    A = workloads.cfg2(N=r, d=d, seed=r, cond=1e3)["X"] if r >= d and d > 1 else \
        np.random.default_rng(0).standard_normal((r, d))
    R, H = slse.qr(dev(A))
    Ro = linalg.householder_r(A)
    nA = np.linalg.norm(A, 2)
    np.testing.assert_allclose(host(R), Ro, rtol=0, atol=1e-11 * nA)
    Hi = np.linalg.inv(Ro.T @ Ro)
    np.testing.assert_allclose(host(H), Hi, rtol=0, atol=1e-8 * np.abs(Hi).max())


# ------------------------------------------------------------------ a7/a8: the whole method
def _cfg1_schedule(slse, prec="fp64", T=100, tol=0.0):
    return slse.Schedule(m=[200 * 2 ** t for t in range(6)], a=[2] * 6, r=300, mu=(1 - 50 / 300) ** 2,
                         eta=50 / 300, T=T, tol=tol, prec=prec)


def test_fit_fp64_iterates_match_oracle_cfg1(slse):
    p = workloads.cfg1()
    X, Y = p["X"], p["Y"]
    sched = _cfg1_schedule(slse, T=60)
    res = slse.fit(dev(X), dev(Y), sched, seed=0, trace_cap=60)
    osched = osl.Schedule(m=sched.m, a=sched.a, r=sched.r, mu=sched.mu, eta=sched.eta, T=60, tol=0.0)
    ores = osl.slse_fit(X, Y, osched, seed=0, trace=True)
    bh = linalg.ols(X, Y)
    hist = host(res.beta_hist)
    assert hist.shape[0] == len(ores.trace) == 60
    nb = np.linalg.norm(bh)
    for t, (a, b) in enumerate(zip(hist, ores.trace)):
        assert np.linalg.norm(a - b) <= 1e-10 * nb, t
    assert np.linalg.norm(res.beta - bh) <= 1e-10 * nb
    assert res.report["iters_stage1"] == 12 and res.report["iters_stage2"] == 48


def test_fit_fp64_iterates_match_oracle_momentum_reset(slse):
    # the proof's reading (momentum restarted per subproblem) is an option of both sides
    p = workloads.gaussian(8192, 24, seed=5)
    X, Y = p["X"], p["Y"]
    sched = slse.Schedule(m=[192, 384, 768, 1536], a=[3, 2, 2, 2], r=144, mu=(1 - 1 / 6) ** 2, eta=1 / 6, T=30,
                          momentum_reset=True)
    res = slse.fit(dev(X), dev(Y), sched, seed=4, trace_cap=30)
    ores = osl.slse_fit(X, Y, osl.Schedule(m=sched.m, a=sched.a, r=sched.r, mu=sched.mu, eta=sched.eta, T=30,
                                           momentum_reset=True), seed=4, trace=True)
    bh = linalg.ols(X, Y)
    for t, (a, b) in enumerate(zip(host(res.beta_hist), ores.trace)):
        assert np.linalg.norm(a - b) <= 1e-10 * np.linalg.norm(bh), t


def test_fit_hessian_sketch_prefix_fallback(slse):
    # m_K + r > N': S-hat takes the prefix rows sigma[0:r) (the disjoint block does not fit)
    p = workloads.gaussian(3000, 20, seed=12)
    X, Y = p["X"], p["Y"]
    m = [120 * 2 ** t for t in range(6)]                 # m_K = 3840, r = 400, N' = 4096
    sched = slse.Schedule(m=m, a=[2] * 6, r=400, mu=(1 - 20 / 400) ** 2, eta=20 / 400, T=40)
    assert m[-1] + 400 > padded(3000)
    res = slse.fit(dev(X), dev(Y), sched, seed=3, trace_cap=40)
    ores = osl.slse_fit(X, Y, osl.Schedule(m=m, a=[2] * 6, r=400, mu=sched.mu, eta=sched.eta, T=40, tol=0.0),
                        seed=3, trace=True)
    bh = linalg.ols(X, Y)
    nb = np.linalg.norm(bh)
    for t, (a, b) in enumerate(zip(host(res.beta_hist), ores.trace)):
        assert np.linalg.norm(a - b) <= 1e-10 * nb, t
    # the mixed path (two-pass transform, N' = 8192) in the same situation
    q = workloads.cfg3(N=6000, d=40, seed=13)
    mm = [320, 640, 1280, 2560, 5120, 7800]              # m_K + r = 8280 > 8192
    sm = slse.Schedule(m=mm, a=[2] * 6, r=480, mu=(1 - 40 / 480) ** 2, eta=40 / 480, T=100, tol=1e-10,
                       prec="mixed_bf16")
    rm = slse.fit(dev(q["X"]), dev(q["Y"]), sm, seed=4)
    bq = linalg.ols(q["X"].astype(np.float64), q["Y"].astype(np.float64))
    assert np.linalg.norm(rm.beta - bq) <= 1e-8 * np.linalg.norm(bq)


@pytest.mark.parametrize("name,N,d,kappa", [("paper", 1 << 15, 32, 1e4), ("cfg2", 1 << 16, 64, 1e4)])
def test_fit_fp64_reaches_ols(slse, name, N, d, kappa):
    p = workloads.paper(N, d, kappa=kappa, sigma2=1e-8, seed=1) if name == "paper" else \
        workloads.cfg2(N=N, d=d, seed=2, cond=kappa)
    X, Y = p["X"], p["Y"]
    res = slse.fit(dev(X), dev(Y), slse.default_schedule(N, d, T=100, tol=1e-13), seed=1)
    bh = linalg.ols(X, Y)
    assert np.linalg.norm(res.beta - bh) <= 1e-10 * np.linalg.norm(bh)


@pytest.mark.parametrize("stage2", ["correction", "full"])
@pytest.mark.parametrize("N,d", [(1 << 17, 64), ((1 << 16) + 333, 100), (20000, 50), ((1 << 15) + 5, 8)])
def test_fit_mixed_reaches_ols_1e8(slse, N, d, stage2):
    p = workloads.cfg3(N=N, d=d, seed=6)
    X, Y = p["X"], p["Y"]
    sched = slse.default_schedule(N, d, prec="mixed_bf16", T=100, tol=1e-10, stage2=stage2)
    res = slse.fit(dev(X), dev(Y), sched, seed=2)
    bh = linalg.ols(X.astype(np.float64), Y.astype(np.float64))
    err = np.linalg.norm(res.beta - bh) / np.linalg.norm(bh)
    assert err <= 1e-8, err
    assert res.report["rebases"] >= 1
    # the correction form's correction steps (products with the Gram matrix of the BF16 copy,
    # formed once) are counted apart from the exact passes; well-conditioned data never need the
    # fallback to the full form
    if stage2 == "correction":
        assert res.report["n_corr"] > 0 and res.report["stage2_full"] == 0
        assert res.report["ms_gram"] > 0.0
    else:
        assert res.report["n_corr"] == 0


def test_fit_mixed_correction_falls_back_on_ill_conditioned_x(slse):
    """With cond(X) = 1e4 the BF16 Hessian term cannot carry the iteration (its relative error
    2^-9 is far above 1/cond): the correction form gives up after its first cycles and the
    full form finishes; the estimate is as good as the full form's own."""
    N, d = 1 << 16, 64
    p = workloads.cfg2(N=N, d=d, seed=2, cond=1e4)
    X, Y = p["X"].astype(np.float32), p["Y"].astype(np.float32)
    bh = linalg.ols(X.astype(np.float64), Y.astype(np.float64))
    errs, status = {}, {}
    for stage2 in ("correction", "full"):
        sched = slse.default_schedule(N, d, prec="mixed_bf16", T=100, tol=1e-10, stage2=stage2)
        res = slse.fit(dev(X), dev(Y), sched, seed=2)
        errs[stage2] = np.linalg.norm(res.beta - bh) / np.linalg.norm(bh)
        status[stage2] = res.status
        if stage2 == "correction":
            assert res.report["stage2_full"] == 1
    print("cond 1e4, mixed: relative error correction form %.2e, full form %.2e, status %s"
          % (errs["correction"], errs["full"], status))
    assert errs["correction"] <= max(1e-8, 10.0 * errs["full"]), errs


# ------------------------------------------------------------------ edge cases
def test_fit_edge_cases(slse):
    rng = np.random.default_rng(3)
    # square system N = d: OLS interpolates
    X = rng.standard_normal((16, 16)) + 4 * np.eye(16)
    Y = rng.standard_normal(16)
    s = slse.Schedule(m=[], a=[], r=16, mu=1.0, eta=0.0, T=100, tol=0.0)
    res = slse.fit(dev(X), dev(Y), s, seed=0)
    np.testing.assert_allclose(res.beta, np.linalg.solve(X, Y), rtol=1e-9)
    # d = 1, N = 1
    res = slse.fit(dev(np.array([[2.0]])), dev(np.array([3.0])), slse.Schedule(m=[], a=[], r=1, mu=1.0, eta=0.0, T=3),
                   seed=0)
    assert res.beta[0] == pytest.approx(1.5, rel=1e-14)
    # T = 0 returns beta_0 = 0
    p = workloads.gaussian(1000, 5, seed=1)
    res = slse.fit(dev(p["X"]), dev(p["Y"]), slse.Schedule(m=[100], a=[2], r=30, mu=0.6, eta=0.2, T=0), seed=0)
    assert np.all(res.beta == 0.0) and res.report["iters_stage1"] == 0 and res.report["iters_stage2"] == 0
    # tol not met within T -> ENOTCONV, last iterate returned
    res = slse.fit(dev(p["X"]), dev(p["Y"]), slse.Schedule(m=[100], a=[2], r=30, mu=0.6, eta=0.2, T=4, tol=1e-15),
                   seed=0)
    assert res.status == slse.ENOTCONV and res.report["iters_stage2"] == 2
    # stage 1 only (no 2nd stage iterations left)
    res = slse.fit(dev(p["X"]), dev(p["Y"]), slse.Schedule(m=[100, 200], a=[2, 2], r=30, mu=0.6, eta=0.2, T=4),
                   seed=0)
    assert res.report["iters_stage1"] == 4 and res.report["iters_stage2"] == 0


def test_fit_is_deterministic(slse):
    p = workloads.cfg3(N=(1 << 15) + 17, d=48, seed=8)
    X, Y = dev(p["X"]), dev(p["Y"])
    for prec in ("fp64", "mixed_bf16"):
        s = slse.default_schedule(X.shape[0], 48, prec=prec, T=30, tol=0.0)
        a = slse.fit(X, Y, s, seed=5).beta
        b = slse.fit(X, Y, s, seed=5).beta
        assert np.array_equal(a, b)


def test_workspace_contract(slse):
    torch = torch_cuda()
    p = workloads.gaussian(4096, 16, seed=2)
    X, Y = dev(p["X"]), dev(p["Y"])
    s = slse.default_schedule(4096, 16, T=40, tol=0.0)
    need = slse.workspace_size(X, Y, slse.OP_FIT, s)
    ws = slse.alloc_workspace(need)
    a = slse.fit(X, Y, s, seed=1, workspace=ws).beta
    b = slse.fit(X, Y, s, seed=1).beta   # library-allocated workspace
    assert np.array_equal(a, b)
    small = slse.alloc_workspace(need - 1024)
    res = slse.fit(X, Y, s, seed=1, workspace=small, raise_on_error=False)
    assert res.status == slse.ENOMEM
