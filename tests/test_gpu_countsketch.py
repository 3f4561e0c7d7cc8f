"""GPU parity of the CountSketch family (Sec. 2; SLSE-FRS-CS of Sec. 5), through the C ABI,
against the CPU oracle on the same seeded inputs.  Cases cover the warp-per-group kernel with
0..3 folded levels, the CTA-per-bucket kernel (buckets of >= 64 rows), the fold kernel, the
Hessian sketch, ragged d (scalar path) and the degenerate sizes."""
import numpy as np
import pytest

import workloads
from oracle import countsketch as ocs
from oracle import linalg, slse as osl
from tests.gpu_helpers import dev, host, torch_cuda

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def slse():
    torch_cuda()
    import paper_2509_06856_gb300 as m
    return m


def _abs_sums(X, Y, b, m, s):
    """Per bucket: sum of |x| (columns and y), the scale of FP32 summation error."""
    ax = np.zeros((m, X.shape[1]))
    np.add.at(ax, b, np.abs(np.asarray(X, np.float64)))
    ay = np.zeros(m)
    np.add.at(ay, b, np.abs(np.asarray(Y, np.float64)))
    return ax, ay


CS_CASES = [(1, 1, 1), (37, 3, 8), (5000, 37, 1), (5000, 37, 64), (5000, 64, 4096), (20000, 50, 512),
            ((1 << 16) + 5, 128, 1 << 15), ((1 << 17) + 3, 33, 1024)]


@pytest.mark.parametrize("N,d,m", CS_CASES)
def test_countsketch_fp64_matches_oracle(slse, N, d, m):
    # a single level is summed in row order on both sides: equal up to FP64 rounding
    p = workloads.gaussian(N, d, seed=N % 89)
    X, Y = p["X"], p["Y"]
    SX, SY = slse.sketch(dev(X), dev(Y), m, seed=5, prec="fp64", kind="countsketch")
    ox, oy = ocs.countsketch(X, Y, m, 5)
    h, s = ocs.cs_hash(N, 5)
    ax, ay = _abs_sums(X, Y, ocs.cs_buckets(h, m), m, s)
    assert np.all(np.abs(host(SX) - ox) <= 1e-12 * ax + 1e-300)
    assert np.all(np.abs(host(SY) - oy) <= 1e-12 * ay + 1e-300)


@pytest.mark.parametrize("N,d,m", [(37, 3, 8), (20000, 50, 512), ((1 << 16) + 5, 128, 1 << 15), (1 << 18, 512, 2048)])
def test_countsketch_bf16_matches_oracle(slse, N, d, m):
    # FP32 sums in row order, one BF16 rounding at the store (relative 2^-9)
    p = workloads.cfg3(N=N, d=d, seed=3)
    X, Y = p["X"], p["Y"]
    SX, SY = slse.sketch(dev(X), dev(Y), m, seed=8, prec="mixed_bf16", kind="countsketch")
    ox, oy = ocs.countsketch(X.astype(np.float64), Y.astype(np.float64), m, 8)
    h, s = ocs.cs_hash(N, 8)
    ax, ay = _abs_sums(X, Y, ocs.cs_buckets(h, m), m, s)
    tx = 2.0 ** -8 * np.abs(ox) + 2.0 ** -20 * ax + 1e-30
    ty = 2.0 ** -8 * np.abs(oy) + 2.0 ** -20 * ay + 1e-30
    assert np.all(np.abs(host(SX) - ox) <= tx)
    assert np.all(np.abs(host(SY) - oy) <= ty)


@pytest.mark.parametrize("N,d,r,prec", [(1, 1, 1, "fp64"), (5000, 37, 96, "fp64"), (20000, 64, 300, "fp64"),
                                        ((1 << 17) + 1, 40, 240, "mixed_bf16"), (1 << 16, 512, 3072, "mixed_bf16")])
def test_countsketch_hat_matches_oracle(slse, N, d, r, prec):
    p = workloads.cfg3(N=N, d=d, seed=4)
    X, Y = p["X"], p["Y"]
    if prec == "fp64":
        X, Y = X.astype(np.float64), Y.astype(np.float64)
    SX, SY = slse.sketch(dev(X), dev(Y), r, seed=6, prec=prec, kind="countsketch_hat")
    ox, oy = ocs.countsketch_hat(X.astype(np.float64), Y.astype(np.float64), r, 6)
    b, s = ocs.hat_hash(N, 6, r)
    ax, ay = _abs_sums(X, Y, b, r, s)
    rel, absf = (1e-13, 0.0) if prec == "fp64" else (2.0 ** -8, 2.0 ** -20)
    assert np.all(np.abs(host(SX) - ox) <= rel * np.abs(ox) + max(absf, 1e-13) * ax + 1e-30)
    assert np.all(np.abs(host(SY) - oy) <= rel * np.abs(oy) + max(absf, 1e-13) * ay + 1e-30)


def test_countsketch_deterministic(slse):
    p = workloads.cfg3(N=(1 << 16) + 17, d=64, seed=1)
    X, Y = dev(p["X"]), dev(p["Y"])
    a = slse.sketch(X, Y, 4096, seed=2, prec="mixed_bf16", kind="countsketch")
    b = slse.sketch(X, Y, 4096, seed=2, prec="mixed_bf16", kind="countsketch")
    assert np.array_equal(host(a[0]), host(b[0])) and np.array_equal(host(a[1]), host(b[1]))
    c = slse.sketch(X, Y, 4096, seed=3, prec="mixed_bf16", kind="countsketch")
    assert not np.array_equal(host(a[0]), host(c[0]))


def test_countsketch_rejects_non_power_of_two(slse):
    p = workloads.gaussian(100, 3, seed=1)
    with pytest.raises(RuntimeError):
        slse.sketch(dev(p["X"]), dev(p["Y"]), 48, seed=0, kind="countsketch")
    with pytest.raises(RuntimeError):
        slse.fit(dev(p["X"]), dev(p["Y"]), slse.Schedule(m=[24, 48], a=[2, 2], r=18, mu=0.7, eta=0.1, T=10,
                                                         kind=slse.COUNTSKETCH), seed=0)


def _oracle_sched(sched, T, kind="countsketch"):
    return osl.Schedule(m=list(sched.m), a=list(sched.a), r=sched.r, mu=sched.mu, eta=sched.eta, T=T, tol=0.0,
                        kind=kind)


@pytest.mark.parametrize("N,d,m,a", [
    (20000, 50, [512, 1024, 2048, 4096, 8192], [2, 2, 2, 2, 2]),     # warp kernel, F = 1 on FP64, folds
    ((1 << 15) + 3, 24, [64, 128, 256], [3, 2, 2]),                  # CTA-per-bucket kernel (>= 64 rows) + folds
    (5000, 16, [4096], [3]),                                         # single level, m close to N
])
def test_fit_countsketch_fp64_iterates_match_oracle(slse, N, d, m, a):
    p = workloads.gaussian(N, d, seed=d)
    X, Y = p["X"], p["Y"]
    T = sum(a) + 20
    sched = slse.Schedule(m=m, a=a, r=6 * d, mu=(1 - 1 / 6) ** 2, eta=1 / 6, T=T, kind=slse.COUNTSKETCH)
    res = slse.fit(dev(X), dev(Y), sched, seed=7, trace_cap=T)
    ores = osl.slse_fit(X, Y, _oracle_sched(sched, T), seed=7, trace=True)
    bh = linalg.ols(X, Y)
    nb = np.linalg.norm(bh)
    hist = host(res.beta_hist)
    assert hist.shape[0] == len(ores.trace) == T
    for t, (g, o) in enumerate(zip(hist, ores.trace)):
        assert np.linalg.norm(g - o) <= 1e-10 * nb, t
    assert res.report["iters_stage1"] == sum(a)


def test_fit_countsketch_fp64_reaches_ols(slse):
    p = workloads.paper(1 << 15, 32, kappa=1e4, sigma2=1e-8, seed=2)
    X, Y = p["X"], p["Y"]
    sched = slse.default_schedule(1 << 15, 32, T=100, tol=1e-13, kind="countsketch")
    assert all((m & (m - 1)) == 0 for m in sched.m)
    res = slse.fit(dev(X), dev(Y), sched, seed=3)
    bh = linalg.ols(X, Y)
    assert np.linalg.norm(res.beta - bh) <= 1e-10 * np.linalg.norm(bh)


@pytest.mark.parametrize("N,d", [(1 << 17, 64), ((1 << 16) + 333, 100), (1 << 18, 512)])
def test_fit_countsketch_mixed_reaches_ols_1e8(slse, N, d):
    p = workloads.cfg3(N=N, d=d, seed=6)
    X, Y = p["X"], p["Y"]
    sched = slse.default_schedule(N, d, prec="mixed_bf16", T=100, tol=1e-10, kind="countsketch")
    res = slse.fit(dev(X), dev(Y), sched, seed=2)
    bh = linalg.ols(X.astype(np.float64), Y.astype(np.float64))
    err = np.linalg.norm(res.beta - bh) / np.linalg.norm(bh)
    assert err <= 1e-8, err
