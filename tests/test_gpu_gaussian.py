"""GPU parity of the Gaussian Hessian sketch (Sec. 2; S = G / sqrt(m)) through the C ABI
against the CPU oracle on the same seeds.

MIXED_BF16 (tensor cores): the entries are drawn in FP32 with hardware approximations
(absolute error < 1e-4, relative 2^-20 away from the smallest radii) and rounded to BF16,
X is rounded to BF16, products are summed in FP32 (within a CTA's chunk range, then the
per-split sums in FP64) and the result is rounded to BF16.  So against the exact FP64
sketch o = G X / sqrt(m) an output differs by at most 2^-8 |o| (output rounding) plus the
sum of N independent operand roundings, each below 2^-8 |g_k x_k| (bounded here by 6 of
their root-sum-square), plus FP32 accumulation.  Against the sketch of the BF16-rounded
operands the operand term disappears except where the FP32 draw and the FP64 draw round to
different BF16 values (a few per 10^4 entries).

Cases: identity X (the entries themselves), ragged N, m and d, one and two MMAs per K step
(d <= 256 and d > 256), two column groups (d = 512 with Y), several K splits, the FP64
path, and fits with a Gaussian Hessian sketch (FP64 iterates against the oracle, mixed
convergence to OLS)."""
import math

import numpy as np
import pytest

import workloads
from oracle import gaussian as ogs
from oracle import linalg, slse as osl
from tests.gpu_helpers import dev, host, torch_cuda

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def slse():
    torch_cuda()
    import paper_2509_06856_gb300 as m
    return m


def _bf16(a):
    torch = torch_cuda()
    return torch.from_numpy(np.asarray(a, np.float64)).to(torch.bfloat16).to(torch.float64).numpy()


@pytest.mark.parametrize("n,m", [(256, 1024), (300, 1000), (16, 128), (512, 130)])
def test_entries_bf16_match_oracle(slse, n, m):
    # X = I_n: S X = G[:, :n] / sqrt(m), so the output shows the drawn entries themselves
    torch = torch_cuda()
    X = np.eye(n, dtype=np.float32)
    SX, _ = slse.sketch(dev(X), dev(np.zeros(n, np.float32)), m, seed=11, prec="mixed_bf16", kind="gaussian",
                        want_y=False)
    got = host(SX.to(torch.float64)) * math.sqrt(m)
    G = ogs.gaussian_rows(11, 0, m, n)
    scale_exact = (m & (m - 1)) == 0 and int(round(math.log2(m))) % 2 == 0
    tol = 2.0 ** -8 * np.abs(G) + 1e-4 + (0.0 if scale_exact else 2.0 ** -8 * np.abs(G))
    assert np.all(np.abs(got - G) <= tol)
    if scale_exact:
        # 1/sqrt(m) a power of two: the output is the BF16 entry itself; the FP32 and FP64
        # draws round to different BF16 values only near a rounding midpoint
        mism = np.mean(got != _bf16(G))
        assert mism < 2e-3, mism


def test_entries_fp64_match_oracle(slse):
    n, m = 200, 300
    X = np.eye(n)
    SX, SY = slse.sketch(dev(X), dev(np.ones(n)), m, seed=5, prec="fp64", kind="gaussian")
    G = ogs.gaussian_rows(5, 0, m, n)
    np.testing.assert_allclose(host(SX) * math.sqrt(m), G, rtol=1e-13, atol=1e-14)
    np.testing.assert_allclose(host(SY) * math.sqrt(m), G.sum(axis=1), rtol=1e-12, atol=1e-12)


def _oracle_parts(X, Y, m, seed):
    """Exact sketch, sketch of BF16-rounded operands, and the error scales sqrt(sum (g x)^2),
    sum |g x| of every output (X with Y appended as the last column)."""
    XY = np.concatenate([np.asarray(X, np.float64), np.asarray(Y, np.float64)[:, None]], axis=1)
    XYb = _bf16(XY)
    N = XY.shape[0]
    ex = np.empty((m, XY.shape[1]))
    em = np.empty_like(ex)
    rss = np.empty_like(ex)
    s1 = np.empty_like(ex)
    for i0 in range(0, m, 32):
        i1 = min(m, i0 + 32)
        G = ogs.gaussian_rows(seed, i0, i1, N)
        ex[i0:i1] = G @ XY
        em[i0:i1] = _bf16(G) @ XYb
        rss[i0:i1] = np.sqrt((G ** 2) @ (XY ** 2))
        s1[i0:i1] = np.abs(G) @ np.abs(XY)
    c = 1.0 / math.sqrt(m)
    return ex * c, em * c, rss * c, s1 * c


GAUSS_CASES = [((1 << 16) + 37, 100, 600), (5000, 300, 256), (1 << 15, 512, 130), (100, 1, 5), (1, 1, 1),
               (20000, 256, 384), ((1 << 17) + 5, 40, 128)]


@pytest.mark.parametrize("N,d,m", GAUSS_CASES)
def test_sketch_bf16_matches_oracle(slse, N, d, m):
    torch = torch_cuda()
    p = workloads.cfg3(N=N, d=d, seed=N % 97) if N >= d + 1 and N > 2 else None
    if p is None:
        rng = np.random.default_rng(0)
        X = rng.standard_normal((N, d)).astype(np.float32)
        Y = rng.standard_normal(N).astype(np.float32)
    else:
        X, Y = p["X"], p["Y"]
    SX, SY = slse.sketch(dev(X), dev(Y), m, seed=3, prec="mixed_bf16", kind="gaussian")
    got = np.concatenate([host(SX.to(torch.float64)), host(SY.to(torch.float64))[:, None]], axis=1)
    ex, em, rss, s1 = _oracle_parts(X, Y, m, 3)
    # against the BF16-rounded operands: output rounding, rare draw flips, FP32 accumulation
    tol_em = 2.0 ** -8 * np.abs(em) + 2.0 ** -10 * rss + 2.0 ** -18 * s1 + 1e-30
    assert np.all(np.abs(got - em) <= tol_em), np.max(np.abs(got - em) / tol_em)
    # against the exact sketch: plus the operand roundings (random, each below 2^-8 |g x|)
    tol_ex = 2.0 ** -8 * np.abs(ex) + 6 * 2.0 ** -8 * rss + 2.0 ** -18 * s1 + 1e-30
    assert np.all(np.abs(got - ex) <= tol_ex), np.max(np.abs(got - ex) / tol_ex)


@pytest.mark.parametrize("N,d,m,dtype", [(5000, 37, 96, np.float64), ((1 << 15) + 3, 130, 300, np.float64),
                                         (777, 3, 10, np.float32)])
def test_sketch_fp64_matches_oracle(slse, N, d, m, dtype):
    p = workloads.gaussian(N, d, seed=d)
    X, Y = p["X"].astype(dtype), p["Y"].astype(dtype)
    SX, SY = slse.sketch(dev(X), dev(Y), m, seed=9, prec="fp64", kind="gaussian")
    ex, _, _, s1 = _oracle_parts(X, Y, m, 9)
    got = np.concatenate([host(SX), host(SY)[:, None]], axis=1)
    assert np.all(np.abs(got - ex) <= 1e-13 * s1 + 1e-300)


def test_sketch_deterministic_and_seeded(slse):
    torch = torch_cuda()
    p = workloads.cfg3(N=(1 << 16) + 9, d=64, seed=2)
    X, Y = dev(p["X"]), dev(p["Y"])
    a = slse.sketch(X, Y, 200, seed=4, prec="mixed_bf16", kind="gaussian")
    b = slse.sketch(X, Y, 200, seed=4, prec="mixed_bf16", kind="gaussian")
    c = slse.sketch(X, Y, 200, seed=5, prec="mixed_bf16", kind="gaussian")
    assert torch.equal(a[0], b[0]) and torch.equal(a[1], b[1])
    assert not torch.equal(a[0], c[0])


def test_fit_gaussian_fp64_iterates_match_oracle(slse):
    N, d = 20000, 50
    p = workloads.gaussian(N, d, seed=3)
    X, Y = p["X"], p["Y"]
    T = 30
    sched = slse.Schedule(m=[400, 800, 1600, 3200], a=[2, 2, 2, 2], r=300, mu=(1 - 1 / 6) ** 2, eta=1 / 6, T=T,
                          kind=slse.GAUSSIAN)
    res = slse.fit(dev(X), dev(Y), sched, seed=7, trace_cap=T)
    ores = osl.slse_fit(X, Y, osl.Schedule(m=sched.m, a=sched.a, r=sched.r, mu=sched.mu, eta=sched.eta, T=T,
                                           kind="gaussian"), seed=7, trace=True)
    bh = linalg.ols(X, Y)
    hist = host(res.beta_hist)
    assert hist.shape[0] == len(ores.trace) == T
    for t, (g, o) in enumerate(zip(hist, ores.trace)):
        assert np.linalg.norm(g - o) <= 1e-10 * np.linalg.norm(bh), t


@pytest.mark.parametrize("N,d", [(1 << 17, 64), ((1 << 16) + 333, 100), (1 << 18, 512)])
def test_fit_gaussian_mixed_reaches_ols_1e8(slse, N, d):
    p = workloads.cfg3(N=N, d=d, seed=6)
    X, Y = p["X"], p["Y"]
    sched = slse.default_schedule(N, d, prec="mixed_bf16", T=100, tol=1e-10, kind="gaussian")
    res = slse.fit(dev(X), dev(Y), sched, seed=2, hinv=True)
    bh = linalg.ols(X.astype(np.float64), Y.astype(np.float64))
    err = np.linalg.norm(res.beta - bh) / np.linalg.norm(bh)
    assert err <= 1e-8, err
    assert res.report["status"] == 0
    if d <= 100:
        # the preconditioner is the inverse Gram matrix of the BF16 sketch rows G X / sqrt(r):
        # its product with the exact H-hat = (G X)^T (G X) / r is close to I (BF16 rows)
        ex = _oracle_parts(X, Y, sched.r, 2)[0][:, :d]
        H = ex.T @ ex
        E = host(res.hinv) @ H - np.eye(d)
        assert np.linalg.norm(E, 2) < 0.05


def test_fit_gaussian_fp64_stage2_only_matches_oracle(slse):
    # no subproblems: nothing is sampled from the SRHT (the draws and passes are skipped) and
    # every iteration is a full-data M-IHS step preconditioned by the Gaussian sketch
    N, d = 6000, 20
    p = workloads.gaussian(N, d, seed=8)
    X, Y = p["X"], p["Y"]
    T = 12
    sched = slse.Schedule(m=[], a=[], r=120, mu=(1 - 1 / 6) ** 2, eta=1 / 6, T=T, kind=slse.GAUSSIAN)
    res = slse.fit(dev(X), dev(Y), sched, seed=5, trace_cap=T)
    ores = osl.slse_fit(X, Y, osl.Schedule(m=[], a=[], r=120, mu=sched.mu, eta=sched.eta, T=T, kind="gaussian"),
                        seed=5, trace=True)
    bh = linalg.ols(X, Y)
    hist = host(res.beta_hist)
    assert hist.shape[0] == len(ores.trace) == T and res.report["iters_stage1"] == 0
    for t, (g, o) in enumerate(zip(hist, ores.trace)):
        assert np.linalg.norm(g - o) <= 1e-10 * np.linalg.norm(bh), t
