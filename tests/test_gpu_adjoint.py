"""GPU parity of differentiation through the estimate (slse_solve_normal, slse_ols_vjp and the
torch.autograd binding) against the oracle's dense formulas and central finite differences
(N = 2000, d = 10, h = 1e-6), and at the N = 2^21, d = 128 FP32 workload on sampled rows."""
import numpy as np
import pytest

import workloads
from oracle import adjoint as oadj
from oracle import linalg
from tests.gpu_helpers import dev, host, torch_cuda

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def slse():
    torch_cuda()
    import paper_2509_06856_gb300 as m
    return m


def _fd_problem():
    rng = np.random.default_rng(0)
    X = rng.standard_normal((2000, 10))
    bs = rng.standard_normal(10)
    Y = X @ bs + 0.05 * rng.standard_normal(2000)
    return X, Y, bs


def test_autograd_fp64_matches_formula_and_finite_differences(slse):
    torch = torch_cuda()
    from paper_2509_06856_gb300.autograd import ols
    X, Y, bs = _fd_problem()
    Xt = dev(X).requires_grad_(True)
    Yt = dev(Y).requires_grad_(True)
    beta = ols(Xt, Yt, seed=1)
    loss = 0.5 * ((beta - dev(bs)) ** 2).sum()
    loss.backward()
    gX, gY = host(Xt.grad), host(Yt.grad)
    bh = linalg.ols(X, Y)
    np.testing.assert_allclose(host(beta.detach()), bh, rtol=0, atol=1e-12 * np.linalg.norm(bh))
    _, v = oadj.loss_to_truth(bh, bs)
    _, dX, dY = oadj.ols_vjp(X, Y, bh, v)
    assert np.abs(gX - dX).max() <= 1e-9 * np.abs(dX).max()
    assert np.abs(gY - dY).max() <= 1e-9 * np.abs(dY).max()
    rng = np.random.default_rng(1)
    ex = [(int(i), int(j)) for i, j in zip(rng.integers(0, 2000, 10), rng.integers(0, 10, 10))]
    ey = [int(i) for i in rng.integers(0, 2000, 10)]
    fx, fy = oadj.fd_gradients(X, Y, bs, ex, ey, h=1e-6)
    assert np.all(np.abs(np.array([gX[i, j] for i, j in ex]) - fx) <= 1e-6 * np.abs(dX).max() + 1e-5 * np.abs(fx))
    assert np.all(np.abs(gY[ey] - fy) <= 1e-6 * np.abs(dY).max() + 1e-5 * np.abs(fy))


@pytest.mark.parametrize("N,d,prec", [(1 << 16, 64, "fp64"), ((1 << 15) + 7, 33, "fp64"), (1 << 17, 128, "mixed_bf16")])
def test_solve_normal_matches_oracle(slse, N, d, prec):
    torch = torch_cuda()
    p = workloads.cfg5(N=N, d=d, seed=2) if prec != "fp64" else workloads.gaussian(N, d, seed=3)
    X = p["X"] if prec != "fp64" else p["X"].astype(np.float64)
    Y = p["Y"] if prec != "fp64" else p["Y"].astype(np.float64)
    # the mixed path resolves the solution to ~1e-9, so its relative-step test uses 1e-9
    sched = slse.default_schedule(N, d, prec=prec, T=100, tol=1e-12 if prec == "fp64" else 1e-9)
    Xd, Yd = dev(X), dev(Y)
    res = slse.fit(Xd, Yd, sched, seed=4, hinv=True)
    v = np.random.default_rng(5).standard_normal(d)
    w, rep = slse.solve_normal(Xd, res.hinv, dev(v), sched)
    wo = oadj.normal_solve(np.asarray(X, np.float64), v)
    err = np.linalg.norm(host(w) - wo) / np.linalg.norm(wo)
    assert err <= (1e-10 if prec == "fp64" else 1e-8), err
    if prec != "fp64":
        # from w = 0 the residual base point is kept until the drift matters against the
        # step: the initial rebase and about one more near the solution
        assert 1 <= rep["rebases"] <= 3, rep["rebases"]
    # a caller workspace gives the same bits (fixed reduction order)
    ws = slse.alloc_workspace(slse.solve_normal_workspace(Xd, sched))
    w2, _ = slse.solve_normal(Xd, res.hinv, dev(v), sched, workspace=ws)
    assert np.array_equal(host(w2), host(w))
    assert rep["status"] == 0 and 0 < rep["iters_stage2"] < 100


def test_solve_normal_reports_not_converged(slse):
    p = workloads.gaussian(4096, 16, seed=1)
    Xd, Yd = dev(p["X"]), dev(p["Y"])
    sched = slse.default_schedule(4096, 16, T=100, tol=1e-12)
    res = slse.fit(Xd, Yd, sched, seed=0, hinv=True)
    sched.T = 2
    sched.tol = 1e-15
    w, rep = slse.solve_normal(Xd, res.hinv, dev(np.ones(16)), sched)
    assert rep["status"] == slse.ENOTCONV and rep["iters_stage2"] == 2


def test_vjp_fp32_at_full_size_on_sampled_rows(slse):
    # the N = 2^21, d = 128 FP32 workload: gradients in FP32 from compensated dot products
    torch = torch_cuda()
    N, d = 1 << 21, 128
    p = workloads.cfg5(N=N, d=d, seed=7)
    X, Y = p["X"], p["Y"]
    Xd, Yd = dev(X), dev(Y)
    sched = slse.default_schedule(N, d, prec="mixed_bf16", T=100, tol=1e-9)
    res = slse.fit(Xd, Yd, sched, seed=1, hinv=True)
    beta = res.beta
    v = beta - p["beta_true"]
    w, rep = slse.solve_normal(Xd, res.hinv, dev(v), sched)
    dX, dY = slse.ols_vjp(Xd, Yd, beta, w)
    assert dX.dtype == torch.float32 and dY.dtype == torch.float32
    X64 = X.astype(np.float64)
    wo = oadj.normal_solve(X64, v)
    assert np.linalg.norm(host(w) - wo) <= 1e-7 * np.linalg.norm(wo)
    rows = np.random.default_rng(3).choice(N, 4096, replace=False)
    xs = X64[rows]
    a = xs @ wo
    r = Y[rows].astype(np.float64) - xs @ beta
    ref = np.outer(r, wo) - np.outer(a, beta)
    got = host(dX)[rows]
    scale = np.abs(np.outer(r, wo)) + np.abs(np.outer(a, beta))
    assert np.all(np.abs(got - ref) <= 1e-6 * scale.max(axis=1, keepdims=True) + 1e-6 * np.abs(ref))
    np.testing.assert_allclose(host(dY)[rows], a, rtol=1e-5, atol=1e-6 * np.abs(a).max())


@pytest.mark.parametrize("N,d,pad", [(1037, 36, 0), (4099, 200, 0), (3001, 512, 0), (2053, 130, 0), (5003, 128, 4),
                                     (777, 4, 0), (300, 256, 8)])
def test_vjp_fp32_widths_match_oracle(slse, N, d, pad):
    # FP32 X of each register layout of the row kernel (d <= 128, <= 256, <= 512), the
    # scalar kernel (d % 4 != 0), rows with a leading dimension above d, ragged row counts,
    # and the form that writes into caller buffers; against the oracle's dense formulas
    torch = torch_cuda()
    p = workloads.cfg5(N=N, d=d, seed=11)
    X, Y = p["X"], p["Y"]
    X64, Y64 = X.astype(np.float64), Y.astype(np.float64)
    bh = linalg.ols(X64, Y64)
    v = np.random.default_rng(12).standard_normal(d)
    wo, dXo, dYo = oadj.ols_vjp(X64, Y64, bh, v)
    Xw = torch.zeros((N, d + pad), dtype=torch.float32, device="cuda")
    Xw[:, :d] = dev(X)
    Xd = Xw[:, :d]
    Yd = dev(Y)
    outs = (torch.full((N, d), np.nan, dtype=torch.float32, device="cuda"),
            torch.full((N,), np.nan, dtype=torch.float32, device="cuda"))
    for out in (None, outs):
        dX, dY = slse.ols_vjp(Xd, Yd, bh, dev(wo), out=out)
        torch.cuda.synchronize()
        got, gy = host(dX), host(dY)
        r = Y64 - X64 @ bh
        scale = np.abs(np.outer(r, wo)) + np.abs(np.outer(X64 @ wo, bh))
        assert np.all(np.abs(got - dXo) <= 1e-6 * scale.max(axis=1, keepdims=True) + 1e-6 * np.abs(dXo))
        np.testing.assert_allclose(gy, dYo, rtol=1e-5, atol=1e-6 * np.abs(dYo).max())
    assert outs[0].data_ptr() == dX.data_ptr()


def test_autograd_mixed_fp32_gradients(slse):
    torch = torch_cuda()
    from paper_2509_06856_gb300.autograd import ols
    p = workloads.cfg5(N=1 << 16, d=32, seed=9)
    X, Y = p["X"], p["Y"]
    Xt = dev(X).requires_grad_(True)
    Yt = dev(Y).requires_grad_(True)
    beta = ols(Xt, Yt, seed=2)
    loss = 0.5 * ((beta - dev(p["beta_true"])) ** 2).sum()
    loss.backward()
    assert Xt.grad.dtype == torch.float32
    X64, Y64 = X.astype(np.float64), Y.astype(np.float64)
    bh = linalg.ols(X64, Y64)
    _, v = oadj.loss_to_truth(bh, p["beta_true"])
    _, dX, dY = oadj.ols_vjp(X64, Y64, bh, v)
    assert np.abs(host(Yt.grad) - dY).max() <= 1e-5 * np.abs(dY).max()
    assert np.abs(host(Xt.grad) - dX).max() <= 1e-5 * np.abs(dX).max()
