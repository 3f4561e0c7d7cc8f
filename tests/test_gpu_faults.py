"""Faults injected on the host, none of which faults, traps or hangs the GPU:

* NaN rows in X: the fit reports SLSE_ENUMERIC (the update sees a non-finite step and
  the 2nd stage stops at once) for every sketch kind and precision, and the next fit on the
  same context is correct;
* a forced tiny spin limit (slse_debug_spin_limit): the grid barrier of the FP64
  Householder QR gives up, the fit reports SLSE_ETIMEOUT, and with the limit restored the
  next fit on the same context reaches OLS."""
import numpy as np
import pytest

import workloads
from oracle import linalg
from tests.gpu_helpers import dev, torch_cuda

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def slse():
    torch_cuda()
    import paper_2509_06856_gb300 as m
    return m


def _clean_fit_reaches_ols(slse, prec="fp64"):
    p = workloads.gaussian(20000, 24, seed=9)
    X, Y = p["X"], p["Y"]
    if prec != "fp64":
        X, Y = X.astype(np.float32), Y.astype(np.float32)
    sched = slse.default_schedule(20000, 24, prec=prec, T=100, tol=1e-12 if prec == "fp64" else 1e-10)
    res = slse.fit(dev(X), dev(Y), sched, seed=1)
    bh = linalg.ols(np.asarray(X, np.float64), np.asarray(Y, np.float64))
    assert res.status == slse.OK
    assert np.linalg.norm(res.beta - bh) <= (1e-10 if prec == "fp64" else 1e-8) * np.linalg.norm(bh)


@pytest.mark.parametrize("prec,kind", [("fp64", "srht"), ("mixed_bf16", "srht"), ("mixed_bf16", "countsketch"),
                                       ("mixed_bf16", "gaussian"), ("fp64", "gaussian")])
def test_nan_rows_give_enumeric(slse, prec, kind):
    N, d = 1 << 14, 32
    p = workloads.gaussian(N, d, seed=4)
    X, Y = p["X"].copy(), p["Y"].copy()
    X[[5, 777, N - 1], 3] = np.nan
    if prec != "fp64":
        X, Y = X.astype(np.float32), Y.astype(np.float32)
    sched = slse.default_schedule(N, d, prec=prec, T=100, tol=1e-10, kind=kind)
    res = slse.fit(dev(X), dev(Y), sched, seed=2, raise_on_error=False)
    assert res.status == slse.ENUMERIC, slse.status_string(res.status)
    # the 2nd stage stops at its first non-finite step
    assert res.report["iters_stage2"] <= 1
    _clean_fit_reaches_ols(slse, prec)


def test_forced_spin_limit_gives_etimeout(slse):
    p = workloads.gaussian(20000, 64, seed=5)
    sched = slse.default_schedule(20000, 64, T=60, tol=1e-12)
    prev = slse.debug_spin_limit(1)
    try:
        res = slse.fit(dev(p["X"]), dev(p["Y"]), sched, seed=3, raise_on_error=False)
    finally:
        slse.debug_spin_limit(prev)
    assert res.status == slse.ETIMEOUT, slse.status_string(res.status)
    assert slse.debug_spin_limit(0) == 0
    _clean_fit_reaches_ols(slse)
