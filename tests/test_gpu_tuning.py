"""GPU runs of the SLSE-FRS-tuning schedule (Sec. 5, sketch size tuning): iterates match the
oracle's on the same seed, and the fit reaches OLS."""
import numpy as np
import pytest

import workloads
from oracle import linalg, slse as osl
from tests.gpu_helpers import dev, host, torch_cuda

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def slse():
    torch_cuda()
    import paper_2509_06856_gb300 as m
    return m


def test_tuning_schedule_iterates_match_oracle(slse):
    N, d = 1 << 15, 16
    p = workloads.gaussian(N, d, seed=3)
    X, Y = p["X"], p["Y"]
    s = slse.tuning_schedule(N, d, T=40)
    assert s.a == [3] * len(s.m) and s.m[0] == 16 * d
    res = slse.fit(dev(X), dev(Y), s, seed=5, trace_cap=40)
    o = osl.slse_fit(X, Y, osl.tuning_schedule(N, d, T=40), seed=5, trace=True)
    bh = linalg.ols(X, Y)
    for t, (g, r) in enumerate(zip(host(res.beta_hist), o.trace)):
        assert np.linalg.norm(g - r) <= 1e-10 * np.linalg.norm(bh), t


@pytest.mark.parametrize("prec", ["fp64", "mixed_bf16"])
def test_tuning_schedule_reaches_ols(slse, prec):
    N, d = 1 << 18, 64
    p = workloads.paper(N, d, kappa=1e4, sigma2=1e-8, seed=1) if prec == "fp64" else workloads.cfg3(N=N, d=d, seed=2)
    X, Y = p["X"], p["Y"]
    res = slse.fit(dev(X), dev(Y), slse.tuning_schedule(N, d, prec=prec, T=100, tol=1e-13 if prec == "fp64" else 1e-10),
                   seed=1)
    bh = linalg.ols(np.asarray(X, np.float64), np.asarray(Y, np.float64))
    assert np.linalg.norm(res.beta - bh) <= (1e-10 if prec == "fp64" else 1e-8) * np.linalg.norm(bh)
