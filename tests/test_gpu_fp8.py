"""GPU parity of the FP8 form of the sketch (E4M3 values, one power-of-two scale per 32-column
block of a row) against the FP64 oracle sketch, and fits on the FP8 form reaching OLS.  The
per-element bound is the E4M3 rounding (2^-4 relative, 2^-10 of the block scale below the
normal range) plus the BF16 rounding of the pass-1 intermediate."""
import numpy as np
import pytest

import workloads
from oracle import fp8 as ofp8
from oracle import linalg, sketch as osk
from tests.gpu_helpers import dev, host, torch_cuda

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def slse():
    torch_cuda()
    import paper_2509_06856_gb300 as m
    return m


@pytest.mark.parametrize("N,d,m", [(37, 3, 11), (500, 40, 300), (20000, 50, 6400), ((1 << 17) + 9, 64, 8192),
                                   ((1 << 20), 31, 1 << 14), (1 << 18, 512, 4096)])
def test_fp8_sketch_matches_oracle(slse, N, d, m):
    p = workloads.cfg3(N=N, d=d, seed=5)
    X, Y = p["X"], p["Y"]
    codes, kexp, SY = slse.sketch(dev(X), dev(Y), m, seed=4, prec="mixed_fp8")
    q = ofp8.decode_e4m3(host(codes).astype(np.int64))
    k = host(kexp).astype(np.int64) - 127
    assert not np.isnan(q).any()
    scale = np.repeat(np.ldexp(1.0, k), 32, axis=1)[:, :d]
    gx = q * scale
    ox, oy = osk.sketch(X.astype(np.float64), Y.astype(np.float64), m, 4)
    rms = np.sqrt((ox ** 2).mean(0))
    bound = 2.0 ** -4 * np.abs(ox) + 2.0 ** -10 * scale + 2.0 ** -6 * rms
    assert np.all(np.abs(gx - ox) <= bound)
    assert (np.abs(gx - ox) / rms).mean() < 2.0 ** -5
    # the block exponent is the smallest that fits the block: largest |code value| in [224, 448]
    for b in range(k.shape[1]):
        qa = np.abs(q[:, 32 * b:32 * (b + 1)]).max(axis=1)
        nz = qa > 0
        assert np.all((qa[nz] >= 224.0) & (qa[nz] <= 448.0))
    ey = np.abs(host(SY) - oy) / np.sqrt((oy ** 2).mean())
    assert ey.max() < 2.0 ** -5


@pytest.mark.parametrize("N,d", [(1 << 17, 64), ((1 << 16) + 333, 100), (5000, 40)])
def test_fit_fp8_reaches_ols_1e8(slse, N, d):
    p = workloads.cfg3(N=N, d=d, seed=6)
    X, Y = p["X"], p["Y"]
    sched = slse.default_schedule(N, d, prec="mixed_fp8", T=100, tol=1e-10)
    res = slse.fit(dev(X), dev(Y), sched, seed=2)
    bh = linalg.ols(X.astype(np.float64), Y.astype(np.float64))
    err = np.linalg.norm(res.beta - bh) / np.linalg.norm(bh)
    assert err <= 1e-8, err
