"""GPU parity of the mixed path's Hessian factor: the H-hat^{-1} that slse_fit uses (exported
through slse_trace.hinv_out) against the oracle's (R^T R)^{-1} from a Householder QR of the
same BF16 sketch rows, scaled by sqrt(N'/r) (Appendix, implementation details).  The GPU forms
it as the inverse of the exactly accumulated Gram matrix R^T R by the blocked sweep operator
in FP64."""
import numpy as np
import pytest

import workloads
from oracle import linalg
from tests.gpu_helpers import dev, host, padded, torch_cuda

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def slse():
    torch_cuda()
    import paper_2509_06856_gb300 as m
    return m


@pytest.mark.parametrize("N,d", [(1 << 15, 24), ((1 << 16) + 5, 100), (1 << 17, 256), (1 << 18, 512), (1 << 16, 33)])
def test_mixed_hessian_inverse_matches_oracle(slse, N, d):
    p = workloads.cfg3(N=N, d=d, seed=9)
    X, Y = p["X"], p["Y"]
    Xd, Yd = dev(X), dev(Y)
    sched = slse.default_schedule(N, d, prec="mixed_bf16", T=4)
    res = slse.fit(Xd, Yd, sched, seed=3, hinv=True)
    Np = padded(N)
    mK, r = sched.m[-1], sched.r
    assert mK + r <= Np
    # the fit stores the sampled rows of H D P X / sqrt(N') in BF16; slse_sketch with m = N'
    # rounds exactly the same values (scale sqrt(N'/m) = 1), in sampling order, so rows
    # mK .. mK + r are the fit's S-hat rows before their scale sqrt(N'/r)
    SX, _ = slse.sketch(Xd, Yd, Np, seed=3, prec="mixed_bf16")
    rows = host(SX)[mK:mK + r] * np.sqrt(Np / r)
    R = linalg.householder_r(rows)
    H = np.linalg.inv(R.T @ R)
    G = host(res.hinv)
    assert np.abs(G - H).max() <= 1e-9 * np.abs(H).max()
