"""slse_fit with X and Y in host memory gives the same estimate, bit for bit, as with the
inputs in device memory (same seed; the arithmetic does not depend on where the inputs
start):

* pinned X with contiguous rows on a two-pass transform: the first SRHT pass reads X from
  host memory and stores the device copy as it goes;
* pageable host memory, pinned rows with a leading dimension above d, one-pass transform
  sizes and the CountSketch kind: X is copied to the device first."""
import numpy as np
import pytest

import workloads
from tests.gpu_helpers import dev, torch_cuda

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def slse():
    torch_cuda()
    import paper_2509_06856_gb300 as m
    return m


def _host(a, pinned, pad=0):
    torch = torch_cuda()
    t = torch.from_numpy(np.ascontiguousarray(a))
    if pad:
        w = torch.zeros((a.shape[0], a.shape[1] + pad), dtype=t.dtype, pin_memory=pinned)
        w[:, :a.shape[1]] = t
        return w[:, :a.shape[1]]
    return t.pin_memory() if pinned else t.clone()


@pytest.mark.parametrize("prec,kind,N,d", [("mixed_bf16", "srht", 20000, 50), ("fp64", "srht", (1 << 14) + 3, 24),
                                           ("mixed_bf16", "gaussian", 12000, 40),
                                           ("mixed_fp8", "srht", 1 << 15, 64),
                                           ("mixed_bf16", "countsketch", 20000, 50),
                                           ("mixed_bf16", "srht", 300, 6)])
def test_host_inputs_match_device_inputs(slse, prec, kind, N, d):
    p = workloads.cfg3(N=N, d=d, seed=21) if prec != "fp64" else workloads.gaussian(N, d, seed=21)
    X, Y = p["X"], p["Y"]
    if prec == "fp64":
        X, Y = X.astype(np.float64), Y.astype(np.float64)
    sched = slse.default_schedule(N, d, prec=prec, T=40, tol=1e-12, kind=kind)
    ref = slse.fit(dev(X), dev(Y), sched, seed=6)
    for pinned, pad in ((True, 0), (False, 0), (True, 4)):
        Xh = _host(X, pinned, pad)
        Yh = _host(Y, pinned)
        res = slse.fit(Xh, Yh, sched, seed=6)
        assert res.status == ref.status
        assert np.array_equal(res.beta, ref.beta), (pinned, pad)
        assert res.report["ms_copy_in"] > 0.0
