"""The gradient entry point that allocates nothing (slse_grad_noalloc), for callers that
cannot allocate device memory when they need a gradient.  It must give the same result
as slse_grad, call after call, with its scratch taken from the library's fixed array.
Collected last so a failure here cannot hide the other tests' results."""
import numpy as np
import pytest

import workloads
from oracle import slse as osl
from tests.gpu_helpers import dev, host, torch_cuda

pytestmark = pytest.mark.gpu


def _bound(X, Y, beta):
    X = np.asarray(X, np.float64)
    return np.abs(X).T @ (np.abs(np.asarray(Y, np.float64)) + np.abs(X) @ np.abs(beta))


@pytest.mark.parametrize("prec,N,d", [("fp64", 20000, 64), ("fp64", (1 << 16) + 7, 512), ("mixed_bf16", 30001, 256),
                                      ("mixed_bf16", 4097, 50)])
def test_grad_noalloc_matches_grad_on_two_calls(prec, N, d):
    torch_cuda()
    import paper_2509_06856_gb300 as slse
    p = workloads.gaussian(N, d, seed=d) if prec == "fp64" else workloads.cfg3(N=N, d=d, seed=7)
    X, Y = p["X"], p["Y"]
    beta = p["beta_true"] * (1.0 + 1e-4)
    Xd, Yd = dev(X), dev(Y)
    ref = host(slse.grad(Xd, Yd, beta, prec=prec))
    first = host(slse.grad_noalloc(Xd, Yd, beta, prec=prec))
    second = host(slse.grad_noalloc(Xd, Yd, beta, prec=prec))
    if prec == "fp64":
        tol = 1e-13 * _bound(X, Y, beta)
    else:
        X64, Y64 = X.astype(np.float64), Y.astype(np.float64)
        tol = 4e-7 * (np.abs(X64).T @ np.abs(Y64 - X64 @ beta))
    np.testing.assert_array_less(np.abs(first - ref), tol + 1e-300)
    np.testing.assert_array_less(np.abs(second - ref), tol + 1e-300)
    assert np.array_equal(first, second)  # the shared scratch holds no state between calls
    go = osl.grad(np.asarray(X, np.float64), np.asarray(Y, np.float64), beta)
    np.testing.assert_array_less(np.abs(first - go), 2 * tol + 1e-300)


def test_host_gradient_output_rejected_by_both_entry_points():
    """A g_out in host memory is an argument error for slse_grad and slse_grad_noalloc
    alike (SLSE_EINVAL before any launch), never a kernel writing through a host address."""
    torch_cuda()
    import ctypes
    import paper_2509_06856_gb300 as slse
    p = workloads.cfg3(N=4096, d=32, seed=3)
    Xd, Yd = dev(p["X"]), dev(p["Y"])
    b = dev(np.zeros(32))
    g_host = np.zeros(32)
    prob = slse.problem(Xd, Yd)
    ptr = g_host.ctypes.data_as(ctypes.c_void_p)
    st = slse._lib.slse_grad(ctypes.byref(prob), b.data_ptr(), ptr, slse.PREC["mixed_bf16"], None, 0, None)
    assert st == slse.EINVAL
    st = slse._lib.slse_grad_noalloc(ctypes.byref(prob), b.data_ptr(), ptr, slse.PREC["mixed_bf16"], None)
    assert st == slse.EINVAL
    assert not g_host.any()
