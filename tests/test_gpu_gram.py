"""The Gram matrix of the BF16-rounded data (slse_gram), the Hessian term the mixed 2nd stage's
correction form uses between exact passes: against the same product formed on the CPU in FP64
from the BF16 rounding of X (round to nearest even, PyTorch's CPU cast), at sizes with a ragged
last chunk of rows, d below, at and between multiples of the 128-column tiles.  X with d and the
row stride multiples of 4 and 16-byte aligned rows is read directly (rounded on chip); any other X
(d = 129, a view one column in) is packed to BF16 first: both ways are covered."""
import numpy as np
import pytest

import workloads
from tests.gpu_helpers import dev, host, torch_cuda

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("N,d", [(4096 + 7, 64), ((1 << 16) + 33, 200), (1 << 17, 512), (200, 128), (70000, 129), (1 << 19, 256)])
def test_gram_matches_cpu_product_of_bf16_rows(N, d):
    torch = torch_cuda()
    import paper_2509_06856_gb300 as slse
    X = workloads.cfg3(N=N, d=d, seed=11)["X"]
    G = host(slse.gram(dev(X)))
    Xb = torch.from_numpy(X).bfloat16().double().numpy()
    ref = Xb.T @ Xb
    scale = np.abs(Xb).T @ np.abs(Xb)
    # BF16 products are exact in FP32; the FP32 sums over a range of rows (at most 8192 rows) and
    # the FP64 sum of the ranges stay far inside 1e-4 of sum |x_i x_j|
    err = np.abs(G - ref) / scale
    print(f"N={N} d={d}: max error / sum|x x| = {err.max():.2e}")
    assert np.all(err <= 1e-4)
    assert np.array_equal(G, G.T)  # the upper triangle is formed and mirrored


@pytest.mark.parametrize("N,d,off", [(30011, 200, 4), (30011, 200, 1), (20000, 128, 4)])
def test_gram_of_row_strided_views(N, d, off):
    """X a view of a wider buffer (row stride d + 4): starting 4 columns in keeps the rows 16-byte
    aligned (direct path), 1 column in does not (packed path)."""
    torch = torch_cuda()
    import paper_2509_06856_gb300 as slse
    buf = workloads.cfg3(N=N, d=d + 4, seed=13)["X"]
    Xv = dev(buf)[:, off:off + d]
    assert Xv.stride(0) == d + 4
    G = host(slse.gram(Xv))
    Xb = torch.from_numpy(np.ascontiguousarray(buf[:, off:off + d])).bfloat16().double().numpy()
    err = np.abs(G - Xb.T @ Xb) / (np.abs(Xb).T @ np.abs(Xb))
    print(f"N={N} d={d} offset {off}: max error / sum|x x| = {err.max():.2e}")
    assert np.all(err <= 1e-4)
    assert np.array_equal(G, G.T)


@pytest.mark.parametrize("N,d", [(4096 + 40, 64), (65536 + 17, 200), (1 << 17, 512), (70000, 384), (30000, 129),
                                 (200, 128)])
def test_gram_of_bf16_rows(N, d):
    """BF16 X: the tensor cores read the row-major BF16 tiles directly (MN-major operands, 128-byte
    swizzle, boxes multicast within a cluster); against the FP64 product of the same BF16 values."""
    torch = torch_cuda()
    import paper_2509_06856_gb300 as slse
    X = workloads.cfg3(N=N, d=d, seed=17)["X"]
    ld = (d + 7) // 8 * 8
    buf = torch.zeros((N, ld), dtype=torch.bfloat16)
    buf[:, :d] = torch.from_numpy(X).bfloat16()
    Xd = buf.cuda()[:, :d]
    G = host(slse.gram(Xd))
    Xb = buf[:, :d].double().numpy()
    err = np.abs(G - Xb.T @ Xb) / (np.abs(Xb).T @ np.abs(Xb))
    print(f"BF16 N={N} d={d}: max error / sum|x x| = {err.max():.2e}")
    assert np.all(err <= 1e-4)
    assert np.array_equal(G, G.T)


def test_gram_is_deterministic():
    torch_cuda()
    import paper_2509_06856_gb300 as slse
    Xd = dev(workloads.cfg3(N=50000, d=96, seed=3)["X"])
    assert np.array_equal(host(slse.gram(Xd)), host(slse.gram(Xd)))
