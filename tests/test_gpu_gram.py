"""The Gram matrix of the BF16-rounded data (slse_gram), the Hessian term the mixed 2nd stage's
correction form uses between exact passes: against the same product formed on the CPU in FP64
from the BF16 rounding of X (round to nearest even, PyTorch's CPU cast), at sizes with a ragged
last chunk of rows, d below, at and between multiples of the 128-column tiles."""
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
    assert np.array_equal(G, G.T) or np.max(np.abs(G - G.T) / scale) <= 1e-6


def test_gram_is_deterministic():
    torch_cuda()
    import paper_2509_06856_gb300 as slse
    Xd = dev(workloads.cfg3(N=50000, d=96, seed=3)["X"])
    assert np.array_equal(host(slse.gram(Xd)), host(slse.gram(Xd)))
