"""Shared helpers for the GPU parity tests (device upload, oracle wrappers)."""
import math

import numpy as np


def torch_cuda():
    import torch
    if not torch.cuda.is_available():
        import pytest
        pytest.skip("no CUDA device")
    return torch


def dev(a):
    torch = torch_cuda()
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def host(t):
    return t.detach().float().cpu().numpy().astype(np.float64) if str(t.dtype) == "torch.bfloat16" \
        else t.detach().cpu().numpy()


def padded(N):
    return 1 << max(0, int(N - 1).bit_length())


def sketch_entry(X, Y, D, P, sigma, m, s, cols):
    """Oracle value of sketch entries (row s, given columns) computed one by one from the
    definition sqrt(N'/m) * (H D P X_pad)[sigma[s]] / sqrt(N'), for sampled checks at full size."""
    Np = D.shape[0]
    N = X.shape[0]
    k = int(sigma[s])
    j = np.arange(Np, dtype=np.int64)
    sgn = np.where(np.bitwise_count(j & k) % 2 == 0, 1.0, -1.0) * D
    live = P < N
    w = sgn[live]
    src = P[live]
    out = []
    for c in cols:
        col = Y if c == X.shape[1] else X[:, c]
        out.append(float(np.dot(w, np.asarray(col[src], np.float64))) / math.sqrt(m))
    return np.array(out)
