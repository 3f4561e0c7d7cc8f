"""Seeded synthetic inputs for the SLSE-FRS workloads.

This module only draws data: it holds none of the method's arithmetic (no sketch,
no gradient, no solve).  Both the CUDA path (tests, bench) and the CPU oracle read
the arrays it returns, so both sides see identical bits.

Every generator is deterministic for a given ``seed``: rows are produced in
fixed-size blocks, each block drawing from its own ``numpy.random.Generator``
(PCG64) seeded by ``SeedSequence(seed, spawn_key=(tag, block))``.  The result
therefore does not depend on the number of worker threads.

Workloads (the paper's experiments are all synthetic, Sec. 5 first paragraph):

* ``paper``  - Sec. 5 recipe: X = G diag(s), s log-spaced from 1 to 1/kappa,
  beta ~ N(0, I), noise variance sigma2 (the paper uses 1e-8).
* ``cfg1``   - N=20000, d=50, FP64, X_ij ~ N(0,1), beta ~ N(0,I), noise N(0, 0.1^2).
* ``cfg2``   - N=2^20, d=256, FP64, X = G diag(s) V^T with s log-spaced 1 -> 1e-4
  (cond ~ 1e4) and V Haar-orthogonal (QR of a Gaussian with the sign fix of
  Mezzadri 2007), beta ~ N(0,I), noise sd 1e-2.
* ``cfg3``   - N=2^22, d=512, stored FP32, rows N(0, Sigma) with
  Sigma_ij = 0.5^|i-j| drawn by the exact AR(1) recursion
  x_1 = z_1, x_j = 0.5 x_{j-1} + sqrt(0.75) z_j; beta ~ N(0,I); noise sd 0.1.
* ``cfg4``   - N=2^24, d=256, stored FP32, i.i.d. Student-t(3) entries
  (z / sqrt(chi2_3 / 3)) with 0.1 % of the rows scaled by 100 (high leverage),
  beta ~ U(-1, 1), noise sd 1.
* ``cfg5``   - N=2^21, d=128, stored FP32, X ~ N(0,1), Y = X beta* + N(0, 0.05^2).
* ``cfg5fd`` - the N=2000, d=10 FP64 copy of cfg5 used for finite differences.
"""
from __future__ import annotations

import math
import os
from concurrent.futures import ThreadPoolExecutor

import numpy as np

BLOCK_ROWS = 1 << 16

# name -> (N, d, storage dtype, default seed)
CONFIGS = {
    "cfg1": (20000, 50, np.float64, 0),
    "cfg2": (1 << 20, 256, np.float64, 1002),
    "cfg3": (1 << 22, 512, np.float32, 1003),
    "cfg4": (1 << 24, 256, np.float32, 1004),
    "cfg5": (1 << 21, 128, np.float32, 1005),
    "cfg5fd": (2000, 10, np.float64, 1005),
}


def _rng(seed: int, tag: int, block: int) -> np.random.Generator:
    return np.random.Generator(np.random.PCG64(np.random.SeedSequence(seed, spawn_key=(tag, block))))


def _threads(threads: int | None) -> int:
    if threads is not None:
        return max(1, threads)
    return max(1, min(32, os.cpu_count() or 1))


def _fill_blocks(N: int, fn, threads: int | None) -> None:
    nblk = (N + BLOCK_ROWS - 1) // BLOCK_ROWS
    if nblk == 1 or _threads(threads) == 1:
        for b in range(nblk):
            fn(b, b * BLOCK_ROWS, min(N, (b + 1) * BLOCK_ROWS))
        return
    with ThreadPoolExecutor(_threads(threads)) as ex:
        list(ex.map(lambda b: fn(b, b * BLOCK_ROWS, min(N, (b + 1) * BLOCK_ROWS)), range(nblk)))


def _finish(X: np.ndarray, Y: np.ndarray, beta: np.ndarray, name: str, seed: int, **meta) -> dict:
    return {"X": X, "Y": Y, "beta_true": beta, "name": name, "seed": seed,
            "N": X.shape[0], "d": X.shape[1], **meta}


def gaussian(N: int, d: int, *, seed: int = 0, noise_sd: float = 0.1,
             dtype=np.float64, threads: int | None = None) -> dict:
    """X_ij ~ N(0,1), beta ~ N(0,I), Y = X beta + N(0, noise_sd^2)."""
    beta = _rng(seed, 0, 0).standard_normal(d)
    X = np.empty((N, d), dtype=dtype)
    Y = np.empty(N, dtype=dtype)

    def blk(b, lo, hi):
        g = _rng(seed, 1, b)
        x = g.standard_normal((hi - lo, d))
        X[lo:hi] = x
        Y[lo:hi] = x @ beta + noise_sd * g.standard_normal(hi - lo)

    _fill_blocks(N, blk, threads)
    return _finish(X, Y, beta, "gaussian", seed, noise_sd=noise_sd)


def paper(N: int, d: int, *, kappa: float = 1e4, sigma2: float = 1e-8, seed: int = 0,
          threads: int | None = None) -> dict:
    """Sec. 5 recipe: X = G diag(s) with s log-spaced 1 -> 1/kappa (the paper's
    'predetermined' column scales), beta ~ N(0,I), noise variance sigma2."""
    s = np.logspace(0.0, -math.log10(kappa), d)
    beta = _rng(seed, 0, 0).standard_normal(d)
    X = np.empty((N, d))
    Y = np.empty(N)

    def blk(b, lo, hi):
        g = _rng(seed, 1, b)
        x = g.standard_normal((hi - lo, d)) * s
        X[lo:hi] = x
        Y[lo:hi] = x @ beta + math.sqrt(sigma2) * g.standard_normal(hi - lo)

    _fill_blocks(N, blk, threads)
    return _finish(X, Y, beta, "paper", seed, kappa=kappa, sigma2=sigma2)


def haar_orthogonal(d: int, seed: int) -> np.ndarray:
    """Haar-distributed orthogonal d x d matrix: QR of a Gaussian matrix with the
    columns of Q multiplied by sign(diag(R)) (Mezzadri 2007)."""
    A = _rng(seed, 7, 0).standard_normal((d, d))
    Q, R = np.linalg.qr(A)
    return Q * np.sign(np.diag(R))


def cfg2(N: int = 1 << 20, d: int = 256, *, seed: int = 1002, cond: float = 1e4,
         noise_sd: float = 1e-2, threads: int | None = None) -> dict:
    s = np.logspace(0.0, -math.log10(cond), d)
    V = haar_orthogonal(d, seed)
    SVt = s[:, None] * V.T
    beta = _rng(seed, 0, 0).standard_normal(d)
    X = np.empty((N, d))
    Y = np.empty(N)

    def blk(b, lo, hi):
        g = _rng(seed, 1, b)
        x = g.standard_normal((hi - lo, d)) @ SVt
        X[lo:hi] = x
        Y[lo:hi] = x @ beta + noise_sd * g.standard_normal(hi - lo)

    _fill_blocks(N, blk, threads)
    return _finish(X, Y, beta, "cfg2", seed, cond=cond, noise_sd=noise_sd)


def cfg3(N: int = 1 << 22, d: int = 512, *, seed: int = 1003, rho: float = 0.5,
         noise_sd: float = 0.1, dtype=np.float32, threads: int | None = None) -> dict:
    beta = _rng(seed, 0, 0).standard_normal(d)
    X = np.empty((N, d), dtype=dtype)
    Y = np.empty(N, dtype=dtype)
    c = math.sqrt(1.0 - rho * rho)

    def blk(b, lo, hi):
        g = _rng(seed, 1, b)
        z = g.standard_normal((d, hi - lo))   # column-major draw: the recursion runs along d
        for j in range(1, d):
            z[j] = rho * z[j - 1] + c * z[j]
        x = z.T
        X[lo:hi] = x
        Y[lo:hi] = x @ beta + noise_sd * g.standard_normal(hi - lo)

    _fill_blocks(N, blk, threads)
    return _finish(X, Y, beta, "cfg3", seed, rho=rho, noise_sd=noise_sd)


def cfg4(N: int = 1 << 24, d: int = 256, *, seed: int = 1004, frac_lev: float = 1e-3,
         lev_scale: float = 100.0, noise_sd: float = 1.0, dtype=np.float32,
         threads: int | None = None) -> dict:
    beta = _rng(seed, 0, 0).uniform(-1.0, 1.0, d)
    n_lev = int(round(frac_lev * N))
    lev_rows = np.sort(_rng(seed, 2, 0).choice(N, size=n_lev, replace=False))
    X = np.empty((N, d), dtype=dtype)
    Y = np.empty(N, dtype=dtype)

    def blk(b, lo, hi):
        g = _rng(seed, 1, b)
        z = g.standard_normal((hi - lo, d))
        chi = g.chisquare(3.0, (hi - lo, d))
        x = z / np.sqrt(chi / 3.0)
        sel = lev_rows[(lev_rows >= lo) & (lev_rows < hi)] - lo
        x[sel] *= lev_scale
        X[lo:hi] = x
        Y[lo:hi] = x @ beta + noise_sd * g.standard_normal(hi - lo)

    _fill_blocks(N, blk, threads)
    return _finish(X, Y, beta, "cfg4", seed, lev_rows=lev_rows, noise_sd=noise_sd)


def cfg5(N: int = 1 << 21, d: int = 128, *, seed: int = 1005, dtype=np.float32,
         threads: int | None = None) -> dict:
    out = gaussian(N, d, seed=seed, noise_sd=0.05, dtype=dtype, threads=threads)
    out["name"] = "cfg5"
    return out


def cfg1(seed: int = 0, **kw) -> dict:
    out = gaussian(20000, 50, seed=seed, noise_sd=0.1, **kw)
    out["name"] = "cfg1"
    return out


def make(name: str, **kw) -> dict:
    """Build a named workload with its default sizes (overridable by keyword)."""
    if name == "cfg1":
        return cfg1(**kw)
    if name == "cfg2":
        return cfg2(**kw)
    if name == "cfg3":
        return cfg3(**kw)
    if name == "cfg4":
        return cfg4(**kw)
    if name == "cfg5":
        return cfg5(**kw)
    if name == "cfg5fd":
        kw.setdefault("seed", 1005)
        out = gaussian(2000, 10, noise_sd=0.05, **kw)
        out["name"] = "cfg5fd"
        return out
    raise KeyError(name)
