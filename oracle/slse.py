"""SLSE-FRS itself (Algorithm 2 of the paper), plus its schedule helpers, in FP64.

* ``default_schedule``: the experimental settings of Sec. 5 (first subsection
  preamble): Hessian-sketch size r = 6d, eta = d/r, mu = (1 - eta)^2, sketch sizes
  m_1 = 8d doubling up to m_K = N/2 (Sec. 3: m_{i+1}/m_i = 2, K = log2(N/m_1)),
  a_i = 2 inner iterations (Sec. 5.1), T = 100 total iterations.
* ``ai_bound``: the lower bound of Theorem 4.3,
  a_i >= log_3[((1 + omega) r(i-1, i) + 1) / omega],  r(i-1,i) = sqrt((m_i - d)/(m_{i-1} - d)).
* ``grad``: g = X^T (Y - X beta).  This is minus the paper's gradient
  nabla f = X^T (X beta - Y) (Sec. 1); the update below adds mu H^{-1} g accordingly.
* ``mihs_step``: the M-IHS update of Eqs. (7) and (8) (Sec. 3),
  beta_{t+1} = beta_t + mu H-hat^{-1} g_t + eta (beta_t - beta_{t-1}),
  with H-hat^{-1} v = R^{-1} R^{-T} v from S-hat X = Q R (Appendix, implementation details).
* ``slse_fit``: Algorithm 2 step by step: one transform of [X|Y], nested prefixes of
  the sampled rows for the K sketched subproblems (a_i M-IHS steps each, 1st stage),
  then full-data M-IHS steps (2nd stage).  ``kind="countsketch"`` runs the same
  iteration on the CountSketch family of ``oracle.countsketch`` (the SLSE-FRS-CS
  experiment of Sec. 5): S_i X is the m_i-bucket sketch (no scale factor, since
  E[S^T S] = I), S-hat X the independent r-bucket sketch.  ``kind="gaussian"`` keeps
  the SRHT subproblems and takes S-hat X from the r x N Gaussian sketch of
  ``oracle.gaussian`` (Sec. 2) instead of the sampled SRHT rows.

Readings taken where the paper is silent:
* beta_0 = 0 (Thm 4.2 allows any beta_0).
* Momentum follows the listing of Algorithm 2: one global iteration counter t, so
  beta_{t-1} carries across subproblems and into the 2nd stage (default).
  ``momentum_reset=True`` restarts it at every subproblem and at the 2nd stage,
  beta_{-1}^i = beta_0^i, as the proof of Theorem 4.1 does.
* The 2nd stage stops early when ||beta_{t+1} - beta_t|| <= tol (1 - rho)/rho ||beta_{t+1}||
  with rho = sqrt(d/r) (the M-IHS rate quoted in Sec. 1); tol <= 0 runs to T.
  T counts all iterations of both stages.
"""
import math
from dataclasses import dataclass, field

import numpy as np

from . import countsketch as cs
from . import gaussian as gs
from . import sketch as sk
from .linalg import householder_r, solve_lower, solve_upper


@dataclass
class Schedule:
    m: list            # sketch sizes m_1 < ... < m_K
    a: list            # inner iterations a_i
    r: int             # Hessian sketch size
    mu: float
    eta: float
    T: int = 100
    tol: float = 0.0
    momentum_reset: bool = False
    kind: str = "srht"   # or "countsketch", or "gaussian" (SRHT subproblems, Gaussian S-hat)

    @property
    def K(self):
        return len(self.m)


def default_schedule(N: int, d: int, T: int = 100, tol: float = 0.0, a: int = 2,
                     kind: str = "srht") -> Schedule:
    """Sec. 5 settings.  For the CountSketch family the sizes must be powers of two, so
    m_1 = 8d is rounded up to the next power of two."""
    Np = sk.padded_size(N)
    r = 6 * d
    eta = d / r
    mu = (1.0 - eta) ** 2
    mi = 8 * d
    if kind == "countsketch":
        mi = sk.padded_size(mi)
    m = []
    while mi <= Np // 2:
        m.append(mi)
        mi *= 2
    return Schedule(m=m, a=[a] * len(m), r=r, mu=mu, eta=eta, T=T, tol=tol, kind=kind)


def tuning_schedule(N: int, d: int, T: int = 100, tol: float = 0.0, kind: str = "srht") -> Schedule:
    """The SLSE-FRS-tuning schedule (Sec. 5, sketch size tuning): a few small sketched
    problems and one large one, a_i = 3.  The paper's sizes for d = 2^6 are 2^10 .. 2^16
    and 2^19, i.e. 16d 2^j (j = 0..6) and 8192d; sizes above N'/2 are dropped.  r, eta and mu
    as in the default schedule."""
    base = default_schedule(N, d, T=T, tol=tol, kind=kind)
    Np = sk.padded_size(N)
    m = [16 * d * 2 ** j for j in range(7)] + [8192 * d]
    if kind == "countsketch":
        m = [sk.padded_size(v) for v in m]
    m = sorted(set(v for v in m if v <= Np // 2))
    return Schedule(m=m, a=[3] * len(m), r=base.r, mu=base.mu, eta=base.eta, T=T, tol=tol, kind=kind)


def ai_bound(omega: float, m_prev: float, m_i: float, d: float) -> float:
    """Theorem 4.3 lower bound on a_i (i >= 2)."""
    rr = math.sqrt((m_i - d) / (m_prev - d))
    return math.log(((1.0 + omega) * rr + 1.0) / omega, 3.0)


def ai_bound_limit(omega: float) -> float:
    """alpha of Theorem 4.4, log_3{[1 + (1 + omega)/sqrt(2)]/omega}: the bound's value
    with the ratio sqrt((m_{i-1} - d)/(m_i - d)) -> 1/sqrt(2) that the proof of
    Theorem 4.4 uses (the reciprocal of the ratio in the statement of Theorem 4.3)."""
    return math.log((1.0 + (1.0 + omega) / math.sqrt(2.0)) / omega, 3.0)


def grad(X, Y, beta, block_rows: int = 1 << 16) -> np.ndarray:
    """g = X^T (Y - X beta) in FP64 (row blocks keep the FP64 copy of X small)."""
    N, d = X.shape
    g = np.zeros(d)
    beta = np.asarray(beta, np.float64)
    for lo in range(0, N, block_rows):
        Xb = np.asarray(X[lo:lo + block_rows], np.float64)
        rb = np.asarray(Y[lo:lo + block_rows], np.float64) - Xb @ beta
        g += Xb.T @ rb
    return g


def hinv_apply(R: np.ndarray, v: np.ndarray) -> np.ndarray:
    """H-hat^{-1} v = R^{-1} (R^{-T} v)."""
    return solve_upper(R, solve_lower(R.T, v))


def mihs_step(beta, beta_prev, g, R, mu, eta):
    """One M-IHS update; returns (beta_next, beta)."""
    return beta + mu * hinv_apply(R, g) + eta * (beta - beta_prev), beta


@dataclass
class FitResult:
    beta: np.ndarray
    iters_stage1: int
    iters_stage2: int
    converged: bool
    trace: list = field(default_factory=list)
    R: np.ndarray = None


def slse_fit(X, Y, sched: Schedule, seed: int, trace: bool = False,
             sketch_override=None) -> FitResult:
    """Algorithm 2 on the sketches drawn from ``seed``.

    ``sketch_override``: optional (ZX, ZY) full transformed data (all N' rows,
    already divided by sqrt(N')), used by tests to run the iteration on a
    modified sketch.
    """
    X = np.asarray(X)
    N, d = X.shape
    Np = sk.padded_size(N)
    if sched.kind == "countsketch":
        def subproblem(m):
            SX, SY = cs.countsketch(X, Y, m, seed)
            return SX, SY, 1.0
        R = householder_r(cs.countsketch_hat(X, Y, sched.r, seed)[0])
    else:
        D, P, sigma = sk.draws(Np, seed)
        if sketch_override is None:
            ZX = sk.hdp(X, D, P)
            ZY = sk.hdp(Y, D, P)
        else:
            ZX, ZY = sketch_override
        mK = sched.m[-1] if sched.K else 0
        if sched.kind == "gaussian":
            R = householder_r(gs.gaussian_sketch(X, Y, sched.r, seed)[0])
        else:
            h0, h1 = sk.hessian_rows(Np, mK, sched.r)
            SX_hat = math.sqrt(Np / sched.r) * ZX[sigma[h0:h1]]
            R = householder_r(SX_hat)

        def subproblem(m):
            # S_i X = sqrt(N'/m) U with U the first m sampled rows; the gradient of the
            # sketched problem is (N'/m) U^T (V - U beta)
            return ZX[sigma[:m]], ZY[sigma[:m]], Np / m

    beta = np.zeros(d)
    beta_prev = beta.copy()
    hist = []
    t = 0
    for m, a in zip(sched.m, sched.a):
        U, V, scale = subproblem(m)
        if sched.momentum_reset:
            beta_prev = beta.copy()
        for _ in range(a):
            if t >= sched.T:
                break
            g = scale * (U.T @ (V - U @ beta))
            beta, beta_prev = mihs_step(beta, beta_prev, g, R, sched.mu, sched.eta)
            t += 1
            if trace:
                hist.append(beta.copy())
    it1 = t
    if sched.momentum_reset:
        beta_prev = beta.copy()
    rho = math.sqrt(d / sched.r)
    thr = sched.tol * (1.0 - rho) / rho
    converged = sched.tol <= 0.0
    while t < sched.T:
        g = grad(X, Y, beta)
        beta, beta_prev = mihs_step(beta, beta_prev, g, R, sched.mu, sched.eta)
        t += 1
        if trace:
            hist.append(beta.copy())
        if sched.tol > 0.0 and np.linalg.norm(beta - beta_prev) <= thr * np.linalg.norm(beta):
            converged = True
            break
    return FitResult(beta=beta, iters_stage1=it1, iters_stage2=t - it1, converged=converged,
                     trace=hist, R=R)
