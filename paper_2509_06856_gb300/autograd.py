"""torch.autograd binding of the estimator: beta-hat = slse_fit(X, Y), with the input
gradients from slse_solve_normal (w = (X^T X)^{-1} dL/d(beta-hat), preconditioned by the
fit's own H-hat^{-1}) and slse_ols_vjp (one pass for dL/dX and dL/dY).  Argument
marshalling only: every step runs in the CUDA library."""
import dataclasses

import torch

from . import default_schedule, fit, ols_vjp, solve_normal


class _OLS(torch.autograd.Function):
    @staticmethod
    def forward(ctx, X, Y, schedule, seed, adjoint_tol):
        res = fit(X, Y, schedule, seed=seed, hinv=True)
        beta = torch.from_numpy(res.beta).to(X.device)
        ctx.save_for_backward(X, Y, beta, res.hinv)
        ctx.schedule = dataclasses.replace(schedule, tol=adjoint_tol)
        return beta

    @staticmethod
    def backward(ctx, gbeta):
        X, Y, beta, H = ctx.saved_tensors
        w, _ = solve_normal(X, H, gbeta, ctx.schedule)
        dX, dY = ols_vjp(X, Y, beta, w)
        return dX, dY, None, None, None


def ols(X, Y, schedule=None, seed: int = 0, adjoint_tol: float | None = None):
    """Differentiable least-squares estimate by SLSE-FRS.  X: device N x d (float64, or
    float32 with the mixed path), Y: device N.  Returns beta-hat (float64, device).
    adjoint_tol: relative-step tolerance of the backward solve (default 1e-12 in FP64,
    1e-9 on the mixed path, whose passes resolve the solution to about that level)."""
    fp64 = X.dtype == torch.float64
    if schedule is None:
        schedule = default_schedule(X.shape[0], X.shape[1], prec="fp64" if fp64 else "mixed_bf16", T=100,
                                    tol=1e-12 if fp64 else 1e-10)
    if adjoint_tol is None:
        adjoint_tol = 1e-12 if schedule.prec == "fp64" else 1e-9
    return _OLS.apply(X, Y, schedule, seed, adjoint_tol)
