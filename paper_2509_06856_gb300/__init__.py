"""GB300 (sm_103a) SLSE-FRS: Python binding over the C ABI declared in include/slse.h.

Argument marshalling only: every step of the method runs in the CUDA kernels of
``libslse.so``.  PyTorch is used for device memory and the current CUDA stream.
The library must be built first (``python paper_2509_06856_gb300/build.py`` or
``__graft_entry__.build()``); importing this package without it raises ImportError.

Paper: "Sequential Least-Squares Estimators with Fast Randomized Sketching for
Linear Statistical Models" (arXiv 2509.06856), Algorithm 2.
"""
from __future__ import annotations

import ctypes
import math
import os
from dataclasses import dataclass, field

import numpy as np

LIB_PATH = os.path.join(os.path.dirname(os.path.abspath(__file__)), "libslse.so")

if not os.path.exists(LIB_PATH):
    raise ImportError(f"libslse.so is not built ({LIB_PATH}); run python paper_2509_06856_gb300/build.py")

_lib = ctypes.CDLL(LIB_PATH)

# ----------------------------------------------------------------------------- C types
OK, EINVAL, ENOMEM, ECUDA, ENOTCONV, ENUMERIC, ETIMEOUT = range(7)
F64, F32, BF16 = 0, 1, 2
SRHT, COUNTSKETCH, GAUSSIAN, COUNTSKETCH_HAT = 0, 1, 2, 3
KIND = {"srht": SRHT, "countsketch": COUNTSKETCH, "countsketch_hat": COUNTSKETCH_HAT, "gaussian": GAUSSIAN}
PREC = {"fp64": 0, "mixed_bf16": 1, "mixed_fp8": 2}
STAGE2 = {"full": 0, "correction": 1}
OP_FIT, OP_SKETCH, OP_GRAD, OP_DRAWS, OP_QR, OP_GRAM = range(6)


class CProblem(ctypes.Structure):
    _fields_ = [("N", ctypes.c_int64), ("d", ctypes.c_int32), ("dtype", ctypes.c_int32),
                ("X", ctypes.c_void_p), ("ldx", ctypes.c_int64), ("Y", ctypes.c_void_p)]


class CSchedule(ctypes.Structure):
    _fields_ = [("K", ctypes.c_int32), ("m", ctypes.POINTER(ctypes.c_int64)), ("a", ctypes.POINTER(ctypes.c_int32)),
                ("r", ctypes.c_int64), ("mu", ctypes.c_double), ("eta", ctypes.c_double), ("T", ctypes.c_int32),
                ("tol", ctypes.c_double), ("kind", ctypes.c_int32), ("prec", ctypes.c_int32),
                ("momentum_reset", ctypes.c_int32), ("stage2", ctypes.c_int32)]


class CReport(ctypes.Structure):
    _fields_ = [("ms_copy_in", ctypes.c_double), ("ms_draws", ctypes.c_double), ("ms_sketch", ctypes.c_double),
                ("ms_qr", ctypes.c_double), ("ms_stage1", ctypes.c_double), ("ms_stage2", ctypes.c_double),
                ("ms_total", ctypes.c_double), ("ms_srht_pass1", ctypes.c_double), ("ms_srht_pass2", ctypes.c_double),
                ("ms_grad2", ctypes.c_double), ("n_grad2", ctypes.c_int32), ("kernels", ctypes.c_int32),
                ("iters_stage1", ctypes.c_int32), ("iters_stage2", ctypes.c_int32),
                ("final_rel_step", ctypes.c_double), ("bytes_moved", ctypes.c_double),
                ("bytes_grad2", ctypes.c_double), ("rebases", ctypes.c_int32), ("status", ctypes.c_int32),
                ("ms_corr", ctypes.c_double), ("n_corr", ctypes.c_int32), ("stage2_full", ctypes.c_int32),
                ("ms_gram", ctypes.c_double), ("flops_gram", ctypes.c_double), ("bytes_gram", ctypes.c_double)]


class CTrace(ctypes.Structure):
    _fields_ = [("beta_hist", ctypes.c_void_p), ("ms_hist", ctypes.POINTER(ctypes.c_float)),
                ("cap", ctypes.c_int32), ("count", ctypes.c_int32), ("hinv_out", ctypes.c_void_p)]


_vp, _sz, _i32, _i64, _u64 = ctypes.c_void_p, ctypes.c_size_t, ctypes.c_int32, ctypes.c_int64, ctypes.c_uint64
_lib.slse_workspace_size.restype = _sz
_lib.slse_workspace_size.argtypes = [ctypes.POINTER(CProblem), ctypes.POINTER(CSchedule), _i32, _i64]
_lib.slse_fit.restype = _i32
_lib.slse_fit.argtypes = [ctypes.POINTER(CProblem), ctypes.POINTER(CSchedule), _u64, ctypes.POINTER(ctypes.c_double),
                          ctypes.POINTER(CReport), ctypes.POINTER(CTrace), _vp, _sz, _vp]
_lib.slse_sketch.restype = _i32
_lib.slse_sketch.argtypes = [ctypes.POINTER(CProblem), _i32, _i32, _u64, _i64, _vp, _i64, _vp, _vp, _sz, _vp]
_lib.slse_grad.restype = _i32
_lib.slse_grad.argtypes = [ctypes.POINTER(CProblem), _vp, _vp, _i32, _vp, _sz, _vp]
_lib.slse_gram.restype = _i32
_lib.slse_gram.argtypes = [ctypes.POINTER(CProblem), _vp, _vp, _sz, _vp]
_lib.slse_grad_noalloc.restype = _i32
_lib.slse_grad_noalloc.argtypes = [ctypes.POINTER(CProblem), _vp, _vp, _i32, _vp]
_lib.slse_draws.restype = _i32
_lib.slse_draws.argtypes = [_i64, _u64, _vp, _vp, _vp, _vp, _sz, _vp]
_lib.slse_qr.restype = _i32
_lib.slse_qr.argtypes = [_vp, _i64, _i32, _i64, _vp, _vp, _vp, _sz, _vp]
_lib.slse_default_schedule.restype = _i32
_lib.slse_default_schedule.argtypes = [_i64, _i32, ctypes.POINTER(CSchedule), ctypes.POINTER(ctypes.c_int64),
                                       ctypes.POINTER(ctypes.c_int32), _i32]
_lib.slse_default_schedule_for.restype = _i32
_lib.slse_default_schedule_for.argtypes = [_i64, _i32, _i32, ctypes.POINTER(CSchedule), ctypes.POINTER(ctypes.c_int64),
                                           ctypes.POINTER(ctypes.c_int32), _i32]
_lib.slse_solve_normal.restype = _i32
_lib.slse_solve_normal.argtypes = [ctypes.POINTER(CProblem), _vp, _vp, _vp, ctypes.POINTER(CSchedule),
                                   ctypes.POINTER(CReport), _vp, _sz, _vp]
_lib.slse_solve_normal_workspace.restype = _sz
_lib.slse_solve_normal_workspace.argtypes = [ctypes.POINTER(CProblem), _i32]
_lib.slse_ols_vjp.restype = _i32
_lib.slse_ols_vjp.argtypes = [ctypes.POINTER(CProblem), _vp, _vp, _vp, _i64, _vp, _vp]
_lib.slse_tuning_schedule.restype = _i32
_lib.slse_tuning_schedule.argtypes = [_i64, _i32, _i32, ctypes.POINTER(CSchedule), ctypes.POINTER(ctypes.c_int64),
                                      ctypes.POINTER(ctypes.c_int32), _i32]
_lib.slse_ai_bound.restype = ctypes.c_double
_lib.slse_ai_bound.argtypes = [ctypes.c_double, _i64, _i64, _i32]
_lib.slse_status_string.restype = ctypes.c_char_p
_lib.slse_status_string.argtypes = [_i32]
_lib.slse_version.restype = _i32
_lib.slse_debug_spin_limit.restype = _i64
_lib.slse_debug_spin_limit.argtypes = [_i64]

EXPORTED = ["slse_workspace_size", "slse_fit", "slse_sketch", "slse_grad", "slse_grad_noalloc", "slse_gram", "slse_draws", "slse_qr",
            "slse_default_schedule", "slse_default_schedule_for", "slse_ai_bound", "slse_status_string",
            "slse_version", "slse_solve_normal", "slse_solve_normal_workspace", "slse_ols_vjp",
            "slse_tuning_schedule", "slse_debug_spin_limit"]


class SlseError(RuntimeError):
    def __init__(self, status: int, what: str):
        super().__init__(f"{what}: {_lib.slse_status_string(status).decode()} (status {status})")
        self.status = status


def status_string(s: int) -> str:
    return _lib.slse_status_string(s).decode()


def debug_spin_limit(polls: int) -> int:
    """slse_debug_spin_limit: fault injection for tests; sets the polls a grid-wide wait makes
    before giving up with ETIMEOUT (<= 0 restores the built-in limit); returns the previous value."""
    return int(_lib.slse_debug_spin_limit(int(polls)))


def version() -> int:
    return int(_lib.slse_version())


def ai_bound(omega: float, m_prev: int, m_i: int, d: int) -> float:
    """Theorem 4.3 lower bound on a_i (host helper of the library)."""
    return float(_lib.slse_ai_bound(omega, m_prev, m_i, d))


# ----------------------------------------------------------------------------- schedule
@dataclass
class Schedule:
    m: list
    a: list
    r: int
    mu: float
    eta: float
    T: int = 100
    tol: float = 0.0
    prec: str = "fp64"
    momentum_reset: bool = False
    kind: int = SRHT
    stage2: str = "correction"   # mixed precisions: "full" or "correction" (see slse_stage2_form)
    _keep: list = field(default_factory=list, repr=False)

    def to_c(self) -> CSchedule:
        K = len(self.m)
        m_arr = (ctypes.c_int64 * max(1, K))(*[int(v) for v in self.m])
        a_arr = (ctypes.c_int32 * max(1, K))(*[int(v) for v in self.a])
        self._keep = [m_arr, a_arr]
        return CSchedule(K, ctypes.cast(m_arr, ctypes.POINTER(ctypes.c_int64)),
                         ctypes.cast(a_arr, ctypes.POINTER(ctypes.c_int32)), int(self.r), float(self.mu),
                         float(self.eta), int(self.T), float(self.tol), int(self.kind), PREC[self.prec],
                         1 if self.momentum_reset else 0, STAGE2[self.stage2])


def default_schedule(N: int, d: int, prec: str = "fp64", T: int = 100, tol: float = 0.0,
                     kind: str = "srht", stage2: str | None = None) -> Schedule:
    """The paper's experimental schedule (Sec. 5 preamble), from the library; kind "countsketch"
    rounds m_1 = 8d up to a power of two."""
    c = CSchedule()
    mb = (ctypes.c_int64 * 64)()
    ab = (ctypes.c_int32 * 64)()
    K = _lib.slse_default_schedule_for(N, d, KIND[kind], ctypes.byref(c), mb, ab, 64)
    if K < 0 or K > 64:
        raise ValueError("invalid problem size")
    return Schedule(m=list(mb[:K]), a=list(ab[:K]), r=c.r, mu=c.mu, eta=c.eta, T=T, tol=tol, prec=prec,
                    momentum_reset=bool(c.momentum_reset), kind=c.kind,
                    stage2=stage2 or {v: n for n, v in STAGE2.items()}[c.stage2])


def tuning_schedule(N: int, d: int, prec: str = "fp64", T: int = 100, tol: float = 0.0,
                    kind: str = "srht", stage2: str | None = None) -> Schedule:
    """The SLSE-FRS-tuning schedule (Sec. 5, sketch size tuning), from the library."""
    c = CSchedule()
    mb = (ctypes.c_int64 * 64)()
    ab = (ctypes.c_int32 * 64)()
    K = _lib.slse_tuning_schedule(N, d, KIND[kind], ctypes.byref(c), mb, ab, 64)
    if K < 0 or K > 64:
        raise ValueError("invalid problem size")
    return Schedule(m=list(mb[:K]), a=list(ab[:K]), r=c.r, mu=c.mu, eta=c.eta, T=T, tol=tol, prec=prec,
                    momentum_reset=bool(c.momentum_reset), kind=c.kind,
                    stage2=stage2 or {v: n for n, v in STAGE2.items()}[c.stage2])


# ----------------------------------------------------------------------------- helpers
def _torch():
    import torch
    return torch


def _stream(stream=None) -> int:
    torch = _torch()
    s = stream if stream is not None else torch.cuda.current_stream()
    return int(s.cuda_stream)


def _dtype_code(t) -> int:
    torch = _torch()
    if t.dtype == torch.float64:
        return F64
    if t.dtype == torch.float32:
        return F32
    raise TypeError(f"unsupported dtype {t.dtype}")


def problem(X, Y) -> CProblem:
    """C problem struct for device tensors X (N x d, unit column stride) and Y (N)."""
    if X.dim() != 2 or X.stride(1) != 1:
        raise ValueError("X must be a row-major 2-D tensor")
    if Y.dim() != 1 or Y.stride(0) != 1 or Y.shape[0] != X.shape[0] or Y.dtype != X.dtype:
        raise ValueError("Y must be a contiguous vector matching X")
    return CProblem(X.shape[0], X.shape[1], _dtype_code(X), X.data_ptr(), X.stride(0), Y.data_ptr())


def workspace_size(X, Y, op: int = OP_FIT, schedule: Schedule | None = None, arg: int = 0) -> int:
    p = problem(X, Y)
    cs = schedule.to_c() if schedule is not None else None
    return int(_lib.slse_workspace_size(ctypes.byref(p), ctypes.byref(cs) if cs is not None else None, op, arg))


def alloc_workspace(nbytes: int, device=None):
    torch = _torch()
    return torch.empty(max(256, nbytes), dtype=torch.uint8, device=device or "cuda")


def _check(status: int, what: str, allow=()):
    if status != OK and status not in allow:
        raise SlseError(status, what)


@dataclass
class FitResult:
    beta: np.ndarray
    status: int
    report: dict
    beta_hist: object = None   # torch (count x d) on the device, when traced
    ms_hist: list = None
    hinv: object = None        # torch (d x d) float64 on the device: the fit's H-hat^{-1}, when asked


def fit(X, Y, schedule: Schedule | None = None, seed: int = 0, workspace=None, trace_cap: int = 0,
        stream=None, raise_on_error: bool = True, hinv: bool = False) -> FitResult:
    """slse_fit: Algorithm 2 on device tensors X, Y.  Returns beta-hat on the host."""
    torch = _torch()
    p = problem(X, Y)
    cs = schedule.to_c() if schedule is not None else None
    beta = (ctypes.c_double * p.d)()
    rep = CReport()
    tr = None
    hist = None
    ms = None
    hv = None
    dev = X.device if X.is_cuda else "cuda"
    if trace_cap > 0 or hinv:
        if hinv:
            hv = torch.empty((p.d, p.d), dtype=torch.float64, device=dev)
        if trace_cap > 0:
            hist = torch.zeros((trace_cap, p.d), dtype=torch.float64, device=dev)
            ms = (ctypes.c_float * trace_cap)()
        tr = CTrace(hist.data_ptr() if hist is not None else None,
                    ctypes.cast(ms, ctypes.POINTER(ctypes.c_float)) if ms is not None else None, trace_cap, 0,
                    hv.data_ptr() if hv is not None else None)
    ws_ptr, ws_len = (workspace.data_ptr(), workspace.numel() * workspace.element_size()) if workspace is not None \
        else (None, 0)
    st = _lib.slse_fit(ctypes.byref(p), ctypes.byref(cs) if cs is not None else None, seed, beta, ctypes.byref(rep),
                       ctypes.byref(tr) if tr is not None else None, ws_ptr, ws_len, _stream(stream))
    if raise_on_error:
        _check(st, "slse_fit", allow=(ENOTCONV,))
    report = {f: getattr(rep, f) for f, _ in CReport._fields_}
    out = FitResult(beta=np.frombuffer(beta, dtype=np.float64).copy(), status=st, report=report)
    if tr is not None and trace_cap > 0:
        out.beta_hist = hist[:tr.count]
        out.ms_hist = list(ms[:tr.count])
    out.hinv = hv
    return out


def solve_normal_workspace(X, schedule: Schedule) -> int:
    """slse_solve_normal_workspace: bytes of workspace slse_solve_normal needs for X."""
    if X.dim() != 2 or X.stride(1) != 1:
        raise ValueError("X must be a row-major 2-D tensor")
    p = CProblem(X.shape[0], X.shape[1], _dtype_code(X), X.data_ptr(), X.stride(0), X.data_ptr())
    return int(_lib.slse_solve_normal_workspace(ctypes.byref(p), PREC[schedule.prec]))


def solve_normal(X, Hinv, v, schedule: Schedule, workspace=None, stream=None, raise_on_error: bool = True):
    """slse_solve_normal: w = (X^T X)^{-1} v by preconditioned M-IHS steps (device float64).
    Returns (w, report)."""
    torch = _torch()
    p = CProblem(X.shape[0], X.shape[1], _dtype_code(X), X.data_ptr(), X.stride(0), X.data_ptr())
    if X.dim() != 2 or X.stride(1) != 1:
        raise ValueError("X must be a row-major 2-D tensor")
    v = v.to(torch.float64).contiguous()
    H = Hinv.to(torch.float64).contiguous()
    w = torch.empty(p.d, dtype=torch.float64, device=X.device)
    cs = schedule.to_c()
    rep = CReport()
    ws_ptr, ws_len = (workspace.data_ptr(), workspace.numel() * workspace.element_size()) if workspace is not None \
        else (None, 0)
    st = _lib.slse_solve_normal(ctypes.byref(p), H.data_ptr(), v.data_ptr(), w.data_ptr(), ctypes.byref(cs),
                                ctypes.byref(rep), ws_ptr, ws_len, _stream(stream))
    if raise_on_error:
        _check(st, "slse_solve_normal", allow=(ENOTCONV,))
    return w, {f: getattr(rep, f) for f, _ in CReport._fields_}


def ols_vjp(X, Y, beta, w, stream=None, out=None):
    """slse_ols_vjp: (dL/dX, dL/dY) = (r w^T - (X w) beta^T, X w), r = Y - X beta, in X's dtype.
    out: optional (dX, dY) device tensors to write into (dX row-major, X's shape and dtype)."""
    torch = _torch()
    p = problem(X, Y)
    beta = torch.as_tensor(beta, dtype=torch.float64, device=X.device).contiguous()
    w = w.to(torch.float64).contiguous()
    if out is None:
        dX = torch.empty_like(X, memory_format=torch.contiguous_format)
        dY = torch.empty_like(Y)
    else:
        dX, dY = out
        if (dX.shape != X.shape or dX.dtype != X.dtype or dX.stride(1) != 1 or dY.shape != Y.shape
                or dY.dtype != Y.dtype or not dY.is_contiguous()):
            raise ValueError("out must be (dX, dY) shaped and typed like (X, Y), dX row-major")
    st = _lib.slse_ols_vjp(ctypes.byref(p), beta.data_ptr(), w.data_ptr(), dX.data_ptr(), dX.stride(0), dY.data_ptr(),
                           _stream(stream))
    _check(st, "slse_ols_vjp")
    return dX, dY


def sketch(X, Y, m: int, seed: int = 0, prec: str = "fp64", workspace=None, stream=None, kind: str = "srht",
           want_y: bool = True):
    """slse_sketch: (S X, S Y) for one sketch of size m (kind "srht", "countsketch",
    "countsketch_hat" or "gaussian").  FP64 -> float64, mixed_bf16 -> bfloat16; mixed_fp8 ->
    (E4M3 codes (uint8, m x d), block exponents + 127 (uint8, m x ceil(d/32)), S Y in bfloat16).
    want_y=False (kind "gaussian" only) skips S Y and returns None for it."""
    torch = _torch()
    p = problem(X, Y)
    ws_ptr, ws_len = (workspace.data_ptr(), workspace.numel()) if workspace is not None else (None, 0)
    if prec == "mixed_fp8":
        # E4M3 bytes (m x ldq) followed by the block-exponent bytes (m x ceil(d/32))
        ldq = (p.d + 15) // 16 * 16
        nsb = (p.d + 31) // 32
        buf = torch.empty(m * ldq + m * nsb, dtype=torch.uint8, device=X.device)
        SY = torch.empty(m, dtype=torch.bfloat16, device=X.device)
        st = _lib.slse_sketch(ctypes.byref(p), KIND[kind], PREC[prec], seed, m, buf.data_ptr(), ldq, SY.data_ptr(),
                              ws_ptr, ws_len, _stream(stream))
        _check(st, "slse_sketch")
        return buf[:m * ldq].view(m, ldq)[:, :p.d], buf[m * ldq:].view(m, nsb), SY
    dt = torch.float64 if prec == "fp64" else torch.bfloat16
    SX = torch.empty((m, p.d), dtype=dt, device=X.device)
    SY = torch.empty(m, dtype=dt, device=X.device) if want_y else None
    st = _lib.slse_sketch(ctypes.byref(p), KIND[kind], PREC[prec], seed, m, SX.data_ptr(), p.d,
                          SY.data_ptr() if want_y else None, ws_ptr, ws_len, _stream(stream))
    _check(st, "slse_sketch")
    return SX, SY


def grad(X, Y, beta, prec: str = "fp64", workspace=None, stream=None):
    """slse_grad: g = X^T (Y - X beta) on the device (float64 vector)."""
    torch = _torch()
    p = problem(X, Y)
    b = beta if (torch.is_tensor(beta) and beta.is_cuda) else torch.as_tensor(np.asarray(beta, np.float64),
                                                                                device=X.device)
    b = b.to(torch.float64).contiguous()
    g = torch.empty(p.d, dtype=torch.float64, device=X.device)
    ws_ptr, ws_len = (workspace.data_ptr(), workspace.numel()) if workspace is not None else (None, 0)
    st = _lib.slse_grad(ctypes.byref(p), b.data_ptr(), g.data_ptr(), PREC[prec], ws_ptr, ws_len, _stream(stream))
    _check(st, "slse_grad")
    return g


def gram(X, workspace=None, stream=None):
    """slse_gram: G = Xb^T Xb (d x d float64 on the device) for the BF16 rounding Xb of X (float32),
    or G = X^T X for X in bfloat16 (row stride a multiple of 8)."""
    torch = _torch()
    if X.dim() != 2 or X.stride(1) != 1 or X.dtype not in (torch.float32, torch.bfloat16):
        raise ValueError("X must be a row-major float32 or bfloat16 matrix")
    code = F32 if X.dtype == torch.float32 else BF16
    p = CProblem(X.shape[0], X.shape[1], code, X.data_ptr(), X.stride(0), X.data_ptr())
    G = torch.empty((p.d, p.d), dtype=torch.float64, device=X.device)
    ws_ptr, ws_len = (workspace.data_ptr(), workspace.numel()) if workspace is not None else (None, 0)
    st = _lib.slse_gram(ctypes.byref(p), G.data_ptr(), ws_ptr, ws_len, _stream(stream))
    _check(st, "slse_gram")
    return G


def grad_noalloc(X, Y, beta, prec: str = "fp64", stream=None):
    """slse_grad_noalloc: the residual-gradient pass with the library's fixed scratch array,
    for callers that cannot allocate device memory (the output tensor here is the caller's)."""
    torch = _torch()
    p = problem(X, Y)
    b = beta if (torch.is_tensor(beta) and beta.is_cuda) else torch.as_tensor(np.asarray(beta, np.float64),
                                                                                device=X.device)
    b = b.to(torch.float64).contiguous()
    g = torch.empty(p.d, dtype=torch.float64, device=X.device)
    st = _lib.slse_grad_noalloc(ctypes.byref(p), b.data_ptr(), g.data_ptr(), PREC[prec], _stream(stream))
    _check(st, "slse_grad_noalloc")
    return g


def draws(N: int, seed: int, device="cuda", stream=None):
    """slse_draws: (P, sigma, D) for N' = 2^ceil(log2 N)."""
    torch = _torch()
    Np = 1 << max(0, int(N - 1).bit_length())
    P = torch.empty(Np, dtype=torch.int32, device=device)
    sigma = torch.empty(Np, dtype=torch.int32, device=device)
    D = torch.empty(Np, dtype=torch.int8, device=device)
    st = _lib.slse_draws(N, seed, P.data_ptr(), sigma.data_ptr(), D.data_ptr(), None, 0, _stream(stream))
    _check(st, "slse_draws")
    return P, sigma, D


def qr(A, want_hinv: bool = True, stream=None):
    """slse_qr: FP64 Householder R (non-negative diagonal) and optionally (R^T R)^{-1}."""
    torch = _torch()
    if A.dtype != torch.float64 or A.dim() != 2 or A.stride(1) != 1:
        raise ValueError("A must be a row-major float64 matrix")
    r, d = A.shape
    R = torch.empty((d, d), dtype=torch.float64, device=A.device)
    H = torch.empty((d, d), dtype=torch.float64, device=A.device) if want_hinv else None
    st = _lib.slse_qr(A.data_ptr(), r, d, A.stride(0), R.data_ptr(), H.data_ptr() if H is not None else None, None, 0,
                      _stream(stream))
    _check(st, "slse_qr")
    return R, H
