"""CPU checks of the C ABI: the library builds, loads, exports every function that
include/slse.h declares, and its host-only helpers agree with the oracle.  No kernel
is launched here (no GPU in this environment)."""
import ctypes
import math
import os
import re
import shutil

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    src = open(os.path.join(ROOT, "include", "slse.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(slse_[a-z_0-9]+)\s*\(", src)))


@pytest.fixture(scope="module")
def lib():
    if shutil.which("nvcc") is None and not os.path.exists("/usr/local/cuda/bin/nvcc"):
        pytest.skip("nvcc not available")
    import __graft_entry__
    path = __graft_entry__._build_module().build()
    return ctypes.CDLL(path)


def test_every_declared_symbol_is_exported(lib):
    names = _declared()
    assert "slse_fit" in names and "slse_sketch" in names and "slse_grad" in names
    for n in names:
        assert hasattr(lib, n), n


def test_binding_covers_the_header():
    import paper_2509_06856_gb300 as slse
    assert sorted(slse.EXPORTED) == _declared()


def test_host_helpers_match_oracle(lib):
    import paper_2509_06856_gb300 as slse
    from oracle import slse as osl
    for om, mp, mi, d in [(1 / 16, 1024, 2048, 64), (1.0, 4096, 8192, 64), (0.25, 200, 400, 50)]:
        assert slse.ai_bound(om, mp, mi, d) == pytest.approx(osl.ai_bound(om, mp, mi, d), rel=1e-14)
    assert math.isnan(slse.ai_bound(0.5, 10, 20, 64))
    for N, d in [(1 << 20, 64), (20000, 50), (1 << 22, 512), (100, 64)]:
        a = slse.default_schedule(N, d)
        b = osl.default_schedule(N, d)
        assert a.m == b.m and a.a == b.a and a.r == b.r and a.T == b.T
        assert a.mu == pytest.approx(b.mu, rel=1e-15) and a.eta == pytest.approx(b.eta, rel=1e-15)
    assert slse.status_string(0) == "ok" and slse.version() >= 100


def test_invalid_arguments_rejected_before_any_launch(lib):
    import paper_2509_06856_gb300 as slse
    beta = (ctypes.c_double * 4)()
    bad = [
        slse.CProblem(0, 4, slse.F64, 1, 4, 1),        # N = 0
        slse.CProblem(10, 0, slse.F64, 1, 4, 1),       # d = 0
        slse.CProblem(10, 4, slse.F64, 1, 3, 1),       # ldx < d
        slse.CProblem(3, 4, slse.F64, 1, 4, 1),        # d > N
        slse.CProblem(10, 4, 7, 1, 4, 1),              # bad dtype
        slse.CProblem(10, 4, slse.F64, None, 4, 1),    # null X
        slse.CProblem(10, 600, slse.F64, 1, 600, 1),   # d above the library's limit
        slse.CProblem((1 << 24) + 1, 4, slse.F64, 1, 4, 1),  # N' above 2^24
    ]
    for p in bad:
        assert lib.slse_fit(ctypes.byref(p), None, ctypes.c_uint64(0), beta, None, None, None,
                            ctypes.c_size_t(0), None) == slse.EINVAL
        assert slse._lib.slse_workspace_size(ctypes.byref(p), None, slse.OP_FIT, 0) == 0
    good = slse.CProblem(100, 4, slse.F64, 256, 4, 512)
    sch = slse.Schedule(m=[64, 32], a=[2, 2], r=24, mu=0.7, eta=0.1).to_c()  # not ascending
    assert slse._lib.slse_fit(ctypes.byref(good), ctypes.byref(sch), 0, beta, None, None, None, 0, None) == slse.EINVAL
    sch = slse.Schedule(m=[32], a=[2], r=2, mu=0.7, eta=0.1).to_c()          # r < d
    assert slse._lib.slse_fit(ctypes.byref(good), ctypes.byref(sch), 0, beta, None, None, None, 0, None) == slse.EINVAL
    sch = slse.Schedule(m=[32], a=[2], r=24, mu=0.7, eta=0.1, prec="mixed_bf16").to_c()  # mixed needs F32
    assert slse._lib.slse_fit(ctypes.byref(good), ctypes.byref(sch), 0, beta, None, None, None, 0, None) == slse.EINVAL
    assert slse._lib.slse_draws(0, 0, 1, 1, None, None, 0, None) == slse.EINVAL
    assert slse._lib.slse_qr(1, 3, 4, 4, 1, None, None, 0, None) == slse.EINVAL   # r < d


def test_workspace_size_is_monotone_in_problem_size(lib):
    import paper_2509_06856_gb300 as slse
    sizes = []
    for N in (1 << 12, 1 << 16, 1 << 20):
        p = slse.CProblem(N, 64, slse.F32, 256, 64, 512)
        sch = slse.default_schedule(N, 64, prec="mixed_bf16").to_c()
        sizes.append(slse._lib.slse_workspace_size(ctypes.byref(p), ctypes.byref(sch), slse.OP_FIT, 0))
    assert 0 < sizes[0] < sizes[1] < sizes[2]


def test_countsketch_host_side(lib):
    import paper_2509_06856_gb300 as slse
    from oracle import slse as osl
    for N, d in [(20000, 50), (1 << 22, 512), (1 << 16, 24)]:
        a = slse.default_schedule(N, d, kind="countsketch")
        b = osl.default_schedule(N, d, kind="countsketch")
        assert a.m == b.m and a.a == b.a and a.r == b.r and a.kind == slse.COUNTSKETCH
        assert all(m & (m - 1) == 0 for m in a.m)
    c = slse.CSchedule()
    # the Gaussian Hessian sketch keeps the SRHT subproblems: same sizes as the SRHT schedule
    g, s_ = slse.default_schedule(20000, 50, kind="gaussian"), slse.default_schedule(20000, 50)
    assert g.m == s_.m and g.a == s_.a and g.r == s_.r and g.kind == slse.GAUSSIAN
    assert slse._lib.slse_default_schedule_for(1000, 10, 7, ctypes.byref(c), None, None, 0) == -1
    beta = (ctypes.c_double * 4)()
    good = slse.CProblem(100, 4, slse.F64, 256, 4, 512)
    sch = slse.Schedule(m=[24, 48], a=[2, 2], r=24, mu=0.7, eta=0.1, kind=slse.COUNTSKETCH).to_c()  # not 2^l
    assert slse._lib.slse_fit(ctypes.byref(good), ctypes.byref(sch), 0, beta, None, None, None, 0, None) == slse.EINVAL
    assert slse._lib.slse_workspace_size(ctypes.byref(good), ctypes.byref(sch), slse.OP_FIT, 0) == 0
    ok = slse.Schedule(m=[16, 32], a=[2, 2], r=24, mu=0.7, eta=0.1, kind=slse.COUNTSKETCH).to_c()
    assert slse._lib.slse_workspace_size(ctypes.byref(good), ctypes.byref(ok), slse.OP_FIT, 0) > 0
    assert slse._lib.slse_workspace_size(ctypes.byref(good), ctypes.byref(ok), slse.OP_SKETCH, 48) == 0
    assert slse._lib.slse_workspace_size(ctypes.byref(good), ctypes.byref(ok), slse.OP_SKETCH, 64) > 0
    sch = slse.Schedule(m=[16], a=[2], r=24, mu=0.7, eta=0.1, kind=slse.GAUSSIAN, prec="mixed_fp8").to_c()
    good32 = slse.CProblem(100, 4, slse.F32, 256, 4, 512)
    assert slse._lib.slse_workspace_size(ctypes.byref(good32), ctypes.byref(sch), slse.OP_FIT, 0) == 0
    assert slse._lib.slse_fit(ctypes.byref(good32), ctypes.byref(sch), 0, beta, None, None, None, 0, None) == \
        slse.EINVAL
    gs_ = slse.Schedule(m=[16], a=[2], r=24, mu=0.7, eta=0.1, kind=slse.GAUSSIAN).to_c()
    assert slse._lib.slse_workspace_size(ctypes.byref(good), ctypes.byref(gs_), slse.OP_FIT, 0) > 0
    assert slse._lib.slse_workspace_size(ctypes.byref(good), ctypes.byref(gs_), slse.OP_SKETCH, 30) > 0
    # S Y may be omitted only for the Gaussian kind; the FP8 form is SRHT only
    assert slse._lib.slse_sketch(ctypes.byref(good), slse.SRHT, 0, 0, 16, 1024, 4, None, None, 0, None) == slse.EINVAL
    assert slse._lib.slse_sketch(ctypes.byref(good), slse.GAUSSIAN, 2, 0, 16, 1024, 4, None, None, 0, None) == \
        slse.EINVAL
    assert slse._lib.slse_sketch(ctypes.byref(good), slse.COUNTSKETCH, 0, 0, 48, 1, 4, 1, None, 0, None) == slse.EINVAL


def test_tuning_schedule_matches_oracle(lib):
    import paper_2509_06856_gb300 as slse
    from oracle import slse as osl
    # the paper's tuning sizes at d = 2^6, N = 2^22: 2^10 .. 2^16 and 2^19, a_i = 3
    a = slse.tuning_schedule(1 << 22, 64)
    assert a.m == [1 << k for k in range(10, 17)] + [1 << 19] and a.a == [3] * 8
    for N, d, kind in [(1 << 22, 64, "srht"), (1 << 22, 512, "srht"), (20000, 50, "srht"), (20000, 50, "countsketch")]:
        x = slse.tuning_schedule(N, d, kind=kind)
        y = osl.tuning_schedule(N, d, kind=kind)
        assert x.m == y.m and x.a == y.a and x.r == y.r


def test_debug_spin_limit_set_and_restore(lib):
    import paper_2509_06856_gb300 as slse
    assert slse.debug_spin_limit(0) == 0
    assert slse.debug_spin_limit(7) == 0
    assert slse.debug_spin_limit(-3) == 7      # <= 0 restores the built-in limit
    assert slse.debug_spin_limit(0) == 0


def test_solve_normal_workspace_holds_the_n_vectors(lib):
    # the backward solve keeps a zero right-hand side (N values) and, on the mixed path, the
    # FP32 base residual (N values) besides O(d) state: the size grows by those per row
    import paper_2509_06856_gb300 as slse
    torch = pytest.importorskip("torch")
    d = 32
    s64 = slse.default_schedule(1 << 14, d, prec="fp64")
    smx = slse.default_schedule(1 << 14, d, prec="mixed_bf16")
    X64 = torch.empty((1 << 14, d), dtype=torch.float64)
    X32a = torch.empty((1 << 14, d), dtype=torch.float32)
    X32b = torch.empty((1 << 15, d), dtype=torch.float32)
    a64 = slse.solve_normal_workspace(X64, s64)
    a, b = slse.solve_normal_workspace(X32a, smx), slse.solve_normal_workspace(X32b, smx)
    assert a64 >= 8 * (1 << 14)
    assert b - a == (4 + 4) * (1 << 14)   # r0 (FP32) + the zero right-hand side (FP32)


def test_stage2_form_field(lib):
    """The 2nd-stage form is part of the schedule: the library's default is the correction form,
    and a value outside slse_stage2_form is an argument error."""
    import paper_2509_06856_gb300 as slse
    assert slse.default_schedule(1 << 16, 64, prec="mixed_bf16").stage2 == "correction"
    assert slse.default_schedule(1 << 16, 64, prec="mixed_bf16", stage2="full").stage2 == "full"
    good = slse.CProblem(1 << 12, 16, slse.F32, 256, 16, 512)
    sch = slse.default_schedule(1 << 12, 16, prec="mixed_bf16").to_c()
    assert slse._lib.slse_workspace_size(ctypes.byref(good), ctypes.byref(sch), slse.OP_FIT, 0) > 0
    sch.stage2 = 2
    assert slse._lib.slse_workspace_size(ctypes.byref(good), ctypes.byref(sch), slse.OP_FIT, 0) == 0
    beta = (ctypes.c_double * 16)()
    assert slse._lib.slse_fit(ctypes.byref(good), ctypes.byref(sch), 0, beta, None, None, None, 0, None) == slse.EINVAL


def test_gram_rejects_bad_inputs(lib):
    import paper_2509_06856_gb300 as slse
    p64 = slse.CProblem(1000, 8, slse.F64, 256, 8, 512)
    assert slse._lib.slse_gram(ctypes.byref(p64), 1024, None, 0, None) == slse.EINVAL
    p32 = slse.CProblem(1000, 8, slse.F32, 256, 8, 512)
    assert slse._lib.slse_gram(ctypes.byref(p32), None, None, 0, None) == slse.EINVAL
    assert slse._lib.slse_workspace_size(ctypes.byref(p32), None, slse.OP_GRAM, 0) > 0
    # BF16 X needs a row stride that is a multiple of 8 elements
    pb = slse.CProblem(1000, 12, slse.BF16, 256, 12, 512)
    assert slse._lib.slse_gram(ctypes.byref(pb), 1024, None, 0, None) == slse.EINVAL
    assert slse._lib.slse_workspace_size(ctypes.byref(pb), None, slse.OP_GRAM, 0) == 0
    pb = slse.CProblem(1000, 12, slse.BF16, 256, 16, 512)
    assert slse._lib.slse_workspace_size(ctypes.byref(pb), None, slse.OP_GRAM, 0) > 0
