"""Planted mistakes: each test breaks one step of the oracle (on the CPU, through
monkeypatch) and checks that a pin in tests/test_oracle_*.py then fails.  This shows
the pins would catch a dropped term, a wrong sign or index, or a wrong scale."""
import math

import numpy as np
import pytest

from oracle import gaussian as gs
from oracle import linalg, sketch as sk, slse
import tests.test_oracle_gaussian as tg
import tests.test_oracle_random as tr
import tests.test_oracle_sketch as ts
import tests.test_oracle_solve as tv


def _fails(fn, *args):
    with pytest.raises(AssertionError):
        fn(*args)


def test_fwht_wrong_sign_is_caught(monkeypatch):
    good = sk.fwht

    def bad(A):
        out = good(A)
        out[1] = -out[1]          # one wrong sign in one output row
        return out
    monkeypatch.setattr(sk, "fwht", bad)
    _fails(ts.test_fwht_matches_dense, 16)
    _fails(ts.test_fast_sketch_equals_dense_definition, 16, 5, 0)


def test_missing_normalisation_is_caught(monkeypatch):
    good = sk.hdp
    monkeypatch.setattr(sk, "hdp", lambda X, D, P: good(X, D, P) * math.sqrt(D.shape[0]))
    _fails(ts.test_fast_sketch_equals_dense_definition, 37, 11, 3)
    _fails(tv.test_stage2_limit_is_ols_and_rate_near_sqrt_d_over_r)


def test_signs_not_applied_is_caught(monkeypatch):
    monkeypatch.setattr(sk, "rademacher", lambda Np, seed: np.ones(Np))
    _fails(tr.test_rademacher_balance_and_permutation_uniformity)


def test_identity_permutation_is_caught(monkeypatch):
    monkeypatch.setattr(sk, "uniform_permutation", lambda Np, seed, stream: np.arange(Np))
    _fails(tr.test_draws_deterministic_and_seed_dependent)


def test_transposed_sampling_index_is_caught(monkeypatch):
    # sampling by position instead of by sigma (rows 0..m-1 of the transform)
    good = sk.draws
    monkeypatch.setattr(sk, "draws", lambda Np, seed: (lambda D, P, s: (D, P, np.arange(Np)))(*good(Np, seed)))
    _fails(tr.test_draws_deterministic_and_seed_dependent)


def test_householder_dropped_factor_is_caught(monkeypatch):
    def bad(A):
        A = np.array(A, dtype=np.float64, copy=True)
        r, d = A.shape
        for j in range(min(r, d)):
            x = A[j:, j]
            nrm = np.sqrt(x @ x)
            alpha = -nrm if x[0] >= 0 else nrm
            v = x.copy()
            v[0] -= alpha
            A[j:, j:] -= np.outer(v, (1.0 / (v @ v)) * (v @ A[j:, j:]))   # factor 2 dropped
        R = np.triu(A[:min(r, d)])
        return R * np.where(np.diag(R) < 0, -1.0, 1.0)[:, None]
    monkeypatch.setattr(linalg, "householder_r", bad)
    _fails(tv.test_householder_r_properties, 30, 5)


def test_gradient_sign_flip_is_caught(monkeypatch):
    good = slse.grad
    monkeypatch.setattr(slse, "grad", lambda X, Y, b, block_rows=1 << 16: -good(X, Y, b, block_rows))
    _fails(tv.test_gradient_sign_and_value)
    _fails(tv.test_noiseless_fit_recovers_beta)


def test_momentum_sign_flip_is_caught(monkeypatch):
    def bad(beta, beta_prev, g, R, mu, eta):
        return beta + mu * slse.hinv_apply(R, g) - eta * (beta - beta_prev), beta
    monkeypatch.setattr(slse, "mihs_step", bad)
    _fails(tv.test_theory_parameters_contract_by_one_third)


def test_transposed_preconditioner_is_caught(monkeypatch):
    # H^{-1} applied as R^{-T} R^{-1} (operands transposed) instead of R^{-1} R^{-T}
    monkeypatch.setattr(slse, "hinv_apply",
                        lambda R, v: linalg.solve_lower(R.T, linalg.solve_upper(R, v)))
    _fails(tv.test_hinv_apply_inverts_sketched_hessian)


# ---- CountSketch oracle (tests/test_oracle_countsketch.py)
import tests.test_oracle_countsketch as tc  # noqa: E402
from oracle import countsketch as cs  # noqa: E402


def test_countsketch_signs_dropped_is_caught(monkeypatch):
    good = cs.cs_hash
    monkeypatch.setattr(cs, "cs_hash", lambda N, seed: (good(N, seed)[0], np.ones(N)))
    _fails(tc.test_expectation_of_sts_is_identity)
    _fails(tc.test_bucket_and_sign_uniformity)


def test_countsketch_srht_style_scale_is_caught(monkeypatch):
    good = cs.countsketch
    monkeypatch.setattr(cs, "countsketch",
                        lambda X, Y, m, seed: tuple(math.sqrt(np.asarray(X).shape[0] / m) * a for a in good(X, Y, m, seed)))
    _fails(tc.test_dense_matrix_structure_and_product, 64, 16, 2)


def test_countsketch_high_bits_bucket_is_caught(monkeypatch):
    def bad(h, m):
        l = m.bit_length() - 1
        return (h >> np.uint64(32 - l)).astype(np.int64) if l else np.zeros(h.shape, np.int64)
    monkeypatch.setattr(cs, "cs_buckets", bad)
    _fails(tc.test_folding_identity, 8)


def test_countsketch_hessian_sketch_not_independent_is_caught(monkeypatch):
    def bad(N, seed, r):
        h, s = cs.cs_hash(N, seed)
        return ((h * np.uint64(r)) >> np.uint64(32)).astype(np.int64), s
    monkeypatch.setattr(cs, "hat_hash", bad)
    _fails(tc.test_bucket_and_sign_uniformity)


def test_countsketch_fold_wrong_offset_is_caught(monkeypatch):
    def bad(SX, m):
        M = SX.shape[0]
        return SX.reshape((m, M // m) + SX.shape[1:]).sum(axis=1)   # adds neighbours, not b + q m
    monkeypatch.setattr(cs, "fold", bad)
    _fails(tc.test_folding_identity, 8)


def test_gaussian_log_base_is_caught(monkeypatch):
    def bad(w):
        w = np.asarray(w, np.uint64)
        u1 = ((w & np.uint64(0xFFFF)).astype(np.float64) + 0.5) / 65536.0
        u2 = ((w >> np.uint64(16)).astype(np.float64) + 0.5) / 65536.0
        rad = np.sqrt(-2.0 * np.log10(u1))          # log10 in place of ln
        return rad * np.cos(2 * math.pi * u2), rad * np.sin(2 * math.pi * u2)
    monkeypatch.setattr(gs, "normals_from_words", bad)
    _fails(tg.test_box_muller_closed_form_values)
    _fails(tg.test_normal_law_moments_and_ks)


def test_gaussian_swapped_cosine_and_sine_is_caught(monkeypatch):
    good = gs.normals_from_words
    monkeypatch.setattr(gs, "normals_from_words", lambda w: good(w)[::-1])
    _fails(tg.test_box_muller_closed_form_values)


def test_gaussian_row_counter_ignored_is_caught(monkeypatch):
    good = gs.gaussian_rows
    monkeypatch.setattr(gs, "gaussian_rows", lambda seed, i0, i1, N: np.repeat(good(seed, 0, 1, N), i1 - i0, 0))
    _fails(tg.test_rows_and_columns_are_independent)
    _fails(tg.test_prediction_efficiency_exact_gaussian_value)


def test_gaussian_missing_scale_is_caught(monkeypatch):
    monkeypatch.setattr(gs, "gaussian_matrix_dense", lambda N, m, seed: gs.gaussian_rows(seed, 0, m, N))
    _fails(tg.test_expectation_of_sts_is_identity)
