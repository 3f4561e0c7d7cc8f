"""Pins of the FP8 (E4M3, 32-element power-of-two block scales) oracle against the OCP
bit-field definition's known values, PyTorch's float8_e4m3fn conversion (a library routine
written independently), round-to-nearest-even ties, and the error bound of the scaled form."""
import math

import numpy as np
import pytest

from oracle import fp8


def test_value_set_from_the_definition():
    v = fp8.e4m3_values()
    assert len(v) == 253
    assert v.max() == 448.0 and v.min() == -448.0
    pos = v[v > 0]
    assert pos.min() == 2.0 ** -9                    # smallest subnormal
    assert 2.0 ** -6 in pos and 1.0 in pos and 0.875 in pos and 240.0 in pos
    assert 464.0 not in pos                          # 1.8125 * 2^8 is the NaN code


def test_rounding_matches_torch_float8():
    torch = pytest.importorskip("torch")
    if not hasattr(torch, "float8_e4m3fn"):
        pytest.skip("no float8_e4m3fn in this torch")
    rng = np.random.default_rng(0)
    x = np.concatenate([rng.standard_normal(20000) * s for s in (1e-3, 0.1, 1.0, 30.0, 200.0)])
    x = x[np.abs(x) <= 448.0]
    ours = fp8.round_e4m3(x)
    ref = torch.from_numpy(x).to(torch.float32).to(torch.float8_e4m3fn).to(torch.float64).numpy()
    # float32 first: x -> float32 rounding can move an exact tie, so compare on float32 inputs
    ours32 = fp8.round_e4m3(x.astype(np.float32).astype(np.float64))
    assert np.array_equal(ours32, ref)
    assert np.all(np.abs(ours - x) <= np.maximum(2.0 ** -4 * np.abs(x), 2.0 ** -10))


@pytest.mark.parametrize("x,want", [(1.0625, 1.0), (1.1875, 1.25), (-1.0625, -1.0), (1.5 * 2.0 ** -9, 2.0 * 2.0 ** -9),
                                    (0.5 * 2.0 ** -9, 0.0), (460.0, 448.0), (1e6, 448.0), (0.0, 0.0)])
def test_ties_to_even_and_saturation(x, want):
    assert fp8.round_e4m3(x) == want


@pytest.mark.parametrize("amax,k", [(448.0, 0), (449.0, 1), (224.0, -1), (224.5, 0), (1.0, -8), (0.0, -127)])
def test_block_exponent_rule(amax, k):
    assert fp8.block_exponent(amax) == k
    if amax > 0:
        assert amax <= 448.0 * 2.0 ** k and amax > 448.0 * 2.0 ** (k - 1)


def test_scaled_rows_error_bound_and_exact_values():
    rng = np.random.default_rng(1)
    A = rng.standard_normal((64, 100)) * np.logspace(-3, 3, 100)
    Q, K = fp8.quantize_rows(A)
    assert K.shape == (64, 4)
    D = fp8.dequantize_rows(Q, K)
    S = np.repeat(np.ldexp(1.0, K), 32, axis=1)[:, :100]
    assert np.all(np.abs(D - A) <= 2.0 ** -4 * np.abs(A) + 2.0 ** -10 * S)
    # every block's largest element lands in (224, 448] before rounding: no saturation
    for b in range(4):
        blk = np.abs(A[:, 32 * b:32 * (b + 1)]).max(axis=1)
        r = blk / np.ldexp(1.0, K[:, b])
        assert np.all((r > 224.0) & (r <= 448.0))
    # values already on the grid times a power of two come back exactly
    E = np.ldexp(fp8.round_e4m3(rng.standard_normal((8, 32)) * 100), 5)
    assert np.array_equal(fp8.dequantize_rows(*fp8.quantize_rows(E)), E)


def test_planted_mistakes_are_caught(monkeypatch):
    good = fp8.round_e4m3

    def truncating(x):  # round toward zero instead of to nearest
        x = np.asarray(x, np.float64)
        r = good(x)
        return np.where(np.abs(r) > np.abs(x), np.copysign(fp8._POS[np.maximum(np.searchsorted(fp8._POS, np.abs(r)) - 1, 0)], x), r)
    monkeypatch.setattr(fp8, "round_e4m3", truncating)
    with pytest.raises(AssertionError):
        test_ties_to_even_and_saturation(1.1875, 1.25)
    monkeypatch.setattr(fp8, "round_e4m3", good)
    monkeypatch.setattr(fp8, "block_exponent", lambda amax: math.frexp(amax / 448.0)[1] - 1 if amax else -127)
    with pytest.raises(AssertionError):
        test_scaled_rows_error_bound_and_exact_values()
