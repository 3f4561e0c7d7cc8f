"""Pins for the oracle's random draws (Philox4x32-10 and the SRHT draws D, P, sigma)."""
import os

import numpy as np
import pytest

from oracle import philox, sketch as sk

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _kat():
    rows = []
    for line in open(os.path.join(GOLDEN, "philox4x32_10_kat.txt")):
        line = line.split("#")[0].strip()
        if not line:
            continue
        lhs, rhs = line.split("->")
        rows.append(([int(v, 16) for v in lhs.split()], [int(v, 16) for v in rhs.split()]))
    return rows


@pytest.mark.parametrize("case", range(3))
def test_philox_known_answers(case):
    (c0, c1, c2, c3, k0, k1), want = _kat()[case]
    got = philox.philox4x32_10([c0], [c1], [c2], [c3], k0, k1)
    assert [int(w[0]) for w in got] == want


def test_stream_words_counter_layout():
    # counter i -> (i mod 2^32, i div 2^32, stream, 0); key -> (seed lo, seed hi)
    seed = (7 << 32) | 11
    w = philox.stream_words(seed, 2, 5)
    for i in range(5):
        ref = philox.philox4x32_10([i], [0], [2], [0], 11, 7)
        assert all(int(a[i]) == int(b[0]) for a, b in zip(w, ref))


def test_padded_size():
    assert [sk.padded_size(n) for n in (1, 2, 3, 4, 5, 20000, 1 << 20, (1 << 20) + 1)] == \
        [1, 2, 4, 4, 8, 32768, 1 << 20, 1 << 21]


@pytest.mark.parametrize("Np", [1, 2, 64, 4096])
def test_draws_are_permutations(Np):
    D, P, sigma = sk.draws(Np, seed=5)
    assert set(np.unique(D)) <= {-1.0, 1.0}
    assert np.array_equal(np.sort(P), np.arange(Np))
    assert np.array_equal(np.sort(sigma), np.arange(Np))


def test_draws_deterministic_and_seed_dependent():
    a = sk.draws(1024, 3)
    b = sk.draws(1024, 3)
    c = sk.draws(1024, 4)
    assert all(np.array_equal(x, y) for x, y in zip(a, b))
    assert not np.array_equal(a[1], c[1]) and not np.array_equal(a[2], c[2])
    assert not np.array_equal(a[1], a[2])  # P and sigma come from different streams


def test_rademacher_balance_and_permutation_uniformity():
    # Rademacher: mean ~ 0.  Permutation: the position of element 0 is uniform
    # over [0, n) (chi-square over many seeds), and P is not the identity.
    D = sk.rademacher(1 << 16, 9)
    assert abs(D.mean()) < 4.0 / np.sqrt(1 << 16)
    n, seeds = 8, 4000
    counts = np.zeros(n)
    for s in range(seeds):
        P = sk.uniform_permutation(n, s, sk.STREAM_P)
        counts[int(np.where(P == 0)[0][0])] += 1
    chi2 = ((counts - seeds / n) ** 2 / (seeds / n)).sum()
    assert chi2 < 30.0  # 7 dof: P(chi2 > 30) ~ 1e-4


def test_argsort_tie_rule():
    # ties between equal keys go to the smaller index (stable sort)
    keys = np.array([5, 3, 5, 3, 1], dtype=np.uint64)
    assert list(np.argsort(keys, kind="stable")) == [4, 1, 3, 0, 2]
