"""Pins for the oracle's randomness: Philox4x32-10, bf16 rounding, Box-Muller, hashes.

Each check compares against something other than the oracle itself: published
known-answer vectors, torch's float32->bfloat16 conversion, scipy's Hadamard matrix,
closed-form moments of the distributions.
"""
import math
import os

import numpy as np
import pytest
import torch
from scipy import stats
from scipy.linalg import hadamard

from oracle import slso_oracle as O


def _kat_rows(golden_dir):
    rows = []
    with open(os.path.join(golden_dir, "philox4x32_10_kat.txt")) as f:
        for line in f:
            if line.startswith("#") or not line.strip():
                continue
            rows.append([int(x, 16) for x in line.split()])
    return rows


def test_philox_known_answers(golden_dir):
    rows = _kat_rows(golden_dir)
    assert len(rows) == 3
    for r in rows:
        c, k, want = r[0:4], r[4] | (r[5] << 32), r[6:10]
        got = O.philox4x32_10(*c, k)
        assert [int(x) for x in got] == want


def test_philox_vectorised_matches_scalar():
    i = np.arange(1000, dtype=np.uint64) * np.uint64(2654435761)
    w = O.philox4x32_10(i & O._MASK32, i >> O._SH32, 7, 3, 0x1234567890ABCDEF)
    for t in (0, 17, 999):
        ii = int(i[t])
        ws = O.philox4x32_10(ii & 0xFFFFFFFF, ii >> 32, 7, 3, 0x1234567890ABCDEF)
        assert [int(x[t]) for x in w] == [int(x) for x in ws]


def test_bf16_round_matches_torch_on_float32_values():
    rng = np.random.default_rng(0)
    x32 = (rng.standard_normal(200000) * np.exp(rng.uniform(-20, 20, 200000))).astype(np.float32)
    want = torch.from_numpy(x32).to(torch.bfloat16).to(torch.float64).numpy()
    got = O.bf16_round(x32.astype(np.float64))
    np.testing.assert_array_equal(got, want)


def test_bf16_round_ties_to_even_and_no_double_rounding():
    one = 1.0
    ulp = 2.0**-7
    # exact midpoints go to the even neighbour
    assert O.bf16_round(np.array([one + ulp / 2]))[0] == one
    assert O.bf16_round(np.array([one + 3 * ulp / 2]))[0] == one + 2 * ulp
    # just above a midpoint rounds up even though float32 would first round it to the midpoint
    x = one + ulp / 2 + 2.0**-40
    assert np.float32(x) == np.float32(one + ulp / 2)
    assert O.bf16_round(np.array([x]))[0] == one + ulp
    assert O.bf16_round(np.array([-x]))[0] == -(one + ulp)
    assert O.bf16_round(np.array([0.0]))[0] == 0.0


def test_box_muller_is_standard_normal():
    i = np.arange(400000, dtype=np.uint64)
    w = O.philox4x32_10(i, 0, 0, 99, 42)
    z = O.box_muller(w[0], w[1])
    assert abs(z.mean()) < 5 / math.sqrt(z.size)
    assert abs(z.var() - 1.0) < 5 * math.sqrt(2.0 / z.size)
    assert stats.kstest(z, "norm").pvalue > 1e-3


def test_countsketch_hash_uniform_buckets_and_balanced_signs():
    n, s = 200000, 64
    b, sg = O.countsketch_hash(n, s, 7)
    assert b.min() >= 0 and b.max() < s
    counts = np.bincount(b, minlength=s)
    assert stats.chisquare(counts).pvalue > 1e-4
    assert set(np.unique(sg)) == {-1.0, 1.0}
    assert abs(sg.mean()) < 5 / math.sqrt(n)


def test_hadamard_entries_match_scipy_sylvester():
    n = 64
    H = O.hadamard_entries(np.arange(n), np.arange(n))
    np.testing.assert_array_equal(H, hadamard(n).astype(np.float64))


def test_srht_sample_is_distinct_sorted_and_uniform():
    n_pad, s = 1024, 100
    hits = np.zeros(n_pad)
    for seed in range(200):
        smp = O.srht_sample(n_pad, s, seed)
        assert smp.size == s and np.all(np.diff(smp) > 0) and smp[0] >= 0 and smp[-1] < n_pad
        hits[smp] += 1
    # each index kept with probability s / n_pad
    expect = 200 * s / n_pad
    assert stats.chisquare(hits, np.full(n_pad, expect)).pvalue > 1e-4


def test_gaussian_entries_are_bf16_normal():
    G = O.gaussian_block(np.arange(64), np.arange(5000), 11)
    np.testing.assert_array_equal(G, O.bf16_round(G))
    assert abs(G.mean()) < 5 / math.sqrt(G.size)
    assert abs(G.var() - 1.0) < 0.02
    # distinct (row, column) counters give independent-looking entries
    assert abs(np.corrcoef(G[0], G[1])[0, 1]) < 0.05


def test_gaussian_four_entries_per_philox_block():
    """Columns 4b..4b+3 of row j come from one Philox block (lo b, hi b, j, 4): entries 4b, 4b+1
    are rho(w0) cos, rho(w0) sin of the angle 2 pi w1 2^-32 (so their squares sum to
    -2 ln((w0+1) 2^-32)), entries 4b+2, 4b+3 likewise from (w2, w3).  Checked against
    high-precision values computed from the Philox words alone."""
    mpmath = pytest.importorskip("mpmath")
    mpmath.mp.dps = 30
    rows = np.array([0, 5, 77])
    cols = np.arange(4 * 6) + 4 * (2**32 + 3)  # blocks whose index has a nonzero high word
    G = O.gaussian_block(rows, cols, 1234)
    for a, j in enumerate(rows):
        for b in range(6):
            blk = int(cols[4 * b]) // 4
            w = O.philox4x32_10(np.uint64(blk & 0xFFFFFFFF), np.uint64(blk >> 32), np.uint64(j),
                                O.TAG_GAUSSIAN, 1234)
            w = [int(x) for x in w]
            for pair in range(2):
                wr, wt = w[2 * pair], w[2 * pair + 1]
                rho = mpmath.sqrt(-2 * mpmath.log(mpmath.mpf(wr + 1) / 2**32))
                th = 2 * mpmath.pi * mpmath.mpf(wt) / 2**32
                for k, exact in enumerate((rho * mpmath.cos(th), rho * mpmath.sin(th))):
                    got = G[a, 4 * b + 2 * pair + k]
                    # bf16 keeps 8 significant bits: within half a bf16 ulp of the exact value
                    assert abs(got - float(exact)) <= 2.0**-8 * abs(float(exact)) + 1e-30


def test_gaussian_cos_sin_entries_uncorrelated():
    G = O.gaussian_block(np.arange(4000), np.arange(8), 99)
    for k in range(0, 8, 2):
        assert abs(np.corrcoef(G[:, k], G[:, k + 1])[0, 1]) < 0.05
    assert abs(np.corrcoef(G[:, 0], G[:, 2])[0, 1]) < 0.05


def test_box_muller_sine_by_shifted_word():
    """sin(2 pi w 2^-32) is evaluated as the cosine of the word shifted by 2^30 (mod 2^32)."""
    mpmath = pytest.importorskip("mpmath")
    mpmath.mp.dps = 40
    rng = np.random.default_rng(4)
    w0 = np.array(list(rng.integers(0, 2**32, 200)) + [2**31, 7], dtype=np.uint64)
    w1 = np.array(list(rng.integers(0, 2**32, 200)) + [0, 2**30], dtype=np.uint64)
    got = O.box_muller(w0, (w1 - np.uint64(2**30)) & np.uint64(0xFFFFFFFF))
    for a, b, g in zip(w0, w1, got):
        rho = mpmath.sqrt(-2 * mpmath.log(mpmath.mpf(int(a) + 1) / 2**32))
        exact = rho * mpmath.sin(2 * mpmath.pi * mpmath.mpf(int(b)) / 2**32)
        if abs(exact) < 1e-30:
            assert g == 0.0
        else:
            assert abs(g - float(exact)) <= 8 * np.spacing(abs(float(exact)))


def test_jl_matrix_moments():
    d, k = 300, 200
    P = O.jl_matrix(d, k, 5)
    assert P.shape == (d, k)
    assert abs((P * P).sum() / d - 1.0) < 0.03  # E ||row||^2 = 1
    P2 = O.jl_matrix(d, k, 6)
    assert not np.allclose(P, P2)


def test_box_muller_accurate_to_few_ulp_against_high_precision():
    """The float64 normal is within a few ulp (relative) of the exact value everywhere,
    including u1 near 1 (tiny radius) and angles near the zeros of the cosine."""
    mpmath = pytest.importorskip("mpmath")
    mpmath.mp.dps = 40
    rng = np.random.default_rng(3)
    w0 = list(rng.integers(0, 2**32, 300)) + [0, 1, 2**31 - 1, 2**31, 2**32 - 2, 2**32 - 1]
    w1 = list(rng.integers(0, 2**32, 300)) + [0, 2**30, 2**30 - 1, 2**30 + 1, 3 * 2**30 + 7, 2**29]
    w0 = np.array(w0, dtype=np.uint64)
    w1 = np.array(w1[: len(w0)], dtype=np.uint64)
    got = O.box_muller(w0, w1)
    for a, b, g in zip(w0, w1, got):
        u1 = mpmath.mpf(int(a) + 1) / 2**32
        u2 = mpmath.mpf(int(b)) / 2**32
        exact = mpmath.sqrt(-2 * mpmath.log(u1)) * mpmath.cos(2 * mpmath.pi * u2)
        if abs(exact) < 1e-30:  # an exact zero of the cosine, left at 1e-40 by mpmath
            assert g == 0.0
        else:
            assert abs((g - exact) / exact) < 8 * 2.0**-53
