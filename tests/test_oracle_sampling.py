"""Pins for the sampling policies "dec, swr" and "dec, swor" (Sec. 5.2; Algorithm 4 steps 3-4).

Checked against closed forms and brute force, not against the oracle's own formulas:
* swor on two points: P(i before j) = P_i / (P_i + P_j) (one draw between two points);
* swor on three points: each of the 6 orders has the successive-draw (Plackett-Luce)
  probability, enumerated by hand; frequencies over many seeds agree (chi-square);
* swor with equal scores is a uniform random permutation; weight-0 points never precede others;
* swr: draw frequencies follow n P (chi-square), weight-0 points never drawn, and the inverse CDF
  on hand-computed cumulative sums;
* the uniforms: exact construction from the Philox words, inside (0, 1).
"""
import itertools
import math

import numpy as np
import pytest
from scipy import stats

from oracle import slso_oracle as O


def test_uniforms_from_philox_words():
    u = O.sample_uniforms(1000, 17)
    assert np.all((u > 0.0) & (u < 1.0))
    lo = np.arange(1000, dtype=np.uint64) & np.uint64(0xFFFFFFFF)
    w = O.philox4x32_10(lo, 0, 0, O.TAG_SAMPLE, 17)
    for t in (0, 1, 999):
        m = (int(w[0][t]) << 20) + (int(w[1][t]) >> 12)
        assert u[t] == (m + 0.5) / 2**52
    assert abs(u.mean() - 0.5) < 4 / math.sqrt(12 * 1000)


def test_swr_inverse_cdf_by_hand():
    sc = np.array([1.0, 0.0, 3.0, 2.0])  # cumulative 1, 1, 4, 6
    u = np.array([0.1, 1 / 6 - 1e-12, 1 / 6 + 1e-12, 0.5, 0.999])  # targets 0.6, ~1-, ~1+, 3, 5.994
    np.testing.assert_array_equal(O.order_swr_from_uniforms(sc, u), [0, 0, 2, 2, 3])


def test_swr_frequencies_follow_p_and_skip_zero_weights():
    sc = np.array([5.0, 0.0, 1.0, 3.0, 1.0, float("nan")])
    draws = np.concatenate([O.order_swr(sc, seed) for seed in range(2000)])  # 12000 draws
    counts = np.bincount(draws, minlength=sc.size)
    assert counts[1] == 0 and counts[5] == 0
    p = np.array([5.0, 1.0, 3.0, 1.0]) / 10.0
    assert stats.chisquare(counts[[0, 2, 3, 4]], p * draws.size).pvalue > 1e-4


def test_swr_needs_positive_total():
    with pytest.raises(ValueError):
        O.order_swr(np.zeros(5), 1)


def test_swor_two_points_pairwise_probability():
    sc = np.array([1.0, 3.0])
    first = np.array([O.order_swor(sc, seed)[0] for seed in range(4000)])
    k = int(np.sum(first == 1))  # P(point 1 first) = 3 / 4
    assert stats.binomtest(k, first.size, 0.75).pvalue > 1e-4


def test_swor_three_points_plackett_luce_brute_force():
    w = np.array([1.0, 2.0, 5.0])
    P = w / w.sum()
    perms = list(itertools.permutations(range(3)))
    exact = []
    for a, b, c in perms:  # successive draws without replacement
        exact.append(P[a] * P[b] / (1 - P[a]))
    counts = {p: 0 for p in perms}
    n = 6000
    for seed in range(n):
        counts[tuple(O.order_swor(w, seed))] += 1
    assert stats.chisquare([counts[p] for p in perms], np.array(exact) * n).pvalue > 1e-4


def test_swor_equal_scores_is_uniform_permutation_and_zero_weights_last():
    n, reps = 6, 3000
    pos = np.zeros((n, n))
    for seed in range(reps):
        o = O.order_swor(np.ones(n), seed)
        pos[o, np.arange(n)] += 1
    assert stats.chisquare(pos.ravel(), np.full(n * n, reps / n)).pvalue > 1e-4
    sc = np.array([0.0, 2.0, 0.0, 1.0, float("nan")])
    for seed in range(50):
        o = O.order_swor(sc, seed)
        assert sorted(o[:2].tolist()) == [1, 3]
        assert o[2:].tolist() == [0, 2, 4]  # weight 0 in increasing index, NaN last
