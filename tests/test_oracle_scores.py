"""Pins for the oracle's leverage scores, QR, rank and ordering.

Anchors: exact rational hat matrices (brute force), LAPACK QR as an independent
routine, closed forms (orthonormal columns, d = 1), the projection invariants of the
leverage score definition (Sec. 2.2), and the subspace-embedding band (Sec. 2.1).
"""
import math
from fractions import Fraction

import numpy as np
import pytest
import scipy.linalg as sla
from scipy.linalg import hadamard

from oracle import slso_oracle as O


# ---------------------------------------------------------------- brute force
def _frac_inverse(M):
    n = len(M)
    A = [row[:] + [Fraction(int(i == j)) for j in range(n)] for i, row in enumerate(M)]
    for c in range(n):
        p = next(r for r in range(c, n) if A[r][c] != 0)
        A[c], A[p] = A[p], A[c]
        piv = A[c][c]
        A[c] = [x / piv for x in A[c]]
        for r in range(n):
            if r != c and A[r][c] != 0:
                f = A[r][c]
                A[r] = [x - f * y for x, y in zip(A[r], A[c])]
    return [row[n:] for row in A]


def _hat_diag_exact(X, cols):
    """diag of X_c (X_c^T X_c)^-1 X_c^T in exact rationals, X_c = the columns ``cols``."""
    Xc = [[Fraction(int(X[i][j])) for j in cols] for i in range(len(X))]
    d = len(cols)
    G = [[sum(Xc[i][a] * Xc[i][b] for i in range(len(X))) for b in range(d)] for a in range(d)]
    Gi = _frac_inverse(G)
    return [sum(Xc[i][a] * Gi[a][b] * Xc[i][b] for a in range(d) for b in range(d)) for i in range(len(X))]


@pytest.mark.parametrize("seed", range(6))
def test_exact_scores_match_rational_hat_matrix(seed):
    rng = np.random.default_rng(seed)
    n, d = int(rng.integers(4, 9)), int(rng.integers(1, 4))
    X = rng.integers(-5, 6, size=(n, d))
    while np.linalg.matrix_rank(X) < d:
        X = rng.integers(-5, 6, size=(n, d))
    want = [float(v) for v in _hat_diag_exact(X.tolist(), list(range(d)))]
    np.testing.assert_allclose(O.exact_leverage(X.astype(float)), want, rtol=0, atol=1e-13)


def test_exact_scores_rank_deficient_match_rational_projection():
    # third column = first + second: rank 2; the hat matrix is that of the first two columns
    X = np.array([[1, 2, 3], [0, 1, 1], [2, -1, 1], [1, 1, 2], [3, 0, 3], [-1, 2, 1]])
    want = [float(v) for v in _hat_diag_exact(X.tolist(), [0, 1])]
    np.testing.assert_allclose(O.exact_leverage(X.astype(float)), want, atol=1e-13)


def test_exact_scores_rows_variant_agrees():
    rng = np.random.default_rng(3)
    X = rng.standard_normal((3000, 20)) * np.exp(rng.standard_normal((3000, 1)))
    rows = np.arange(0, 3000, 7)
    np.testing.assert_allclose(O.exact_leverage_rows(X, rows, block=512), O.exact_leverage(X)[rows],
                               rtol=1e-10)


# ---------------------------------------------------------------- closed forms
def test_orthonormal_hadamard_columns_give_uniform_scores():
    n, d = 256, 12
    X = hadamard(n)[:, :d] / math.sqrt(n)
    np.testing.assert_allclose(O.exact_leverage(X), d / n, rtol=1e-12)


def test_single_column_closed_form():
    x = np.random.default_rng(1).standard_normal((500, 1))
    np.testing.assert_allclose(O.exact_leverage(x), (x[:, 0] ** 2) / np.sum(x**2), rtol=1e-12)


def test_projection_invariants():
    rng = np.random.default_rng(2)
    n, d = 400, 17
    X = rng.standard_normal((n, d)) * np.exp(rng.standard_normal((n, 1)))
    l = O.exact_leverage(X)
    assert np.all(l >= -1e-15) and np.all(l <= 1 + 1e-12)
    assert abs(l.sum() - d) < 1e-10 * n
    T = rng.standard_normal((d, d)) + 3 * np.eye(d)
    np.testing.assert_allclose(O.exact_leverage(X @ T), l, rtol=1e-9)
    np.testing.assert_allclose(O.exact_leverage(X * rng.uniform(0.1, 10, d)), l, rtol=1e-10)
    p = rng.permutation(n)
    np.testing.assert_allclose(O.exact_leverage(X[p]), l[p], rtol=1e-10)


# ---------------------------------------------------------------- Householder R
def test_householder_r_against_lapack_and_gram():
    rng = np.random.default_rng(4)
    A = rng.standard_normal((300, 40)) * np.exp(rng.standard_normal(40))
    R = O.householder_r(A)
    assert np.allclose(R, np.triu(R)) and np.all(np.diag(R) > 0)
    Rl = np.linalg.qr(A, mode="r")
    Rl = Rl * np.sign(np.diag(Rl))[:, None]
    np.testing.assert_allclose(R, Rl, rtol=1e-10, atol=1e-10 * np.abs(R).max())
    np.testing.assert_allclose(R.T @ R, A.T @ A, rtol=1e-11, atol=1e-11 * np.abs(A.T @ A).max())


def test_cholesky_of_gram_is_the_householder_r_and_gives_the_same_m():
    # With R_jj > 0 and full column rank, R is unique: the Cholesky factor of A^T A is the oracle's
    # Householder R, so R^-1 Pi (JL included) is the oracle's SVD-route M.  The GPU's Gram route
    # for R rests on this.
    rng = np.random.default_rng(11)
    A = rng.standard_normal((300, 40)) * np.exp(rng.standard_normal(40))
    R = O.householder_r(A)
    C = np.linalg.cholesky(A.T @ A).T
    np.testing.assert_allclose(C, R, rtol=1e-9, atol=1e-12 * np.abs(R).max())
    Pi = O.jl_matrix(40, 16, 5)
    sv = O.sketched_svd(A)
    M = O.m_matrix(sv["sigma"], sv["V"], sv["U_R"], sv["rank"], Pi)
    M_chol = np.linalg.solve(C, Pi)
    np.testing.assert_allclose(M_chol, M, rtol=1e-8, atol=1e-10 * np.abs(M).max())


def test_rank_deficient_r_is_not_unique_and_only_jl_scores_notice():
    # A repeated column: R_77 = 0 and a rotation of rows 7 and 8 gives another R with the same
    # R^T R.  The k = 0 scores (x R^+) do not change; R^+ Pi does.
    rng = np.random.default_rng(12)
    A = rng.standard_normal((60, 10))
    A[:, 7] = A[:, 2]
    R1 = O.householder_r(A)
    assert abs(R1[7, 7]) < 1e-12 * abs(R1).max()
    R1[7, 7] = 0.0
    G = np.eye(10)
    c, s_ = np.cos(0.7), np.sin(0.7)
    G[7, 7], G[7, 8], G[8, 7], G[8, 8] = c, s_, -s_, c
    R2 = G @ R1
    np.testing.assert_allclose(R2.T @ R2, R1.T @ R1, atol=1e-12 * np.abs(A.T @ A).max())
    P1, P2 = np.linalg.pinv(R1, rcond=1e-10), np.linalg.pinv(R2, rcond=1e-10)
    np.testing.assert_allclose(((A @ P1) ** 2).sum(1), ((A @ P2) ** 2).sum(1), rtol=1e-9)
    Pi = O.jl_matrix(10, 6, 3)
    assert np.max(np.abs((A @ P1 @ Pi) ** 2 - (A @ P2 @ Pi) ** 2).sum(1)) > 1e-3


def test_householder_r_exact_integer_gram():
    A = np.array([[2, 1, 0], [1, 3, 1], [0, 1, 4], [1, 0, 1], [2, 2, 2]], dtype=float)
    R = O.householder_r(A)
    G = [[sum(Fraction(int(A[i, a] * A[i, b])) for i in range(5)) for b in range(3)] for a in range(3)]
    np.testing.assert_allclose(R.T @ R, np.array(G, dtype=float), rtol=0, atol=1e-13)


def test_householder_r_zero_column_gives_exact_zero_column():
    rng = np.random.default_rng(5)
    A = rng.standard_normal((50, 8))
    A[:, 3] = 0.0
    R = O.householder_r(A)
    assert np.all(R[:, 3] == 0.0)
    np.testing.assert_allclose(R.T @ R, A.T @ A, atol=1e-12)
    sv = O.sketched_svd(A)
    assert sv["rank"] == 7 and sv["sigma"][-1] < 1e-14 * sv["sigma"][0]


def test_m_matrix_full_rank_equals_triangular_solve():
    rng = np.random.default_rng(6)
    A = rng.standard_normal((200, 30))
    sv = O.sketched_svd(A)
    Pi = O.jl_matrix(30, 16, 3)
    M = O.m_matrix(sv["sigma"], sv["V"], sv["U_R"], sv["rank"], Pi)
    np.testing.assert_allclose(M, sla.solve_triangular(sv["R"], Pi), rtol=1e-9, atol=1e-12)
    M0 = O.m_matrix(sv["sigma"], sv["V"], sv["U_R"], sv["rank"], None)
    x = rng.standard_normal((5, 30))
    np.testing.assert_allclose(np.sum((x @ M0) ** 2, 1),
                               np.sum(sla.solve_triangular(sv["R"], x.T, trans="T") ** 2, 0), rtol=1e-10)


# ---------------------------------------------------------------- sketched scores
def test_identity_and_orthogonal_sketch_reproduce_exact_scores():
    rng = np.random.default_rng(7)
    X = rng.standard_normal((120, 9)) * np.exp(rng.standard_normal((120, 1)))
    l = O.exact_leverage(X)
    sc, _, _ = O.scores_from_sketch(X, X)
    np.testing.assert_allclose(sc, l, rtol=1e-10)
    Q, _ = np.linalg.qr(rng.standard_normal((120, 120)))
    sc, _, _ = O.scores_from_sketch(X, Q @ X)
    np.testing.assert_allclose(sc, l, rtol=1e-9)


def test_approx_u_with_identity_sketch_is_the_exact_left_singular_basis():
    """S = I: U = X V Sigma^-1 are X's left singular vectors (numpy's SVD, up to column signs),
    orthonormal, and U Sigma V^T = X; with zero columns only r = rank columns are kept."""
    rng = np.random.default_rng(21)
    X = rng.standard_normal((200, 7)) * np.exp(rng.standard_normal(7))
    U, info = O.approx_u_from_sketch(X, X)
    Uw, sw, _ = np.linalg.svd(X, full_matrices=False)
    assert info["rank"] == 7
    np.testing.assert_allclose(np.abs(np.sum(U * Uw, axis=0)), 1.0, atol=1e-10)
    np.testing.assert_allclose(U.T @ U, np.eye(7), atol=1e-10)
    np.testing.assert_allclose(U * info["sigma"] @ info["V"].T, X, atol=1e-10 * np.abs(X).max())
    X[:, [1, 4]] = 0.0
    U, info = O.approx_u_from_sketch(X, X)
    assert info["rank"] == 5 and U.shape == (200, 5)
    np.testing.assert_allclose(U.T @ U, np.eye(5), atol=1e-10)


@pytest.mark.parametrize("kind", ["countsketch", "gaussian"])
def test_approx_u_row_norms_are_the_sketched_scores(kind):
    """||U_i||^2 equals Algorithm 3's score of row i (k = 0, same sketch)."""
    X = np.random.default_rng(22).standard_normal((3000, 12))
    U, info = O.approx_u(X, kind, 256, 9)
    sc, _ = O.sketched_leverage(X, kind, 256, 0, 9, 0)
    np.testing.assert_allclose(np.sum(U * U, axis=1), sc, rtol=1e-9)


@pytest.mark.parametrize("kind", ["countsketch", "srht", "gaussian", "osnap"])
def test_sketch_of_identity_has_unit_columns_in_expectation(kind):
    n, s = 256, 64
    SI = O.sketch(np.eye(n), kind, s, 9)
    norms = np.sum(SI**2, axis=0)
    if kind == "gaussian":
        assert abs(norms.mean() - 1.0) < 5 * math.sqrt(2.0 / s) / math.sqrt(n)
    else:  # one +-1 per column (CountSketch); (1/s) sum of s squared +-1 entries (SRHT);
        # z entries +-1/sqrt(z) in z distinct rows (OSNAP)
        np.testing.assert_allclose(norms, 1.0, rtol=1e-14)


def test_full_srht_is_an_isometry():
    rng = np.random.default_rng(8)
    n, d = 64, 6
    X = rng.standard_normal((n, d))
    SX = O.sketch_srht(X, n, 3)  # s = n_pad: every Hadamard row kept
    np.testing.assert_allclose(SX.T @ SX, X.T @ X, rtol=1e-12, atol=1e-12)
    sc, _ = O.sketched_leverage(X, "srht", n, 0, 3, 0)
    np.testing.assert_allclose(sc, O.exact_leverage(X), rtol=1e-10)


def test_collision_free_countsketch_is_an_isometry():
    n, s = 12, 1 << 24
    seed = next(sd for sd in range(100) if len(set(O.countsketch_hash(n, s, sd)[0])) == n)
    X = np.random.default_rng(9).standard_normal((n, 3))
    SX = O.sketch_countsketch(X, s, seed)
    np.testing.assert_allclose(SX.T @ SX, X.T @ X, rtol=1e-14)


@pytest.mark.parametrize("z", [1, 2, 4, 8])
def test_osnap_columns_have_one_entry_per_block(z):
    """Column i of S: exactly z nonzeros, one in each block of s/z rows, each +-1/sqrt(z)."""
    n, s = 300, 64
    SI = O.sketch(np.eye(n), "osnap", s, 5, nnz=z)
    m = s // z
    for b in range(z):
        blk = SI[b * m:(b + 1) * m]
        np.testing.assert_array_equal(np.count_nonzero(blk, axis=0), np.ones(n))
    np.testing.assert_allclose(np.abs(SI[SI != 0]), 1 / math.sqrt(z), rtol=1e-15)


def test_collision_free_osnap_is_an_isometry():
    n, s, z = 12, 1 << 24, 4
    seed = next(sd for sd in range(100) if len(set(O.osnap_hash(n, s, z, sd)[0].ravel().tolist())) == n * z)
    X = np.random.default_rng(9).standard_normal((n, 3))
    SX = O.sketch_osnap(X, s, seed, z)
    np.testing.assert_allclose(SX.T @ SX, X.T @ X, rtol=1e-13)
    sc, _, _ = O.scores_from_sketch(X, SX)
    np.testing.assert_allclose(sc, O.exact_leverage(X), rtol=1e-10)


@pytest.mark.parametrize("kind,s", [("countsketch", 2048), ("srht", 512), ("gaussian", 256), ("osnap", 512)])
def test_sketched_scores_lie_in_subspace_embedding_band(kind, s):
    """For Pi = I: l_i / sigma_max(SU)^2 <= l~_i <= l_i / sigma_min(SU)^2, U an orthonormal basis."""
    rng = np.random.default_rng(10)
    n, d = 3000, 16
    X = rng.standard_normal((n, d)) * np.exp(rng.standard_normal((n, 1)))
    l = O.exact_leverage(X)
    sc, info = O.sketched_leverage(X, kind, s, 0, 21, 0)
    U, _ = np.linalg.qr(X)
    sig = np.linalg.svd(O.sketch(U, kind, s, 21), compute_uv=False)
    lo, hi = l / sig[0] ** 2, l / sig[-1] ** 2
    assert np.all(sc >= lo * (1 - 1e-9)) and np.all(sc <= hi * (1 + 1e-9))
    assert info["rank"] == d
    # the sketch is a good embedding at these sizes: the band is narrow
    assert sig[0] ** 2 < 1.6 and sig[-1] ** 2 > 0.6


def test_rank_from_zero_columns_and_duplicates():
    rng = np.random.default_rng(11)
    n, d = 4000, 24
    X = rng.standard_normal((n, d))
    X[:, [2, 5, 11]] = 0.0
    for kind, s in (("countsketch", 1024), ("srht", 256), ("gaussian", 128)):
        _, info = O.sketched_leverage(X, kind, s, 0, 5, 0)
        assert info["rank"] == d - 3
    # Fig. 2 analogue: rank d/2 through duplicated columns
    B = rng.standard_normal((n, d // 2))
    Xd = np.hstack([B, B @ np.diag(rng.uniform(0.5, 2, d // 2))])
    sc, info = O.sketched_leverage(Xd, "countsketch", 1024, 0, 5, 0)
    assert info["rank"] == d // 2
    l = O.exact_leverage(Xd)
    assert np.median(np.abs(sc / l - 1)) < 0.2
    # without truncation (tau = 0) the inverted tiny singular values wreck the scores
    sc0, info0 = O.sketched_leverage(Xd, "countsketch", 1024, 0, 5, 0, tau=0.0)
    assert info0["rank"] == d
    assert not np.all(np.isfinite(sc0)) or np.median(np.abs(sc0 / l - 1)) > 1.0


def test_jl_scores_are_unbiased():
    rng = np.random.default_rng(12)
    n, d, k = 600, 12, 32
    X = rng.standard_normal((n, d)) * np.exp(rng.standard_normal((n, 1)))
    base, _ = O.sketched_leverage(X, "gaussian", 96, 0, 4, 0)
    ratios = np.mean([O.sketched_leverage(X, "gaussian", 96, k, 4, sp)[0] / base for sp in range(64)], axis=0)
    assert np.all(np.abs(ratios - 1) < 4 * math.sqrt(2.0 / k) / math.sqrt(64) * 1.5)


# ---------------------------------------------------------------- ordering
def test_order_dec_matches_brute_force_sort():
    vals = [0.5, 0.1, float("nan"), 0.5, -0.0, 0.0, 0.9, 0.1, float("nan"), 1e-30, -math.inf, math.inf,
            -math.inf]
    want = sorted(range(len(vals)), key=lambda i: (math.isnan(vals[i]), -vals[i] if not math.isnan(vals[i]) else 0, i))
    assert O.order_dec(np.array(vals)).tolist() == want
    assert O.order_dec(np.full(7, 0.25)).tolist() == list(range(7))


def test_sampling_probabilities_sum_to_one():
    p = O.sampling_probabilities(np.array([1.0, 3.0, 0.0, 4.0]))
    np.testing.assert_allclose(p, [0.125, 0.375, 0.0, 0.5])


def test_image_like_rank_is_live_column_count():
    """Image-like data with 68 all-zero columns: numerical rank 716 from every sketch."""
    from paper_1812_07903_gb300 import inputs
    X, zero_cols = inputs.image_like(n=6000, seed=1001)
    X = X.numpy().astype(np.float64)
    assert zero_cols.size == 68 and np.all(X[:, zero_cols] == 0)
    for kind, s in (("countsketch", 2048), ("srht", 1024)):
        _, info = O.sketched_leverage(X, kind, s, 0, 2002, 0)
        assert info["rank"] == 716


def test_lapack_householder_matches_column_loop_including_zero_columns():
    """dgeqrf and the column loop give the same R, also for exactly zero columns (leftover rows)."""
    rng = np.random.default_rng(21)
    A = rng.standard_normal((400, 30)) * np.exp(rng.standard_normal(30))
    A[:, [4, 17]] = 0.0
    R1, R2 = O.householder_r(A), O.householder_r_lapack(A)
    np.testing.assert_allclose(R2, R1, rtol=0, atol=1e-12 * np.abs(R1).max())
    assert np.any(R1[4, 5:] != 0.0)  # the leftover row of a zero column is not zero
    B = rng.standard_normal((300, 50))
    np.testing.assert_allclose(O.householder_r_lapack(B), O.householder_r(B), atol=1e-12 * np.abs(B).max() * 20)


def test_partial_householder_steps_are_a_prefix():
    rng = np.random.default_rng(22)
    A = rng.standard_normal((80, 12))
    R = O.householder_r(A)
    Rp = O.householder_r(A, steps=5)
    np.testing.assert_allclose(Rp[:5], R[:5], atol=1e-13)


def _gram_fractions(A):
    """SX^T SX in exact rationals, each entry rounded once to float64 (Fraction -> float rounds
    to nearest)."""
    F = [[Fraction(float(v)) for v in row] for row in A]
    s, d = len(F), len(F[0])
    G = np.empty((d, d))
    for i in range(d):
        for j in range(d):
            G[i, j] = float(sum(F[r][i] * F[r][j] for r in range(s)))
    return G


@pytest.mark.parametrize("case", ["gaussian", "spread", "integers", "zero_column", "tiny"])
def test_gram_is_the_exactly_rounded_sx_t_sx(case):
    rng = np.random.default_rng(7)
    if case == "gaussian":
        A = rng.standard_normal((37, 6))
    elif case == "spread":  # entries over 30 binary orders within each column, mixed signs
        A = rng.standard_normal((41, 5)) * np.exp2(rng.integers(-30, 1, size=(41, 5)))
    elif case == "integers":
        A = rng.integers(-(2**16) + 1, 2**16, size=(29, 4)).astype(np.float64)
    elif case == "zero_column":
        A = rng.standard_normal((23, 4))
        A[:, 2] = 0.0
    else:  # columns scaled far below 1 and far above (cross products of order 1, squares near the ends)
        A = rng.standard_normal((19, 3)) * np.array([1e-160, 1.0, 1e150])
    G = O.gram(A)
    np.testing.assert_array_equal(G, _gram_fractions(A))
    assert np.array_equal(G, G.T)
