"""FP64 CPU oracle for Sketched Leverage Score Ordering (Chin & Liang, ACML 2018).

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` may import or call this module.  The product path
(the CUDA library under ``paper_1812_07903_gb300/``) never imports it, and this module
imports nothing from the product: the two share no code.  The only thing both sides
consume in common is seeded input data, produced by a module that holds none of the
method's arithmetic.

Every function is a plain, slow restatement of the paper's definitions in float64,
written for a reader to check against the paper by eye.  Library primitives (matrix
products, LAPACK's SVD, sorting) serve as single steps; nothing is blocked, fused or
reordered beyond that.

Randomness.  The paper's sketches are random; here every random draw comes from
Philox4x32-10 (Salmon, Moraes, Dror, Shaw, "Parallel random numbers: as easy as 1, 2,
3", SC'11), written from its published definition.  The CUDA side implements the same
generator independently.  Counter layouts (word 3 of the counter is a stream tag):

  CountSketch row i      ctr=(lo(i), hi(i), 0, 1)  bucket=(w0*s)>>32, sign=1-2*(w1&1)
  SRHT sign of row i     ctr=(lo(i), hi(i), 0, 2)  D_i = 1-2*(w0&1)
  SRHT sample key of j   ctr=(lo(j), hi(j), 0, 3)  key_j = w0; keep the s smallest (key, j)
  Gaussian entry (j, i)  ctr=(lo(b), hi(b), j, 4), b = i // 4: i % 4 = 0, 1, 2, 3 give
                         bf16 of BoxMuller(w0, w1), BoxMuller(w0, w1 - 2^30),
                         BoxMuller(w2, w3), BoxMuller(w2, w3 - 2^30)  (cos, sin of each pair)
  JL entry (j, c)        ctr=(lo(c), hi(c), j, 5)  Pi_jc = BoxMuller(w0, w1) / sqrt(k)
  sampling draw t        ctr=(lo(t), hi(t), 0, 6)  u_t = (m + 1/2) 2^-52, m = w0 2^20 + (w1 >> 12)
  OSNAP row i, block b   ctr=(lo(i), hi(i), b, 7)  bucket = b s/z + ((w0 s/z) >> 32), sign = 1-2*(w1&1)

with key = (lo(seed), hi(seed)), BoxMuller(w0, w1) = sqrt(-2 ln u1) cos(2 pi u2),
u1 = (w0 + 1) 2^-32 in (0, 1], u2 = w1 2^-32 in [0, 1).

Parity status of each function is stated in its docstring; every function here is
pinned by a test in ``tests/test_oracle_*.py`` to something other than itself.
"""
from __future__ import annotations

import math
from fractions import Fraction

import numpy as np

# ---------------------------------------------------------------------------
# Philox4x32-10 (Salmon et al., SC'11, Sec. 4 "Philox")
# ---------------------------------------------------------------------------
_PHILOX_M0 = np.uint64(0xD2511F53)
_PHILOX_M1 = np.uint64(0xCD9E8D57)
_PHILOX_W0 = 0x9E3779B9
_PHILOX_W1 = 0xBB67AE85
_MASK32 = np.uint64(0xFFFFFFFF)
_SH32 = np.uint64(32)

TAG_COUNTSKETCH = 1
TAG_SRHT_SIGN = 2
TAG_SRHT_SAMPLE = 3
TAG_GAUSSIAN = 4
TAG_JL = 5
TAG_SAMPLE = 6
TAG_OSNAP = 7
OSNAP_DEFAULT_NNZ = 4


def philox4x32_10(c0, c1, c2, c3, key):
    """Philox4x32 with 10 rounds, vectorised over the counter words.

    Counter words are integer arrays (or scalars) holding 32-bit values; ``key`` is a
    64-bit seed split into two 32-bit key words (low word first).  Each round multiplies
    words 0 and 2 by the two Philox multipliers, and mixes the high halves with the odd
    words and the round key; the key is bumped by the two Weyl constants between rounds.
    Returns four uint64 arrays holding 32-bit outputs.
    """
    c = [np.asarray(x, dtype=np.uint64) & _MASK32 for x in (c0, c1, c2, c3)]
    k0 = int(key) & 0xFFFFFFFF
    k1 = (int(key) >> 32) & 0xFFFFFFFF
    for r in range(10):
        if r:
            k0 = (k0 + _PHILOX_W0) & 0xFFFFFFFF
            k1 = (k1 + _PHILOX_W1) & 0xFFFFFFFF
        p0 = _PHILOX_M0 * c[0]
        p1 = _PHILOX_M1 * c[2]
        c = [
            (p1 >> _SH32) ^ c[1] ^ np.uint64(k0),
            p1 & _MASK32,
            (p0 >> _SH32) ^ c[3] ^ np.uint64(k1),
            p0 & _MASK32,
        ]
    return c


def _split64(i):
    i = np.asarray(i, dtype=np.uint64)
    return i & _MASK32, i >> _SH32


def box_muller(w0, w1):
    """Standard normal from two 32-bit words: sqrt(-2 ln u1) cos(2 pi u2), in float64.

    u1 = (w0 + 1) 2^-32 and u2 = w1 2^-32.  Both factors are evaluated from exact
    arguments so the float64 value is accurate to a few ulp everywhere:
    * ln u1 = log1p(-m 2^-32) with m = 2^32 - 1 - w0 when w0 >= 2^31, else log(u1);
    * the angle 2 pi u2 is split into its octant o = w1 >> 29 and the exact fraction
      a = (w1 mod 2^29) 2^-29, so cos(2 pi u2) is +-sin or +-cos of (pi/4) c with
      c = a (even octant) or c = 1 - a (odd octant), c in [0, 1].
    """
    w0 = np.asarray(w0, dtype=np.uint64)
    w1 = np.asarray(w1, dtype=np.uint64)
    hi = w0 >= np.uint64(1 << 31)
    m = (np.uint64(0xFFFFFFFF) - w0).astype(np.float64)
    u1 = (w0.astype(np.float64) + 1.0) * 2.0**-32
    ln_u1 = np.where(hi, np.log1p(-m * 2.0**-32), np.log(u1))
    rho = np.sqrt(-2.0 * ln_u1)
    octant = (w1 >> np.uint64(29)).astype(np.int64)
    frac = (w1 & np.uint64((1 << 29) - 1)).astype(np.float64) * 2.0**-29
    odd = (octant & 1) == 1
    c = np.where(odd, 1.0 - frac, frac)
    phi = (np.pi / 4.0) * c
    sn, cs = np.sin(phi), np.cos(phi)
    q = np.where(odd, (octant + 1) // 2, octant // 2)  # quarter turns, 0..4
    # cos(q pi/2 + phi) for even octants, cos(q pi/2 - phi) for odd ones
    val = np.select(
        [q == 0, q == 1, q == 2, q == 3, q == 4],
        [cs, np.where(odd, sn, -sn), -cs, np.where(odd, -sn, sn), cs],
    )
    return rho * val


def bf16_round(x):
    """Round float64 values to bfloat16 (8 significant bits), round-to-nearest-even.

    Done on the float64 bit pattern in one step (no double rounding through float32):
    drop the low 45 mantissa bits, adding half an ulp minus one plus the kept lsb.
    Valid for finite values inside bfloat16's normal range and zero, which covers every
    Box-Muller output.  Returns float64 values that are exactly bfloat16-representable.
    """
    b = np.ascontiguousarray(x, dtype=np.float64).view(np.uint64)
    lsb = (b >> np.uint64(45)) & np.uint64(1)
    b = (b + np.uint64((1 << 44) - 1) + lsb) & ~np.uint64((1 << 45) - 1)
    return b.view(np.float64)


# ---------------------------------------------------------------------------
# Seeded sketch ingredients (Sec. 2.1 sketch families; Sec. 3.1.2 implementations)
# ---------------------------------------------------------------------------
def countsketch_hash(n, s, seed):
    """CountSketch's pair of hash functions (Sec. 3.1.2): bucket h(i) in [s], sign(i) = +-1.

    bucket = floor(w0 * s / 2^32) (multiply-shift), sign = 1 - 2 (w1 & 1).
    """
    lo, hi = _split64(np.arange(n, dtype=np.uint64))
    w = philox4x32_10(lo, hi, 0, TAG_COUNTSKETCH, seed)
    bucket = ((w[0] * np.uint64(s)) >> _SH32).astype(np.int64)
    sign = 1.0 - 2.0 * (w[1] & np.uint64(1)).astype(np.float64)
    return bucket, sign


def srht_signs(n, seed):
    """Diagonal of random signs D of the SRHT (Sec. 2.1, Sec. 3.1.2)."""
    lo, hi = _split64(np.arange(n, dtype=np.uint64))
    w = philox4x32_10(lo, hi, 0, TAG_SRHT_SIGN, seed)
    return 1.0 - 2.0 * (w[0] & np.uint64(1)).astype(np.float64)


def srht_sample(n_pad, s, seed):
    """Row sample P of the SRHT: s distinct rows of the n_pad-point Hadamard transform.

    A uniform s-subset drawn without replacement: each j gets a 32-bit key, and the s
    smallest (key, j) pairs are kept.  Returned in ascending j, the row order of SX.
    """
    j = np.arange(n_pad, dtype=np.uint64)
    lo, hi = _split64(j)
    key = philox4x32_10(lo, hi, 0, TAG_SRHT_SAMPLE, seed)[0].astype(np.int64)
    first = np.lexsort((j.astype(np.int64), key))[:s]
    return np.sort(first).astype(np.int64)


def gaussian_block(rows, cols, seed):
    """Entries G[rows, cols] of the s x n Gaussian sketch matrix, before the 1/sqrt(s) scale.

    G_ji = bf16(N(0,1)).  Four consecutive columns share one Philox block: the block of
    column i is b = i // 4 with counter (lo(b), hi(b), j, 4), and its words (w0, w1, w2, w3)
    give the two independent normals of a Box-Muller pair each,
      i % 4 = 0: rho(w0) cos(2 pi w1 2^-32)      i % 4 = 1: rho(w0) sin(2 pi w1 2^-32)
      i % 4 = 2: rho(w2) cos(2 pi w3 2^-32)      i % 4 = 3: rho(w2) sin(2 pi w3 2^-32)
    with sin(2 pi w 2^-32) = cos(2 pi (w - 2^30) 2^-32) evaluated by ``box_muller`` on the
    shifted word (exact modulo 2^32).
    """
    rows = np.asarray(rows, dtype=np.uint64)
    cols = np.asarray(cols, dtype=np.uint64)
    J, I = np.meshgrid(rows, cols, indexing="ij")
    lo, hi = _split64(I >> np.uint64(2))
    w = philox4x32_10(lo, hi, J, TAG_GAUSSIAN, seed)
    r = I & np.uint64(3)
    wa = np.where(r < 2, w[0], w[2])
    wb = np.where(r < 2, w[1], w[3])
    wb = np.where((r & np.uint64(1)) == 1, (wb - np.uint64(1 << 30)) & _MASK32, wb)
    return bf16_round(box_muller(wa, wb))


def jl_matrix(d, k, seed):
    """Johnson-Lindenstrauss matrix Pi (d x k), entries N(0, 1/k), float64 (not rounded)."""
    J, C = np.meshgrid(np.arange(d, dtype=np.uint64), np.arange(k, dtype=np.uint64), indexing="ij")
    lo, hi = _split64(C)
    w = philox4x32_10(lo, hi, J, TAG_JL, seed)
    return box_muller(w[0], w[1]) / math.sqrt(k)


def hadamard_entries(rows, cols):
    """Entries of the unnormalised Sylvester-Walsh-Hadamard matrix: (-1)^popcount(j & i)."""
    a = np.bitwise_and.outer(np.asarray(rows, dtype=np.uint64), np.asarray(cols, dtype=np.uint64))
    return 1.0 - 2.0 * (np.bitwise_count(a) & 1).astype(np.float64)


def next_pow2(n):
    return 1 << max(0, int(n - 1).bit_length())


# ---------------------------------------------------------------------------
# Sketch SA (Algorithm 2/3 step 1).  S normalised so that E[S^T S] = I.
# ---------------------------------------------------------------------------
_CHUNK = 1 << 15


def sketch_countsketch(X, s, seed):
    """SX for CountSketch: row b of SX is the signed sum of the rows i with h(i) = b.

    Written as the sparse product S X with S[h(i), i] = sign(i); each row of S sums its
    nonzeros in ascending i.
    """
    import scipy.sparse as sp

    n, d = X.shape
    bucket, sign = countsketch_hash(n, s, seed)
    SX = np.zeros((s, d), dtype=np.float64)
    for a in range(0, n, _CHUNK):
        b = min(n, a + _CHUNK)
        S = sp.csr_matrix((sign[a:b], (bucket[a:b], np.arange(b - a))), shape=(s, b - a))
        SX += S @ np.asarray(X[a:b], dtype=np.float64)
    return SX


def osnap_hash(n, s, z, seed):
    """OSNAP (Nelson and Nguyen; the paper's variant of CountSketch, Sec. 3.1.2) in its block
    form: the s rows of S are z blocks of s/z rows, and column i of S has one nonzero in each
    block, +-1/sqrt(z) at row b s/z + h_b(i), with (h_b, sign_b) hashed like CountSketch from
    the Philox block (lo i, hi i, b, 7).  Returns (bucket, sign) arrays of shape (z, n)."""
    if s % z != 0:
        raise ValueError("OSNAP needs s divisible by z")
    m = s // z
    lo, hi = _split64(np.arange(n, dtype=np.uint64))
    buckets, signs = [], []
    for b in range(z):
        w = philox4x32_10(lo, hi, b, TAG_OSNAP, seed)
        buckets.append(((w[0] * np.uint64(m)) >> _SH32).astype(np.int64) + b * m)
        signs.append(1.0 - 2.0 * (w[1] & np.uint64(1)).astype(np.float64))
    return np.stack(buckets), np.stack(signs)


def sketch_osnap(X, s, seed, nnz=OSNAP_DEFAULT_NNZ):
    """SX for OSNAP with nnz nonzeros per column of S: the sparse product S X, rows of S summing
    their nonzeros in ascending i."""
    import scipy.sparse as sp

    n, d = X.shape
    bucket, sign = osnap_hash(n, s, nnz, seed)
    SX = np.zeros((s, d), dtype=np.float64)
    for a in range(0, n, _CHUNK):
        b = min(n, a + _CHUNK)
        rows = bucket[:, a:b].ravel()
        cols = np.tile(np.arange(b - a), nnz)
        vals = sign[:, a:b].ravel() / math.sqrt(nnz)
        S = sp.csr_matrix((vals, (rows, cols)), shape=(s, b - a))
        SX += S @ np.asarray(X[a:b], dtype=np.float64)
    return SX


def sketch_srht(X, s, seed):
    """SX for the subsampled randomized Hadamard transform sqrt(n_pad/s) P (H/sqrt(n_pad)) D.

    X is zero-padded to n_pad = 2^ceil(log2 n) rows (padding rows contribute nothing),
    so SX = (1/sqrt(s)) H[sample, :n] D X with H the unnormalised Hadamard matrix.
    """
    n, d = X.shape
    n_pad = next_pow2(n)
    if s > n_pad:
        raise ValueError("SRHT needs s <= n_pad")
    D = srht_signs(n, seed)
    sample = srht_sample(n_pad, s, seed)
    SX = np.zeros((s, d), dtype=np.float64)
    for a in range(0, n, _CHUNK):
        b = min(n, a + _CHUNK)
        H = hadamard_entries(sample, np.arange(a, b))
        SX += H @ (D[a:b, None] * np.asarray(X[a:b], dtype=np.float64))
    return SX / math.sqrt(s)


def sketch_gaussian(X, s, seed):
    """SX for the dense Gaussian sketch (1/sqrt(s)) G X, G_ji = bf16(N(0,1))."""
    n, d = X.shape
    SX = np.zeros((s, d), dtype=np.float64)
    rows = np.arange(s)
    for a in range(0, n, _CHUNK):
        b = min(n, a + _CHUNK)
        SX += gaussian_block(rows, np.arange(a, b), seed) @ np.asarray(X[a:b], dtype=np.float64)
    return SX / math.sqrt(s)


SKETCHES = {"countsketch": sketch_countsketch, "srht": sketch_srht, "gaussian": sketch_gaussian,
            "osnap": sketch_osnap}


def sketch(X, kind, s, seed, nnz=None):
    """Algorithm 2/3 step 1: the sketch SA of the data matrix (nnz: OSNAP's nonzeros per column)."""
    if kind == "osnap" and nnz:
        return sketch_osnap(X, s, seed, nnz)
    return SKETCHES[kind](X, s, seed)


# ---------------------------------------------------------------------------
# Small solve: Householder QR -> R, SVD of R, rank, M (Algorithm 3 steps 2-4)
# ---------------------------------------------------------------------------
def householder_r(A, steps=None):
    """R factor of an unpivoted Householder QR of A (s x d, s >= d), in float64.

    Column j: alpha = A[j, j], xnorm = ||A[j+1:, j]||.  If xnorm = 0 no reflection is
    applied (H_j = I) and R_jj = alpha.  Otherwise beta = -sign(alpha) sqrt(alpha^2 +
    xnorm^2) with sign(alpha) = +1 for alpha >= 0 (including -0), tau = (beta - alpha) /
    beta, v = A[j:, j] / (alpha - beta) with v_0 = 1, R_jj = beta, and H_j = I - tau v v^T
    is applied to the trailing columns.  Finally every row of R with a negative diagonal
    is negated, so R_jj >= 0 (the unique R for full column rank A).

    ``steps`` stops after that many columns (only used to time a bounded sample).
    """
    A = np.array(A, dtype=np.float64, copy=True)
    s, d = A.shape
    if s < d:
        raise ValueError("householder_r needs s >= d")
    for j in range(d if steps is None else min(d, steps)):
        alpha = A[j, j]
        xnorm = math.sqrt(float(np.dot(A[j + 1:, j], A[j + 1:, j])))
        if xnorm == 0.0:
            continue
        norm = math.sqrt(alpha * alpha + xnorm * xnorm)
        beta = -norm if alpha >= 0.0 else norm
        tau = (beta - alpha) / beta
        v = A[j:, j] / (alpha - beta)
        v[0] = 1.0
        A[j, j] = beta
        A[j + 1:, j] = 0.0
        if j + 1 < d:
            w = v @ A[j:, j + 1:]
            A[j:, j + 1:] -= tau * np.outer(v, w)
    R = np.triu(A[:d, :d])
    neg = np.diag(R) < 0.0
    R[neg, :] *= -1.0
    return R


def gram(SX):
    """G = SX^T SX with every entry the float64 rounding of its exact value (the Gram matrix whose
    Cholesky factor is the R of Algorithm 2/3 step 2 at full column rank).

    Exact arithmetic by integer pieces: column j is scaled by 2^-k_j (k_j from frexp of its
    largest magnitude, so the scaled entries lie in (-1, 1)) and cut into five 17-bit integer
    pieces, a' 2^85 = sum_p P_p 2^(17 (4 - p)) + rem with |rem| < 1.  Float64 matrix products of
    pieces, and the up to five of them of equal order t = p + q, are exact in any summation order
    while s < 2^16 (every partial sum is an integer below 5 s 2^34 < 2^53); they are combined as Python
    integers V = sum_t 2^(17 (8 - t)) C_t, and G_ij = V_ij 2^(k_i + k_j - 170) is rounded once.
    Exact whenever every entry's bits lie within 85 bits of its column's largest magnitude
    (always for entries at least 2^-32 of it); below that, within 2^-85 of it.
    """
    A = np.asarray(SX, dtype=np.float64)
    s, d = A.shape
    if s >= 1 << 16:
        raise ValueError("gram: s must be below 2^16 for exact piece products")
    if not np.all(np.isfinite(A)):
        raise ValueError("gram: SX must be finite")
    colmax = np.max(np.abs(A), axis=0) if s else np.zeros(d)
    k = np.zeros(d, dtype=np.int64)
    nz = colmax > 0
    k[nz] = np.frexp(colmax[nz])[1]
    a = np.ldexp(A, -k[None, :])  # exact: scaling by a power of two
    pieces = []
    for _ in range(5):
        a = a * 131072.0  # 2^17, exact
        P = np.trunc(a)
        a = a - P  # exact: the remainder has fewer bits than a
        pieces.append(P)
    V = np.zeros((d, d), dtype=object)
    for t in range(9):
        C = np.zeros((d, d))
        for p in range(5):
            q = t - p
            if 0 <= q < 5:
                C += pieces[p].T @ pieces[q]  # integers below 2^53: exact
        V = V + np.vectorize(int, otypes=[object])(C) * (1 << (17 * (8 - t)))
    G = np.empty((d, d))
    for i in range(d):
        for j in range(d):
            v, e = int(V[i, j]), int(k[i] + k[j]) - 170
            if v == 0:
                G[i, j] = 0.0
            elif v.bit_length() + e > 1024:
                G[i, j] = math.copysign(math.inf, v)
            elif v.bit_length() + e < -1020:  # subnormal range: round the exact rational once
                G[i, j] = float(Fraction(v) * Fraction(2) ** e)
            else:
                G[i, j] = math.ldexp(float(v), e)  # float(v) rounds once; the scaling is exact
    return G


def householder_r_lapack(A):
    """The same R through LAPACK's Householder QR (dgeqrf, via numpy), rows sign-normalised.

    dgeqrf forms the same reflectors as ``householder_r`` (no reflection for an exactly zero
    subcolumn, beta = -sign(alpha) ||x||), blocked for speed; used at sizes where the
    column loop is too slow.  Agreement with ``householder_r`` is pinned by a test.
    """
    R = np.linalg.qr(np.asarray(A, dtype=np.float64), mode="r")
    neg = np.diag(R) < 0.0
    R[neg, :] *= -1.0
    return R


def default_tau(s, d):
    """Relative rank threshold when none is given: max(s, d) * 2^-52 (FP64 numerical rank)."""
    return max(s, d) * 2.0**-52


def svd_of_r(R):
    """SVD of the small triangular factor, R = U_R diag(sigma) V^T, sigma descending.

    A library step (LAPACK via numpy), as in the paper's own implementation (Sec. 3.1.1).
    sigma equals the singular values of SX, and V its right singular vectors (Alg 3 step 2).
    """
    U, sigma, Vt = np.linalg.svd(R)
    return sigma, Vt.T, U


def numerical_rank(sigma, tau):
    """Algorithm 3 step 3, read as a relative threshold: r = #{sigma_j > tau * sigma_1}."""
    if sigma.size == 0 or sigma[0] == 0.0:
        return 0
    return int(np.count_nonzero(sigma > tau * sigma[0]))


def m_matrix(sigma, V, U_R, rank, Pi):
    """M = R^+_tau Pi = V_r diag(1/sigma_r) U_R,r^T Pi  (Pi is None: M = V_r diag(1/sigma_r)).

    With Pi = I the scores ||x_i M||^2 equal Algorithm 3's ||x_i V' Sigma'^-1||^2 exactly,
    because U_R,r has orthonormal columns.
    """
    Vr = V[:, :rank] / sigma[:rank]
    if Pi is None:
        return Vr
    return Vr @ (U_R[:, :rank].T @ Pi)


def row_scores(X, M):
    """Algorithm 3 step 5: l_i = ||(X M)_i||^2 in float64, rows streamed in chunks."""
    n = X.shape[0]
    out = np.empty(n, dtype=np.float64)
    for a in range(0, n, _CHUNK):
        b = min(n, a + _CHUNK)
        Y = np.asarray(X[a:b], dtype=np.float64) @ M
        out[a:b] = np.einsum("ij,ij->i", Y, Y)
    return out


def sketched_svd(SX, tau=None, qr="loop"):
    """Sketched SVD (Algorithm 2/3 steps 2-3): R, sigma, V, U_R and numerical rank of SX."""
    s, d = SX.shape
    if tau is None or tau < 0:
        tau = default_tau(s, d)
    R = householder_r(SX) if qr == "loop" else householder_r_lapack(SX)
    sigma, V, U_R = svd_of_r(R)
    return {"R": R, "sigma": sigma, "V": V, "U_R": U_R, "rank": numerical_rank(sigma, tau), "tau": tau}


def scores_from_sketch(X, SX, tau=None, Pi=None, qr="loop"):
    """Algorithm 3 steps 2-5 from a given sketch SX: truncated basis, then row norms."""
    sv = sketched_svd(SX, tau, qr)
    M = m_matrix(sv["sigma"], sv["V"], sv["U_R"], sv["rank"], Pi)
    return row_scores(X, M), sv, M


def sketched_leverage(X, kind, s, k, seed_S, seed_Pi, tau=None, qr="loop"):
    """Algorithm 3 (Approximate Leverage Score with Truncation) with a JL step.

    k = 0 gives the algorithm exactly (Pi = I); k > 0 right-multiplies R^+_tau by the
    seeded d x k JL matrix Pi.  Returns (scores, info dict).
    """
    d = X.shape[1]
    SX = sketch(X, kind, s, seed_S)
    Pi = jl_matrix(d, k, seed_Pi) if k > 0 else None
    scores, sv, M = scores_from_sketch(X, SX, tau, Pi, qr)
    info = {
        "rank": sv["rank"],
        "sigma": sv["sigma"],
        "tau": sv["tau"],
        "R": sv["R"],
        "M": M,
        "SX": SX,
        "score_sum": float(np.sum(scores)),
    }
    return scores, info


def approx_u_from_sketch(X, SX, tau=None, qr="loop"):
    """Approximate left singular vectors (Algorithm 2 step 3; Algorithm 3 step 4 with the
    transpose read as a typo) from a given sketch: SX = U' Sigma V^T, U = X V_r Sigma_r^-1 for the
    r retained singular values (n x r).  Returns (U, info dict with rank, sigma, V, tau)."""
    X = np.asarray(X, dtype=np.float64)
    sv = sketched_svd(np.asarray(SX, dtype=np.float64), tau, qr)
    r = sv["rank"]
    U = X @ (sv["V"][:, :r] / sv["sigma"][:r])
    return U, {"rank": r, "sigma": sv["sigma"], "V": sv["V"], "tau": sv["tau"]}


def approx_u(X, kind, s, seed_S, tau=None, qr="loop"):
    """``approx_u_from_sketch`` with the seeded sketch of ``sketch``."""
    return approx_u_from_sketch(X, sketch(np.asarray(X, dtype=np.float64), kind, s, seed_S), tau, qr)


def exact_leverage(X, tau=None):
    """Exact leverage scores (Sec. 2.2; Algorithm 1): l_i = ||U_i||^2 over the numerical rank.

    U from the thin SVD of X; columns kept where sigma_j > tau * sigma_1 (default tau =
    max(n, d) 2^-52).  This is the diagonal of the hat matrix of the rank-r projection.
    """
    X = np.asarray(X, dtype=np.float64)
    n, d = X.shape
    if tau is None or tau < 0:
        tau = default_tau(n, d)
    U, sigma, _ = np.linalg.svd(X, full_matrices=False)
    r = numerical_rank(sigma, tau)
    return np.einsum("ij,ij->i", U[:, :r], U[:, :r])


def exact_leverage_rows(X, rows, tau=None, block=_CHUNK):
    """Exact leverage scores of selected rows of a tall X without forming U (n x d).

    R_X from QR of X accumulated over row blocks (each step a LAPACK QR of [R; block]),
    then the SVD of R_X: l_i = ||x_i V_r diag(1/sigma_r)||^2, equal to ||U_i||^2.
    """
    n, d = X.shape
    if tau is None or tau < 0:
        tau = default_tau(n, d)
    R = np.zeros((0, d))
    for a in range(0, n, block):
        b = min(n, a + block)
        R = np.linalg.qr(np.vstack([R, np.asarray(X[a:b], dtype=np.float64)]), mode="r")
    _, sigma, Vt = np.linalg.svd(R)
    r = numerical_rank(sigma, tau)
    Y = np.asarray(X[rows], dtype=np.float64) @ (Vt[:r].T / sigma[:r])
    return np.einsum("ij,ij->i", Y, Y)


# ---------------------------------------------------------------------------
# Ordering (Algorithm 4 step 4, policy "dec" of Sec. 5.2)
# ---------------------------------------------------------------------------
def order_dec(scores):
    """Policy "dec": indices by decreasing score; ties by increasing index; NaN last.

    -0 and +0 compare equal.  A stable sort of the negated scores.
    """
    sc = np.asarray(scores, dtype=np.float64)
    nan = np.isnan(sc)
    key = np.where(nan, 0.0, -sc)
    key = np.where(key == 0.0, 0.0, key)
    # stable: NaN after every number (-inf included), then decreasing score, ties by index
    return np.lexsort((key, nan)).astype(np.int64)


def sampling_probabilities(scores):
    """Algorithm 4 step 3: P_i = l_i / sum_j l_j."""
    sc = np.asarray(scores, dtype=np.float64)
    return sc / np.sum(sc)


def sample_uniforms(n, seed):
    """Uniform u_t in (0, 1) for the draws t = 0..n-1 of a sampling policy.

    52 bits m = w0 2^20 + (w1 >> 12) from the Philox block (lo t, hi t, 0, 6); u_t = (m + 1/2) 2^-52,
    so 2m + 1 < 2^53 is exact in float64 and u_t is never 0 or 1.
    """
    lo, hi = _split64(np.arange(n, dtype=np.uint64))
    w = philox4x32_10(lo, hi, 0, TAG_SAMPLE, seed)
    m = (w[0] << np.uint64(20)) | (w[1] >> np.uint64(12))
    return (m.astype(np.float64) + 0.5) * 2.0**-52


def _sampling_weights(scores):
    """Weights l_i for the sampling policies: non-finite or negative scores weigh 0 (never drawn)."""
    sc = np.asarray(scores, dtype=np.float64)
    return np.where(np.isfinite(sc) & (sc > 0.0), sc, 0.0)


def order_swor_from_uniforms(scores, u):
    """Policy "dec, swor" (Sec. 5.2; Algorithm 4 step 4): the order of n successive draws without
    replacement, each draw picking one of the points not yet drawn with probability proportional to
    its P_i = l_i / sum l (a weighted random permutation: the largest weights tend to come first).

    The draw order is realised exactly in distribution by Efraimidis and Spirakis's keys: point i
    gets u_i^(1 / P_i) and the points are taken by decreasing key.  Here log(u_i) / l_i stands for
    the key (log is increasing and P_i is l_i times a positive constant, so the order is the same).
    Points of weight 0 are never drawn: they follow all others, in increasing index; NaN scores
    come last.
    """
    sc = np.asarray(scores, dtype=np.float64)
    w = _sampling_weights(sc)
    with np.errstate(divide="ignore"):
        key = np.where(w > 0.0, np.log(u) / np.where(w > 0.0, w, 1.0), -np.inf)
    key = np.where(np.isnan(sc), np.nan, key)
    return order_dec(key)


def order_swor(scores, seed):
    """Policy "dec, swor" with the seeded uniforms of ``sample_uniforms``."""
    return order_swor_from_uniforms(scores, sample_uniforms(np.asarray(scores).shape[0], seed))


def order_swr_from_uniforms(scores, u):
    """Policy "dec, swr" (Sec. 5.2; Algorithm 4 step 4): n successive draws with replacement from P,
    in draw order (points can repeat; points of small P may never appear).  Draw t is the smallest
    index i whose cumulative weight C_i = l_0 + ... + l_i exceeds u_t C_{n-1} (inverse CDF)."""
    C = np.cumsum(_sampling_weights(scores))
    if C.size == 0 or not C[-1] > 0.0:
        raise ValueError("sampling with replacement needs a positive total score")
    return np.searchsorted(C, np.asarray(u) * C[-1], side="right").astype(np.int64)


def order_swr(scores, seed):
    """Policy "dec, swr" with the seeded uniforms of ``sample_uniforms``."""
    return order_swr_from_uniforms(scores, sample_uniforms(np.asarray(scores).shape[0], seed))
