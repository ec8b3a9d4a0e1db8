"""Seeded synthetic inputs shaped like the paper's workloads.

This module only draws data.  It holds none of the method's arithmetic (no sketch,
no factorisation, no scores), so both the CUDA path and the CPU oracle can consume
its output.  Every generator takes an explicit seed and a torch device; the same
(seed, device type) always yields the same matrix.

The paper's datasets (MNIST, SST with GloVe, CMU-MOSI; Sec. 5.1) are not available;
these generators stand in for their shapes and structure:

* ``lognormal_rows``: plain method check, X n x d with N(0,1) entries and each row scaled
  by an independent lognormal(0,1) weight (non-uniform leverage).
* ``image_like``: MNIST-shaped (60000 x 784, Sec. 3.5 and 5.3) uint8/255 data built as a
  rank-50 nonnegative product plus uniform noise, with 68 fixed all-zero columns.
* ``snr_student_t``: rank-200 signal plus Gaussian noise at power SNR 10, rows scaled by
  Student-t(3) draws (heavy-tailed leverage).
* ``gaussian_mixture``: rows from 8 Gaussian clusters (means N(0, 9 I), unit covariance).
* ``outlier_subspace``: N(0, I) rows with 1% of rows replaced by 20 B^T z from a random
  rank-16 subspace.
* ``serving_jobs``: a Poisson arrival trace of jobs of uneven n, d and sketch kind.
* ``text_sequences``: SST-shaped rows (Sec. 5.4): a word sequence of length <= 56, each word a
  300-d vector of a seeded synthetic vocabulary (Zipf word frequencies), left-zero-padded to 56
  steps and flattened, d = 56 x 300 = 16800.
* ``multimodal_sequences``: CMU-MOSI-shaped rows (Sec. 5.5): time steps of early-fused features (a
  300-d word vector, 20 visual and 5 acoustic values, 325 per step), d = 9750 as the paper prints
  it, which with 325 features per step is 30 steps (the paper's "20 x 325 = 9750" does not hold).
"""
from __future__ import annotations

import math

import numpy as np
import torch


def _gen(seed, device):
    g = torch.Generator(device=device)
    g.manual_seed(int(seed))
    return g


def lognormal_rows(n, d, seed, device="cpu", dtype=torch.float64):
    """N(0,1) entries, row i multiplied by w_i = exp(N(0,1))."""
    g = _gen(seed, device)
    X = torch.randn(n, d, generator=g, device=device, dtype=torch.float64)
    w = torch.exp(torch.randn(n, 1, generator=g, device=device, dtype=torch.float64))
    return (X * w).to(dtype)


def image_like(n=60000, d=784, rank=50, n_zero_cols=68, seed=1001, device="cpu"):
    """uint8/255 image-like matrix with a fixed set of all-zero columns.

    W (n x rank) ~ U[0,1), H (rank x (d - n_zero)) ~ Exp(1), P = W H scaled so max(P) = 200,
    v = round(min(P + U[0,56), 255)), X = v / 255 in float32.  The zero columns are the
    first ``n_zero_cols`` entries of a seeded permutation of 0..d-1.
    """
    g = _gen(seed, device)
    d_live = d - n_zero_cols
    W = torch.rand(n, rank, generator=g, device=device, dtype=torch.float64)
    H = -torch.log1p(-torch.rand(rank, d_live, generator=g, device=device, dtype=torch.float64))
    P = W @ H
    P = P * (200.0 / P.max())
    noise = torch.rand(n, d_live, generator=g, device=device, dtype=torch.float64) * 56.0
    v = torch.round(torch.clamp(P + noise, max=255.0))
    perm = torch.randperm(d, generator=g, device=device)
    zero_cols = torch.sort(perm[:n_zero_cols]).values
    live_cols = torch.sort(perm[n_zero_cols:]).values
    X = torch.zeros(n, d, device=device, dtype=torch.float32)
    X[:, live_cols] = (v / 255.0).to(torch.float32)
    return X, zero_cols.cpu().numpy()


def snr_student_t(n, d, rank=200, snr=10.0, nu=3, seed=1003, device="cpu", dtype=torch.float32,
                  chunk=1 << 16):
    """Rank-``rank`` signal A B plus N(0, sigma^2) noise at power SNR ``snr``; rows scaled by t(nu).

    A ~ N(0,1) (n x rank), B ~ N(0, 1/rank) (rank x d), so signal entries have unit variance
    and sigma^2 = 1 / snr.  Row i is multiplied by an independent Student-t(nu) draw.
    Built in float32 in row chunks (matmul precision pinned to full float32).
    """
    g = _gen(seed, device)
    B = torch.randn(rank, d, generator=g, device=device, dtype=torch.float32) / math.sqrt(rank)
    X = torch.empty(n, d, device=device, dtype=dtype)
    sig = math.sqrt(1.0 / snr)
    prev = torch.backends.cuda.matmul.allow_tf32
    torch.backends.cuda.matmul.allow_tf32 = False
    try:
        for a in range(0, n, chunk):
            b = min(n, a + chunk)
            A = torch.randn(b - a, rank, generator=g, device=device, dtype=torch.float32)
            E = torch.randn(b - a, d, generator=g, device=device, dtype=torch.float32) * sig
            z = torch.randn(b - a, 1, generator=g, device=device, dtype=torch.float32)
            chi = torch.zeros(b - a, 1, device=device, dtype=torch.float32)
            for _ in range(nu):
                chi += torch.randn(b - a, 1, generator=g, device=device, dtype=torch.float32) ** 2
            t = z / torch.sqrt(chi / nu)
            X[a:b] = ((A @ B + E) * t).to(dtype)
    finally:
        torch.backends.cuda.matmul.allow_tf32 = prev
    return X


def gaussian_mixture(n, d, clusters=8, seed=10000, device="cpu", dtype=torch.float32):
    """Rows from an equal-weight mixture of ``clusters`` Gaussians, means N(0, 9 I), unit covariance."""
    g = _gen(seed, device)
    means = 3.0 * torch.randn(clusters, d, generator=g, device=device, dtype=torch.float32)
    lab = torch.randint(0, clusters, (n,), generator=g, device=device)
    X = means[lab] + torch.randn(n, d, generator=g, device=device, dtype=torch.float32)
    return X.to(dtype)


def outlier_subspace(n, d, sub_rank=16, frac=0.01, scale=20.0, seed=1005, device="cpu",
                     dtype=torch.bfloat16, chunk=1 << 16):
    """N(0, I) rows; a seeded ``frac`` of the rows replaced by ``scale`` B^T z, z ~ N(0, I_sub).

    B (sub_rank x d) has orthonormal rows (QR of a Gaussian matrix).  Returns (X, outlier rows).
    """
    g = _gen(seed, device)
    G = torch.randn(d, sub_rank, generator=g, device=device, dtype=torch.float64)
    Q, _ = torch.linalg.qr(G.cpu())
    Bt = Q.to(device=device, dtype=torch.float32)  # d x sub_rank, orthonormal columns
    X = torch.empty(n, d, device=device, dtype=dtype)
    for a in range(0, n, chunk):
        b = min(n, a + chunk)
        X[a:b] = torch.randn(b - a, d, generator=g, device=device, dtype=torch.float32).to(dtype)
    n_out = int(round(frac * n))
    rows = torch.sort(torch.randperm(n, generator=g, device=device)[:n_out]).values
    z = torch.randn(n_out, sub_rank, generator=g, device=device, dtype=torch.float32)
    X[rows] = (scale * (z @ Bt.T)).to(dtype)
    return X, rows.cpu().numpy()


SERVING_DIMS = (64, 128, 256, 300, 784)
SERVING_KINDS = ("countsketch", "srht", "gaussian")


def serving_sketch_rows(n, d, kind):
    """Sketch size for a serving job: nextpow2(c d) capped at n/2 (c = 16 CountSketch, else 4)."""
    c = 16 if kind == "countsketch" else 4
    s = 1 << max(0, int(c * d - 1).bit_length())
    s = min(s, n // 2)
    return max(s, d)


def serving_jobs(n_jobs=512, log2_min=12, log2_max=20, rate_per_s=100.0, seed=4004):
    """Poisson arrival trace of leverage jobs: n = round(2^U[lo,hi]), d from SERVING_DIMS.

    Sketch kind: CountSketch, SRHT or Gaussian with probability 1/3 each.  Returns a list of
    dicts (arrival time in seconds, n, d, kind, s, data seed).  Job j's data seed is 10000 + j.
    """
    rng = np.random.default_rng(seed)
    t = np.cumsum(rng.exponential(1.0 / rate_per_s, size=n_jobs))
    jobs = []
    for j in range(n_jobs):
        n = int(round(2.0 ** rng.uniform(log2_min, log2_max)))
        d = int(rng.choice(SERVING_DIMS))
        kind = SERVING_KINDS[int(rng.integers(0, 3))]
        jobs.append({"job": j, "arrival_s": float(t[j]), "n": n, "d": d, "kind": kind,
                     "s": serving_sketch_rows(n, d, kind), "k": 64, "seed": 10000 + j})
    return jobs


def _zipf_words(n_tok, vocab, g, device):
    """Word ids with Zipf(1) frequencies over ``vocab`` words (inverse CDF of seeded uniforms)."""
    w = 1.0 / torch.arange(1, vocab + 1, device=device, dtype=torch.float64)
    cdf = torch.cumsum(w, 0) / w.sum()
    u = torch.rand(n_tok, generator=g, device=device, dtype=torch.float64)
    return torch.clamp(torch.searchsorted(cdf, u), max=vocab - 1)


def text_sequences(n, steps=56, emb=300, vocab=20000, seed=1006, device="cpu", dtype=torch.float32,
                   chunk=1 << 14):
    """SST-shaped sentence matrix: n x (steps * emb), float32.

    The vocabulary holds ``vocab`` seeded embedding vectors (N(0, I/emb) plus a shared offset, as
    word vectors share a common direction).  Sentence lengths are round(16 exp(0.55 z)), z ~ N(0, 1)
    (mean about 19.6 words, a right tail like a sentiment treebank's), clipped to [1, steps], with
    3% of the rows at the maximum (sentences truncated at ``steps`` words).  A sentence of L words
    fills the last L steps (zero padding on the left), so the columns of steps 0..p are nonzero
    only on rows with L >= steps - p; at n = 131072 and emb = 300 those rows outnumber the
    columns 300 (p + 1) at least twice over for every p, so the matrix has full column rank (with
    Poisson lengths the leftmost steps share a few thousand rows and the rank falls short of d).
    """
    g = _gen(seed, device)
    E = torch.randn(vocab, emb, generator=g, device=device, dtype=torch.float32) / math.sqrt(emb)
    E += 0.1 * torch.randn(1, emb, generator=g, device=device, dtype=torch.float32) / math.sqrt(emb)
    X = torch.zeros(n, steps * emb, device=device, dtype=dtype)
    for a in range(0, n, chunk):
        b = min(n, a + chunk)
        m = b - a
        z = torch.randn(m, generator=g, device=device, dtype=torch.float64)
        L = torch.round(16.0 * torch.exp(0.55 * z)).to(torch.int64).clamp(1, steps)
        trunc = torch.rand(m, generator=g, device=device) < 0.03
        L = torch.where(trunc, torch.full_like(L, steps), L)
        ids = _zipf_words(m * steps, vocab, g, device).view(m, steps)
        blk = E[ids]  # m x steps x emb
        pos = torch.arange(steps, device=device).view(1, steps)
        live = (pos >= (steps - L).view(m, 1)).to(blk.dtype).unsqueeze(-1)
        X[a:b] = (blk * live).reshape(m, steps * emb).to(dtype)
    return X


def multimodal_sequences(n, steps=30, emb=300, visual=20, acoustic=5, vocab=20000, seed=1007, device="cpu",
                         dtype=torch.float32, chunk=1 << 14):
    """CMU-MOSI-shaped early-fusion matrix: n x (steps * (emb + visual + acoustic)), float32.

    Every time step concatenates a word vector (the same synthetic vocabulary construction as
    ``text_sequences``, Zipf frequencies), ``visual`` facial-expression-like values (a per-clip
    level plus N(0, 0.5^2) per step) and ``acoustic`` prosody-like values (N(0, 1)).
    """
    g = _gen(seed, device)
    E = torch.randn(vocab, emb, generator=g, device=device, dtype=torch.float32) / math.sqrt(emb)
    feat = emb + visual + acoustic
    X = torch.empty(n, steps * feat, device=device, dtype=dtype)
    for a in range(0, n, chunk):
        b = min(n, a + chunk)
        m = b - a
        ids = _zipf_words(m * steps, vocab, g, device).view(m, steps)
        words = E[ids]  # m x steps x emb
        level = torch.randn(m, 1, visual, generator=g, device=device, dtype=torch.float32)
        vis = level + 0.5 * torch.randn(m, steps, visual, generator=g, device=device, dtype=torch.float32)
        aco = torch.randn(m, steps, acoustic, generator=g, device=device, dtype=torch.float32)
        X[a:b] = torch.cat([words, vis, aco], dim=2).reshape(m, steps * feat).to(dtype)
    return X
