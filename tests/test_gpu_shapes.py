"""The paper's text- and multimodal-shaped feature matrices (Sec. 5.4 SST: 56 words x 300-d word
vectors, d = 16800; Sec. 5.5 CMU-MOSI: 325 early-fused features per step, d = 9750).

* The same generators at reduced widths (12-d and 24-d word vectors) against the whole oracle:
  float32 scores within 1e-4, the rank, R from the Gram route.
* Full size (131072 rows, k = 128 as the benchmark runs them): the Gram route stands (rank d,
  probe residual below 1e-8), sampled sketch rows are the exact bucket sums, and every sampled
  row's score equals ||x_i R^-1 Pi||^2 with R the Cholesky factor (LAPACK, on the host) of
  G = SX^T SX as slso_gram forms it (itself checked against the exact Gram oracle elsewhere) and
  Pi the oracle's JL matrix: the float-float factorisation, its inverse, M and the scores at
  d = 16800 and 9750, stage-wise.
"""
import numpy as np
import pytest
import scipy.linalg as sla
import torch

from oracle import slso_oracle as O
from paper_1812_07903_gb300 import api, inputs

pytestmark = pytest.mark.gpu


def _max_rel(a, b):
    mask = np.abs(b) > 0
    return float(np.max(np.abs(a[mask] - b[mask]) / np.abs(b[mask])))


@pytest.mark.parametrize("name", ["text", "multimodal"])
def test_reduced_width_matches_oracle(name):
    if name == "text":
        X = inputs.text_sequences(20000, steps=56, emb=12, vocab=5000, seed=61)
        s = 2048
    else:
        X = inputs.multimodal_sequences(20000, steps=6, emb=24, vocab=5000, seed=62)
        s = 1024
    n, d = X.shape
    want, oinfo = O.sketched_leverage(X.double().numpy(), "countsketch", s, 64, 71, 72, qr="lapack")
    sc, info = api.leverage(X.cuda(), "countsketch", s, 64, 71, 72, compute="f32")
    assert info["rank"] == oinfo["rank"] == d
    assert info["gram_route"] == 1 and info["gram_resid"] < 1e-8
    assert _max_rel(sc.cpu().numpy().astype(np.float64), want) < 1e-4


@pytest.mark.parametrize("name,n,d,s", [("text", 131072, 16800, 32768), ("multimodal", 131072, 9750, 16384)])
def test_full_size_stagewise(name, n, d, s):
    gen = inputs.text_sequences if name == "text" else inputs.multimodal_sequences
    X = gen(n, seed=1006 if name == "text" else 1007, device="cuda")
    assert X.shape == (n, d)
    seed_S, seed_Pi, k = (2006, 3006, 128) if name == "text" else (2007, 3007, 128)
    sc, info = api.leverage(X, "countsketch", s, k, seed_S, seed_Pi, compute="f32")
    assert info["rank"] == d and info["gram_route"] == 1 and info["gram_resid"] < 1e-8
    SX = api.sketch(X, "countsketch", s, seed_S)
    G = api.gram(SX).cpu().numpy()
    SXh = SX.cpu().numpy()
    del SX
    rng = np.random.default_rng(3)
    # sampled buckets of the sketch: exact sums of their rows
    bucket, sign = O.countsketch_hash(n, s, seed_S)
    for b in rng.choice(s, 8, replace=False):
        rows = np.nonzero(bucket == b)[0]
        Xr = X[torch.from_numpy(rows).cuda()].cpu().numpy().astype(np.float64)
        want = (sign[rows][:, None] * Xr).sum(axis=0)
        assert np.max(np.abs(SXh[b] - want)) <= 1e-12 * max(np.max(np.abs(want)), 1e-300)
    # sampled scores: ||x_i R^-1 Pi||^2 with R = chol(G) by LAPACK on the host (R^T y = x_i^T)
    rows = np.sort(rng.choice(n, 200, replace=False))
    Xh_rows = X[torch.from_numpy(rows).cuda()].cpu().numpy().astype(np.float64)
    R = sla.cholesky(G, lower=False)
    Y = sla.solve_triangular(R, Xh_rows.T, trans="T", lower=False)  # columns: (x_i R^-1)^T
    P = Y.T @ O.jl_matrix(d, k, seed_Pi)
    want = np.einsum("ij,ij->i", P, P)
    got = sc.cpu().numpy()[rows].astype(np.float64)
    assert _max_rel(got, want) < 1e-4
