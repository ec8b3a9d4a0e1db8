"""The Gram route of the factor R (R = chol(SX^T SX), kept when its probe check passes) against the
oracle and against the Householder route.

* well-conditioned inputs on the float32 path take the Gram route (info gram_route = 1, probe
  residual far below 1e-8) and match the float64 oracle within 1e-4, for ragged d and every
  sketch kind, with and without JL;
* the two routes agree: the Gram route's scores are within 1e-6 of factor='householder' ones;
* a column scaling over 1e6 keeps the route (Cholesky-QR's error depends on the column-equilibrated
  condition number), while the same scaling followed by a random rotation of the columns (kappa
  ~ 1e6 after any column scaling) and a rank-deficient X (a repeated column) fail the check or
  break down, fall back to Householder, and then return bit-for-bit the scores of
  factor='householder';
* compute='f64' never takes the Gram route;
* d > 6144 (R^-1 columns above 48 KB of shared memory) on both routes, and s > 16384 (the
  right-looking Householder kernel as the fallback).
"""
import math

import numpy as np
import pytest
import torch

from oracle import slso_oracle as O
from paper_1812_07903_gb300 import api, inputs

pytestmark = pytest.mark.gpu


def _oracle(Xh, kind, s, k, seed_S, seed_Pi, nnz=None):
    SX = O.sketch(Xh, kind, s, seed_S, nnz=nnz)
    Pi = O.jl_matrix(Xh.shape[1], k, seed_Pi) if k > 0 else None
    sc, sv, _ = O.scores_from_sketch(Xh, SX, None, Pi, qr="lapack")
    return sc, sv["rank"]


def _rel(a, b):
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    mask = np.abs(b) > 0
    return float(np.max(np.abs(a[mask] - b[mask]) / np.abs(b[mask])))


@pytest.mark.parametrize("kind,n,d,s,k,nnz", [
    ("countsketch", 20000, 100, 1024, 0, 0),
    ("countsketch", 9000, 33, 300, 64, 0),
    ("srht", 8192, 129, 1024, 0, 0),
    ("gaussian", 5000, 64, 512, 16, 0),
    ("osnap", 12000, 200, 2048, 0, 4),
    ("countsketch", 3000, 1, 64, 0, 0),
])
def test_gram_route_matches_oracle(kind, n, d, s, k, nnz):
    X = inputs.lognormal_rows(n, d, seed=70 + d, dtype=torch.float32)
    sc, info = api.leverage(X.cuda(), kind, s, k, 11, 12, compute="f32", nnz=nnz)
    assert info["gram_route"] == 1
    assert info["gram_resid"] < 1e-9
    want, rank = _oracle(X.double().numpy(), kind, s, k, 11, 12, nnz or None)
    assert info["rank"] == rank == d
    assert _rel(sc.cpu().numpy(), want) < 1e-4
    hh, hinfo = api.leverage(X.cuda(), kind, s, k, 11, 12, compute="f32", nnz=nnz, factor="householder")
    assert hinfo["gram_route"] == 0 and math.isnan(hinfo["gram_resid"])
    assert _rel(sc.cpu().numpy(), hh.cpu().numpy()) < 1e-6


def test_sketch_taller_than_the_left_looking_qr():
    # s > 16384: the Householder fallback is the right-looking kernel, whose R is copied into the
    # buffer the Gram route writes only when that kernel ran
    n, d, s = 200000, 64, 20000
    X = inputs.lognormal_rows(n, d, seed=82, dtype=torch.float32)
    want, rank = _oracle(X.double().numpy(), "countsketch", s, 16, 13, 14)
    assert rank == d
    for factor, route in (("auto", 1), ("householder", 0)):
        sc, info = api.leverage(X.cuda(), "countsketch", s, 16, 13, 14, compute="f32", factor=factor)
        assert info["gram_route"] == route and info["rank"] == d
        assert _rel(sc.cpu().numpy(), want) < 1e-4


def test_gram_route_bf16_x_and_bf16_compute():
    X = inputs.lognormal_rows(16384, 256, seed=77, dtype=torch.bfloat16)
    sc, info = api.leverage(X.cuda(), "countsketch", 2048, 0, 3, 0, compute="bf16")
    assert info["gram_route"] == 1
    hh, _ = api.leverage(X.cuda(), "countsketch", 2048, 0, 3, 0, compute="bf16", factor="householder")
    assert _rel(sc.cpu().numpy(), hh.cpu().numpy()) < 1e-5


def test_column_scaling_keeps_the_route():
    n, d, s = 20000, 96, 1024
    X = inputs.lognormal_rows(n, d, seed=78, dtype=torch.float64)
    X = (X * torch.logspace(0, -6, d, dtype=torch.float64)[None, :]).float()
    sc, info = api.leverage(X.cuda(), "countsketch", s, 0, 5, 0, compute="f32")
    assert info["gram_route"] == 1 and info["gram_resid"] < 1e-8
    want, rank = _oracle(X.double().numpy(), "countsketch", s, 0, 5, 0)
    assert info["rank"] == rank == d
    assert _rel(sc.cpu().numpy(), want) < 1e-4


def test_ill_conditioned_falls_back_bit_exact():
    n, d, s = 20000, 96, 1024
    X = inputs.lognormal_rows(n, d, seed=78, dtype=torch.float64)
    Q, _ = torch.linalg.qr(torch.from_numpy(np.random.default_rng(3).standard_normal((d, d))))
    X = ((X * torch.logspace(0, -6, d, dtype=torch.float64)[None, :]) @ Q).float()
    sc, info = api.leverage(X.cuda(), "countsketch", s, 0, 5, 0, compute="f32")
    assert info["gram_route"] == 0
    assert not (info["gram_resid"] <= 1e-8)
    hh, hinfo = api.leverage(X.cuda(), "countsketch", s, 0, 5, 0, compute="f32", factor="householder")
    assert torch.equal(sc, hh)
    assert info["rank"] == hinfo["rank"] and info["svd_route"] == hinfo["svd_route"]


def test_rank_deficient_falls_back_bit_exact():
    n, d, s = 10000, 64, 512
    X = inputs.lognormal_rows(n, d, seed=79, dtype=torch.float32)
    X[:, 40] = X[:, 3]
    sc, info = api.leverage(X.cuda(), "countsketch", s, 16, 6, 7, compute="f32")
    assert info["gram_route"] == 0
    hh, hinfo = api.leverage(X.cuda(), "countsketch", s, 16, 6, 7, compute="f32", factor="householder")
    assert torch.equal(sc, hh)
    assert info["rank"] == hinfo["rank"] == d - 1 and info["svd_route"] == 1
    # R of a rank-deficient SX is not unique (rows past the repeated column follow rounding), so
    # R^+ Pi depends on the QR; the k = 0 scores do not and are compared with the oracle
    sc0, info0 = api.leverage(X.cuda(), "countsketch", s, 0, 6, 0, compute="f32")
    assert info0["gram_route"] == 0
    want, rank = _oracle(X.double().numpy(), "countsketch", s, 0, 6, 0)
    assert rank == d - 1 == info0["rank"]
    assert _rel(sc0.cpu().numpy(), want) < 1e-4


def test_f64_compute_never_takes_the_gram_route():
    X = inputs.lognormal_rows(4000, 50, seed=80, dtype=torch.float64)
    _, info = api.leverage(X.cuda(), "countsketch", 256, 0, 1, 0, compute="f64")
    assert info["gram_route"] == 0 and math.isnan(info["gram_resid"])


def test_wide_d_above_shared_memory_default():
    n, d, s = 60000, 6200, 6400  # n >> s: CountSketch leaves no bucket empty, SX has full rank
    X = inputs.lognormal_rows(n, d, seed=81, dtype=torch.float32)
    rows = np.random.default_rng(5).choice(n, 256, replace=False)
    Xh = X.double().numpy()
    sv = O.sketched_svd(O.sketch(Xh, "countsketch", s, 9), None, qr="lapack")
    assert sv["rank"] == d
    want = O.row_scores(Xh[rows], O.m_matrix(sv["sigma"], sv["V"], sv["U_R"], sv["rank"], None))
    for compute, Xc, tol in (("f32", X, 1e-4), ("f64", X.double(), 1e-9)):
        sc, info = api.leverage(Xc.cuda(), "countsketch", s, 0, 9, 0, compute=compute)
        assert info["gram_route"] == (1 if compute == "f32" else 0)
        assert info["rank"] == d
        assert _rel(sc.cpu().numpy()[rows], want) < tol
