"""GPU edge cases of the method's degenerate shapes, against the oracle (same seeds):

* one row (n = 1), one column (d = 1), a square sketch (s = d), for every sketch kind;
* the JL width at its limit (k = 4096 >> d) on the float32 and float64 paths;
* approx_u and the streamed entry point on a single row;
* a matrix whose rows are all equal (rank 1; every row gets the same score);
* a row of zeros among others (score exactly 0, ordered after the positive scores).
Tolerances as elsewhere: float64 1e-9, float32 1e-4 relative; orders bit-exact.
"""
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
    mask = np.abs(b) > 0
    return float(np.max(np.abs(a[mask] - b[mask]) / np.abs(b[mask]))) if mask.any() else 0.0


@pytest.mark.parametrize("kind,s,nnz", [("countsketch", 1, 0), ("srht", 1, 0), ("gaussian", 1, 0), ("osnap", 1, 1)])
@pytest.mark.parametrize("compute", ["f64", "f32"])
def test_single_row_single_column(kind, s, nnz, compute):
    X = torch.tensor([[3.0]], dtype=torch.float64 if compute == "f64" else torch.float32)
    sc, info = api.leverage(X.cuda(), kind, s, 0, 5, 0, compute=compute, nnz=nnz)
    want, rank = _oracle(X.double().numpy(), kind, s, 0, 5, 0, nnz or None)
    assert info["rank"] == rank == 1
    np.testing.assert_allclose(sc.cpu().numpy(), want, rtol=1e-6)
    if kind != "gaussian":  # S x = +-x: the one point's score is exactly its leverage, 1
        assert abs(float(sc.cpu()[0]) - 1.0) < 1e-6


@pytest.mark.parametrize("kind", ["countsketch", "srht", "gaussian", "osnap"])
def test_square_sketch_s_equals_d(kind):
    n, d = 4096, 32
    X = inputs.lognormal_rows(n, d, seed=41, dtype=torch.float64)
    nnz = 4 if kind == "osnap" else 0
    sc, info = api.leverage(X.cuda(), kind, d, 0, 6, 0, compute="f64", nnz=nnz)
    want, rank = _oracle(X.numpy(), kind, d, 0, 6, 0, nnz or None)
    assert info["rank"] == rank
    assert _rel(sc.cpu().numpy(), want) < 1e-9


@pytest.mark.parametrize("compute,tol", [("f64", 1e-9), ("f32", 1e-4)])
def test_jl_width_at_its_limit(compute, tol):
    n, d, k = 3000, 8, 4096
    X = inputs.lognormal_rows(n, d, seed=42, dtype=torch.float64 if compute == "f64" else torch.float32)
    sc, info = api.leverage(X.cuda(), "countsketch", 64, k, 7, 8, compute=compute)
    want, rank = _oracle(X.double().numpy(), "countsketch", 64, k, 7, 8)
    assert info["rank"] == rank == d
    assert _rel(sc.cpu().numpy(), want) < tol


def test_single_column_with_jl():
    X = inputs.lognormal_rows(5000, 1, seed=43, dtype=torch.float32)
    sc, info = api.leverage(X.cuda(), "gaussian", 16, 64, 9, 10, compute="f32")
    want, rank = _oracle(X.double().numpy(), "gaussian", 16, 64, 9, 10)
    assert info["rank"] == rank == 1
    assert _rel(sc.cpu().numpy(), want) < 1e-4


def test_approx_u_and_streamed_on_one_row():
    X = torch.tensor([[1.0, -2.0, 0.5]], dtype=torch.float32)
    U, info = api.approx_u(X.cuda(), "countsketch", 4, 3)
    assert info["rank"] == 1 and U.shape == (1, 3)
    assert abs(float((U.double() ** 2).sum()) - 1.0) < 1e-6  # ||U_1||^2 = the one point's score
    assert torch.all(U[:, 1:] == 0)
    sc, od, info2 = api.rank_rows_streamed(X, "countsketch", 4, 0, 3, 0)
    assert info2["rank"] == 1 and od.tolist() == [0] and abs(float(sc[0]) - 1.0) < 1e-6


def test_equal_rows_share_the_mass_and_zero_row_scores_zero():
    n, d = 1000, 4
    row = torch.tensor([1.0, 2.0, -1.0, 0.5], dtype=torch.float64)
    X = row.repeat(n, 1)
    sc, info = api.leverage(X.cuda(), "countsketch", 64, 0, 1, 0, compute="f64")
    want, rank = _oracle(X.numpy(), "countsketch", 64, 0, 1, 0)
    assert info["rank"] == rank == 1
    got = sc.cpu().numpy()
    assert _rel(got, want) < 1e-9
    np.testing.assert_allclose(got, np.full(n, got[0]), rtol=1e-12)
    Y = inputs.lognormal_rows(2000, 6, seed=44, dtype=torch.float64)
    Y[777] = 0.0
    sc, info = api.leverage(Y.cuda(), "srht", 256, 0, 2, 0, compute="f64")
    assert float(sc.cpu()[777]) == 0.0
    od = api.order(sc).cpu().numpy()
    np.testing.assert_array_equal(od, O.order_dec(sc.cpu().numpy()))
    assert od[-1] == 777  # the only zero score comes last


def test_qr_two_ctas_per_sm_at_s_6144():
    # s = 6144 with d >= 4 x 152 columns takes the QR kernel with two 128-thread CTAs per SM and 48
    # rows per thread: 48 KB of dynamic shared memory on top of the kernel's static arrays
    n, d, s = 8192, 640, 6144
    X = inputs.lognormal_rows(n, d, seed=45, dtype=torch.float64)
    sc, info = api.leverage(X.cuda(), "countsketch", s, 16, 11, 12, compute="f64")
    want, rank = _oracle(X.numpy(), "countsketch", s, 16, 11, 12)
    assert info["rank"] == rank == d
    assert _rel(sc.cpu().numpy(), want) < 1e-9


def test_block_jacobi_at_48_kb_of_shared_memory():
    # d = 384: the float32 block sweeps of the sketched SVD ask for exactly 48 KB of dynamic shared
    # memory, which with the kernel's static arrays is above a function's starting limit
    s, d = 1024, 384
    X = inputs.lognormal_rows(4096, d, seed=46, dtype=torch.float64)
    SX = api.sketch(X.cuda(), "countsketch", s, 13)
    sigma, V, R, info = api.sketched_svd(SX)
    sv = O.sketched_svd(SX.cpu().numpy(), qr="lapack")
    got = sigma.cpu().numpy()
    assert info["rank"] == sv["rank"] == d
    assert float(np.max(np.abs(got - sv["sigma"]))) < 1e-10 * float(sv["sigma"][0])
