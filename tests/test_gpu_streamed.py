"""GPU parity of the out-of-core entry point slso_rank_rows_streamed: X stays in host memory and
is streamed through the device in blocks of rows, twice (sketch, then scores).

* every sketch kind, float32 / bfloat16 / float64 X, several blocks with a ragged last block:
  scores within 1e-4 (float32 path) or 1e-9 (float64 path) of the oracle run with the same
  seeds on the whole X, and within 1e-5 / 1e-12 of the in-core call on the device;
* the order is bit-exact to a stable (score, index) sort of the streamed scores;
* one block, two blocks (both still resident for the second pass), strided host rows;
* rank-deficient input keeps the oracle's rank; invalid arguments are refused on the host.
"""
import numpy as np
import pytest
import torch

from oracle import slso_oracle as O
from paper_1812_07903_gb300 import api, inputs
from paper_1812_07903_gb300._lib import SlsoError

pytestmark = pytest.mark.gpu

BLOCK = 65536


def _np(X):
    return X.double().numpy() if X.dtype != torch.bfloat16 else X.float().double().numpy()


def _max_rel(a, b):
    mask = np.abs(b) > 0
    return float(np.max(np.abs(a[mask] - b[mask]) / np.abs(b[mask])))


def _oracle(Xh, kind, s, k, seed_S, seed_Pi, nnz=None):
    SX = O.sketch(Xh, kind, s, seed_S, nnz=nnz)
    Pi = O.jl_matrix(Xh.shape[1], k, seed_Pi) if k > 0 else None
    sc, sv, _ = O.scores_from_sketch(Xh, SX, None, Pi, qr="lapack")
    return sc, sv["rank"]


@pytest.mark.parametrize("kind,n,d,s,k,dtype", [
    ("countsketch", 200001, 64, 1024, 32, torch.float32),
    ("osnap", 200001, 64, 1024, 32, torch.float32),
    ("srht", 140000, 64, 1024, 0, torch.float32),
    ("gaussian", 70000, 32, 128, 16, torch.float32),
    ("gaussian", 70000, 32, 128, 16, torch.bfloat16),
    ("countsketch", 200001, 48, 512, 0, torch.bfloat16),
])
def test_streamed_float32_path_matches_oracle_and_in_core(kind, n, d, s, k, dtype):
    X = inputs.snr_student_t(n, d, seed=n + d).to(dtype)
    Xh = X.pin_memory()
    sc, od, info = api.rank_rows_streamed(Xh, kind, s, k, 11, 12, compute="f32", block_rows=BLOCK)
    want, rank = _oracle(_np(X), kind, s, k, 11, 12)
    assert info["rank"] == rank
    assert _max_rel(sc.numpy(), want) < 1e-4
    inc, _ = api.leverage(X.cuda(), kind, s, k, 11, 12, compute="f32")
    assert _max_rel(sc.numpy(), inc.cpu().numpy()) < 1e-5
    np.testing.assert_array_equal(od.numpy(), O.order_dec(sc.numpy()))
    assert abs(info["score_sum"] - float(np.sum(sc.numpy(), dtype=np.float64))) <= 1e-5 * abs(info["score_sum"])


@pytest.mark.parametrize("kind,s", [("countsketch", 512), ("srht", 512), ("gaussian", 128), ("osnap", 512)])
def test_streamed_float64_path_matches_oracle_and_in_core(kind, s):
    n, d = 140000 if kind != "gaussian" else 70000, 24
    X = inputs.lognormal_rows(n, d, seed=7, dtype=torch.float64)
    sc, od, info = api.rank_rows_streamed(X.pin_memory(), kind, s, 0, 5, 0, compute="f64", block_rows=BLOCK)
    want, rank = _oracle(X.numpy(), kind, s, 0, 5, 0)
    assert info["rank"] == rank
    assert _max_rel(sc.numpy(), want) < 1e-9
    inc, _ = api.leverage(X.cuda(), kind, s, 0, 5, 0, compute="f64")
    assert _max_rel(sc.numpy(), inc.cpu().numpy()) < 1e-12
    np.testing.assert_array_equal(od.numpy(), O.order_dec(sc.numpy()))


@pytest.mark.parametrize("n", [1000, 65536, 100000, 131072, 131073])
def test_streamed_block_counts(n):
    """One block, two blocks (both resident for the second pass), two full blocks, three blocks."""
    X = inputs.snr_student_t(n, 40, seed=n)
    sc, od, info = api.rank_rows_streamed(X.pin_memory(), "countsketch", 256, 16, 2, 3, block_rows=BLOCK)
    want, rank = _oracle(X.numpy().astype(np.float64), "countsketch", 256, 16, 2, 3)
    assert info["rank"] == rank
    assert _max_rel(sc.numpy(), want) < 1e-4
    np.testing.assert_array_equal(od.numpy(), O.order_dec(sc.numpy()))


def test_streamed_strided_host_rows():
    Xf = inputs.snr_student_t(150000, 70, seed=3)
    Xs = Xf[:, :67]  # row stride 70, d = 67
    sc, od, _ = api.rank_rows_streamed(Xs, "countsketch", 512, 0, 4, 0, block_rows=BLOCK)
    want, _ = _oracle(Xs.numpy().astype(np.float64), "countsketch", 512, 0, 4, 0)
    assert _max_rel(sc.numpy(), want) < 1e-4


def test_streamed_rank_deficient_keeps_oracle_rank():
    X, zero_cols = inputs.image_like(n=140000, seed=1002)
    sc, od, info = api.rank_rows_streamed(X, "countsketch", 4096, 64, 8, 9, block_rows=BLOCK)
    want, rank = _oracle(X.double().numpy(), "countsketch", 4096, 64, 8, 9)
    assert info["rank"] == rank == 784 - len(zero_cols)
    assert _max_rel(sc.numpy(), want) < 1e-4


def test_streamed_refuses_correction_and_negative_block():
    X = torch.ones(1000, 4)
    with pytest.raises(SlsoError):
        api.rank_rows_streamed(X, "countsketch", 64, 0, 1, 0, block_rows=-1)
    p = api.make_params("countsketch", 64, 0, 1, 0, -1.0, "bf16", 0.01)
    sc = torch.empty(1000)
    od = torch.empty(1000, dtype=torch.int64)
    from paper_1812_07903_gb300 import _lib as L
    import ctypes
    st = L.load().slso_rank_rows_streamed(api.default_handle().ptr, X.data_ptr(), 1000, 4, 4, L.F32,
                                          ctypes.byref(p), 0, sc.data_ptr(), od.data_ptr(), None, None)
    assert L.STATUS_NAMES.get(st) == "INVALID_ARG"
