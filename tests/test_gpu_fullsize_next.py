"""Full-size GPU parity of the paths the benchmark times beside the main step, on its 1,000,000 x
1024 float32 matrix (rank-200 signal + SNR 10 noise, Student-t(3) rows), CountSketch / OSNAP
s = 16384:

* slso_approx_u: sampled rows of U against X_rows V_r Sigma_r^-1 from the oracle's SVD of the
  GPU's own sketch (stage-wise), columns aligned in sign, within 1e-4 of each column's largest
  sampled entry; every row's ||U_i||^2 equal to slso_leverage's k = 0 score within 2e-4;
* OSNAP with 4 nonzeros per column: sampled rows of SX summed exactly in float64 from the rows
  hashing to them, and sampled scores stage-wise within 1e-4;
* slso_rank_rows_streamed in 4 blocks of 262144 rows from pinned host memory: scores within 1e-5
  of the in-core call with the same seeds, and the order bit-exact to a stable sort of its scores.
"""
import numpy as np
import pytest
import torch

from oracle import slso_oracle as O
from paper_1812_07903_gb300 import api, inputs

pytestmark = pytest.mark.gpu

N, D, S, K = 1_000_000, 1024, 16384, 128
XSEED, SEED_S, SEED_PI = 1003, 2003, 3003


@pytest.fixture(scope="module")
def X():
    return inputs.snr_student_t(N, D, seed=XSEED, device="cuda")


def _max_rel(a, b):
    mask = np.abs(b) > 0
    return float(np.max(np.abs(a[mask] - b[mask]) / np.abs(b[mask])))


def test_approx_u_full_size_sampled_rows(X):
    U, info = api.approx_u(X, "countsketch", S, SEED_S)
    SX = api.sketch(X, "countsketch", S, SEED_S).cpu().numpy()
    sv = O.sketched_svd(SX, None, qr="lapack")
    r = sv["rank"]
    assert info["rank"] == r == D
    rng = np.random.default_rng(7)
    rows = np.unique(rng.choice(N, 4096, replace=False))
    Xr = X[torch.from_numpy(rows).cuda()].cpu().numpy().astype(np.float64)
    want = Xr @ (sv["V"][:, :r] / sv["sigma"][:r])
    got = U[torch.from_numpy(rows).cuda()].cpu().numpy().astype(np.float64)
    for c in range(r):
        sgn = 1.0 if np.dot(got[:, c], want[:, c]) >= 0 else -1.0
        err = np.max(np.abs(sgn * got[:, c] - want[:, c])) / np.max(np.abs(want[:, c]))
        assert err < 1e-4, (c, err)
    sc, _ = api.leverage(X, "countsketch", S, 0, SEED_S, 0, compute="f32")
    rn = (U.double() ** 2).sum(dim=1)
    rel = ((rn - sc.double()).abs() / sc.double().clamp_min(1e-300)).max().item()
    assert rel < 2e-4


def test_osnap_full_size_sketch_and_scores(X):
    z = 4
    SX = api.sketch(X, "osnap", S, SEED_S).cpu().numpy()
    bucket, sign = O.osnap_hash(N, S, z, SEED_S)
    Xh = X.cpu().numpy()
    rng = np.random.default_rng(3)
    for b in rng.choice(S, 16, replace=False):
        blk = b // (S // z)
        rows = np.nonzero(bucket[blk] == b)[0]
        want = (sign[blk, rows][:, None] * Xh[rows].astype(np.float64)).sum(axis=0) / np.sqrt(z)
        assert np.max(np.abs(SX[b] - want)) <= 1e-12 * max(np.max(np.abs(want)), 1e-300)
    sc, info = api.leverage(X, "osnap", S, K, SEED_S, SEED_PI, compute="f32", nnz=z)
    sc = sc.cpu().numpy()
    rows = np.unique(rng.choice(N, 8192, replace=False))
    sv = O.sketched_svd(SX, None, qr="lapack")
    M = O.m_matrix(sv["sigma"], sv["V"], sv["U_R"], sv["rank"], O.jl_matrix(D, K, SEED_PI))
    want = O.row_scores(Xh[rows].astype(np.float64), M)
    assert info["rank"] == sv["rank"] == D
    assert _max_rel(sc[rows], want) < 1e-4


def test_streamed_full_size_equals_in_core(X):
    Xh = X.cpu().pin_memory()
    sc, od, info = api.rank_rows_streamed(Xh, "countsketch", S, K, SEED_S, SEED_PI, compute="f32",
                                          block_rows=262144)
    inc, inc_info = api.leverage(X, "countsketch", S, K, SEED_S, SEED_PI, compute="f32")
    assert info["rank"] == inc_info["rank"] == D
    assert _max_rel(sc.numpy(), inc.cpu().numpy()) < 1e-5
    np.testing.assert_array_equal(od.numpy(), O.order_dec(sc.numpy()))
