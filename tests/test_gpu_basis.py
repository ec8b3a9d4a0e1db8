"""GPU parity of slso_approx_u: U = X V_r Sigma_r^-1 from the sketched SVD (Algorithm 2 step 3).

Columns are defined up to the sign of each right singular vector, so each GPU column is compared
with the oracle's after aligning signs; columns at or beyond the rank must be exactly zero.  Row
norms squared must equal slso_leverage's scores with k = 0 (the same sketch and rank).
Tolerances: float64 X 1e-9, float32 / bfloat16 X 1e-4 of the column's largest entry.
"""
import numpy as np
import pytest
import torch

from oracle import slso_oracle as O
from paper_1812_07903_gb300 import api, inputs

pytestmark = pytest.mark.gpu


def _np(X):
    return X.float().double().numpy() if X.dtype == torch.bfloat16 else X.double().numpy()


def _check(U, Uo, r, tol):
    assert np.all(U[:, r:] == 0.0)
    for c in range(r):
        sgn = 1.0 if np.dot(U[:, c], Uo[:, c]) >= 0 else -1.0
        err = np.max(np.abs(sgn * U[:, c] - Uo[:, c])) / np.max(np.abs(Uo[:, c]))
        assert err < tol, (c, err)


@pytest.mark.parametrize("kind,n,d,s,dtype", [
    ("countsketch", 5000, 40, 512, torch.float32),
    ("gaussian", 4096, 64, 256, torch.float64),
    ("srht", 3000, 30, 256, torch.float32),
    ("countsketch", 20000, 128, 2048, torch.bfloat16),
])
def test_approx_u_matches_oracle(kind, n, d, s, dtype):
    X = inputs.lognormal_rows(n, d, seed=n + d, dtype=dtype)
    U, info = api.approx_u(X.cuda(), kind, s, 17)
    Uo, oinfo = O.approx_u(_np(X), kind, s, 17, qr="lapack")
    assert info["rank"] == oinfo["rank"] == d
    _check(U.cpu().numpy().astype(np.float64), Uo, d, 1e-9 if dtype == torch.float64 else 1e-4)
    sc, _ = api.leverage(X.cuda(), kind, s, 0, 17, 0, compute="f64" if dtype == torch.float64 else "f32")
    rows = (U.double() ** 2).sum(dim=1).cpu().numpy()
    np.testing.assert_allclose(rows, sc.double().cpu().numpy(), rtol=1e-9 if dtype == torch.float64 else 2e-4)


def test_approx_u_rank_deficient_image_like():
    X, _ = inputs.image_like(n=6000, seed=1001)
    U, info = api.approx_u(X.cuda(), "countsketch", 2048, 5)
    Uo, oinfo = O.approx_u(X.double().numpy(), "countsketch", 2048, 5, qr="lapack")
    assert info["rank"] == oinfo["rank"] == 716
    _check(U.cpu().numpy().astype(np.float64), Uo, 716, 1e-4)


@pytest.mark.parametrize("dtype", [torch.float32, torch.bfloat16])
def test_approx_u_tensor_core_column_blocks_and_strides(dtype):
    """d = 300: two 256-column blocks of M (the second ragged); X and U with row strides != d."""
    n, d, s = 9001, 300, 1024
    Xw = inputs.lognormal_rows(n, d + 4, seed=31, dtype=dtype)
    X = Xw[:, :d]
    Ubuf = torch.full((n, d + 3), 7.0, dtype=torch.float32, device="cuda")
    U, info = api.approx_u(Xw.cuda()[:, :d], "countsketch", s, 23, out=Ubuf[:, :d])
    Uo, oinfo = O.approx_u(_np(X), "countsketch", s, 23, qr="lapack")
    assert info["rank"] == oinfo["rank"] == d
    _check(U.cpu().numpy().astype(np.float64), Uo, d, 1e-4)
    assert torch.all(Ubuf[:, d:] == 7.0)  # nothing written past column d
