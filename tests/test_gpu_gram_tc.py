"""slso_gram (G = SX^T SX by the tensor-core digit route of the float32 path) against the exact
oracle (each entry of G the float64 rounding of its exact value).

* Integer-valued columns (16 significant bits): every digit product and every partial sum of the
  exact orders is an integer below 2^24, so G must equal the oracle bit for bit.  This is the
  measurement of the tensor core's float32 accumulation on integer-valued bfloat16 operands:
  ragged windows (s not a multiple of 128), ragged tiles (d not a multiple of 64 or 128), and a
  block of constant columns whose leading digit is +-128 in every row, the largest window sums
  the route allows.
* General float64 SX: |G - G_exact| <= 2^-48 sqrt(G_ii G_jj) for Gaussian columns and 2^-46 with
  rows scaled by Student-t(3) like the benchmark's sketch (digits to 2^-56 of each column's
  maximum, every order up to 4 exact, orders 5 and 6 rounded in float32 far below the leading
  one, orders from 7 dropped); a heavy-tailed column loses the bits between its typical entries
  and its maximum.
"""
import numpy as np
import pytest
import torch

from oracle import slso_oracle as O
from paper_1812_07903_gb300 import api

pytestmark = pytest.mark.gpu


def _gpu_gram(A):
    G = api.gram(torch.from_numpy(np.ascontiguousarray(A)).cuda())
    torch.cuda.synchronize()
    return G.cpu().numpy()


@pytest.mark.parametrize("s,d", [(3000, 200), (256, 64), (1, 1), (4133, 130), (9000, 64)])
def test_integer_columns_are_exact(s, d):
    rng = np.random.default_rng(s + d)
    A = rng.integers(-(2**16) + 1, 2**16, size=(s, d)).astype(np.float64)
    if d >= 8:
        # constant +-(2^16 - 1) columns: leading digit 128 in every row, window sums at the bound
        A[:, :4] = (2.0**16 - 1) * np.where(rng.random((s, 4)) < 0.5, -1.0, 1.0)
        A[:, 4] = 2.0**16 - 1
    G = _gpu_gram(A)
    want = O.gram(A)
    np.testing.assert_array_equal(G, want)


def test_repeated_calls_are_bit_identical():
    rng = np.random.default_rng(3)
    A = rng.standard_normal((5000, 300))
    np.testing.assert_array_equal(_gpu_gram(A), _gpu_gram(A))


def _rel_to_diag(G, want):
    dg = np.sqrt(np.abs(np.diag(want)))
    den = np.outer(dg, dg)
    den[den == 0] = 1.0
    return float(np.max(np.abs(G - want) / den))


@pytest.mark.parametrize("heavy", [False, True])
def test_float64_columns_within_the_route_bound(heavy):
    rng = np.random.default_rng(11 + heavy)
    s, d = 6000, 257
    A = rng.standard_normal((s, d))
    if heavy:
        A *= rng.standard_t(3, size=(s, 1))
    A[:, 7] *= 1e-7  # a column far below the others: its own scale
    G = _gpu_gram(A)
    want = O.gram(A)
    err = _rel_to_diag(G, want)
    assert err <= (2.0**-46 if heavy else 2.0**-48), err
    np.testing.assert_array_equal(G, G.T)


def test_zero_column_gives_zero_row_and_column():
    rng = np.random.default_rng(5)
    A = rng.standard_normal((700, 70))
    A[:, 33] = 0.0
    G = _gpu_gram(A)
    assert np.all(G[33] == 0.0) and np.all(G[:, 33] == 0.0)
    assert _rel_to_diag(G, O.gram(A)) <= 2.0**-48
