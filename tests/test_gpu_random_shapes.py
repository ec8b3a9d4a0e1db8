"""Randomised GPU parity over shapes: 40 seeded draws of (n, d, s, k, sketch kind, X dtype, compute
precision), each compared with the float64 oracle run on the same seeds.

Tolerances as everywhere: float64 path 1e-9 relative, float32 path 1e-4 relative (scores),
the rank exactly, and the order bit-exact to a stable (score, index) sort of the GPU's own
scores.  Shapes cover single rows, d = 1, s = d, ragged tiles (n, d, s not multiples of 32 / 128),
k = 0 and k > d, and OSNAP with every admissible nnz.
"""
import numpy as np
import pytest
import torch

from oracle import slso_oracle as O
from paper_1812_07903_gb300 import api, inputs

pytestmark = pytest.mark.gpu

KINDS = ["countsketch", "srht", "gaussian", "osnap"]


def _draw(i):
    rng = np.random.default_rng(9000 + i)
    kind = KINDS[i % 4]
    d = int(rng.choice([1, 2, 7, 16, 33, 64, 100, 129]))
    n = int(rng.integers(max(d, 1), 6000))
    s = int(rng.integers(d, 4 * d + 64))
    if kind == "srht":
        s = min(s, 1 << int(np.ceil(np.log2(n))))
        if s < d:
            kind = "countsketch"
    nnz = 0
    if kind == "osnap":
        nnz = int(rng.choice([1, 2, 4, 8]))
        s = max(nnz, (s // nnz) * nnz)
        if s < d:
            s = ((d + nnz - 1) // nnz) * nnz
    k = int(rng.choice([0, 0, 8, 64, 300]))
    dtype = [torch.float64, torch.float32, torch.bfloat16][i % 3]
    compute = "f64" if dtype == torch.float64 else "f32"
    return dict(n=n, d=d, s=s, k=k, kind=kind, dtype=dtype, compute=compute, nnz=nnz, seed=i)


def _np(X):
    return X.float().double().numpy() if X.dtype == torch.bfloat16 else X.double().numpy()


@pytest.mark.parametrize("i", range(40))
def test_random_shape_parity(i):
    c = _draw(i)
    X = inputs.lognormal_rows(c["n"], c["d"], seed=100 + i, dtype=c["dtype"])
    Xh = _np(X)
    SX = O.sketch(Xh, c["kind"], c["s"], 7 + i, nnz=c["nnz"] or None)
    Pi = O.jl_matrix(c["d"], c["k"], 11 + i) if c["k"] > 0 else None
    want, sv, _ = O.scores_from_sketch(Xh, SX, None, Pi, qr="lapack")
    sc, info = api.leverage(X.cuda(), c["kind"], c["s"], c["k"], 7 + i, 11 + i, compute=c["compute"], nnz=c["nnz"])
    got = sc.cpu().numpy().astype(np.float64)
    assert info["rank"] == sv["rank"], c
    tol = 1e-9 if c["compute"] == "f64" else 1e-4
    mask = np.abs(want) > 1e-12 * max(np.max(np.abs(want)), 1e-300)
    rel = np.abs(got[mask] - want[mask]) / np.abs(want[mask])
    assert rel.size == 0 or float(np.max(rel)) < tol, (c, float(np.max(rel)))
    assert np.all(np.abs(got[~mask]) <= tol * max(np.max(np.abs(want)), 1e-300)), c
    order = api.order(sc).cpu().numpy()
    np.testing.assert_array_equal(order, O.order_dec(sc.cpu().numpy()))
