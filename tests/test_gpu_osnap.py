"""GPU parity of the OSNAP sketch (Sec. 3.1.2: CountSketch with z nonzeros per column of S, in
block form) against the float64 oracle, through the C ABI.

* slso_sketch (z = 4): every entry of SX within 1e-12 of max |SX| (compensated float32 / float64
  gathers against float64 sums), ragged n, d and leading dimension;
* slso_leverage with slso_params.nnz = z for z in {1, 2, 4, 8}: float64 scores within 1e-9 and
  float32 scores within 1e-4 of the oracle's scores from its own OSNAP sketch;
* z = 1 is not CountSketch (its own Philox stream), and invalid z is refused on the host.
"""
import numpy as np
import pytest
import torch

from oracle import slso_oracle as O
from paper_1812_07903_gb300 import api, inputs
from paper_1812_07903_gb300._lib import SlsoError

pytestmark = pytest.mark.gpu


def _np(X):
    return X.double().numpy() if X.dtype != torch.bfloat16 else X.float().double().numpy()


def _rel_to_max(a, b):
    return float(np.max(np.abs(a - b)) / max(np.max(np.abs(b)), 1e-300))


def _max_rel(a, b):
    mask = np.abs(b) > 0
    return float(np.max(np.abs(a[mask] - b[mask]) / np.abs(b[mask])))


@pytest.mark.parametrize("n,d,s", [(1, 1, 4), (33, 7, 8), (5000, 64, 256), (4097, 300, 1024), (20000, 784, 2048)])
@pytest.mark.parametrize("dtype", [torch.float32, torch.bfloat16, torch.float64])
def test_osnap_sketch_matches_oracle(n, d, s, dtype):
    X = inputs.lognormal_rows(n, d, seed=n + 3 * d, dtype=dtype)
    SX = api.sketch(X.cuda(), "osnap", s, 91).cpu().numpy()
    want = O.sketch(_np(X), "osnap", s, 91, nnz=O.OSNAP_DEFAULT_NNZ)
    assert _rel_to_max(SX, want) < 1e-12


def test_osnap_ragged_leading_dimension():
    Xf = inputs.lognormal_rows(3001, 70, seed=6, dtype=torch.float32)
    Xd = Xf.cuda()[:, :67]
    SX = api.sketch(Xd, "osnap", 512, 12).cpu().numpy()
    want = O.sketch(_np(Xf)[:, :67], "osnap", 512, 12, nnz=4)
    assert _rel_to_max(SX, want) < 1e-12


@pytest.mark.parametrize("z", [1, 2, 4, 8])
@pytest.mark.parametrize("n,d,s,k", [(12345, 200, 1024, 0), (20000, 256, 4096, 128)])
def test_osnap_leverage_matches_oracle(z, n, d, s, k):
    X = inputs.snr_student_t(n, d, seed=n + z)
    Xh = X.numpy().astype(np.float64)
    SX = O.sketch(Xh, "osnap", s, 17, nnz=z)
    Pi = O.jl_matrix(d, k, 27) if k > 0 else None
    want, sv, _ = O.scores_from_sketch(Xh, SX, None, Pi, qr="lapack")
    Xd = X.cuda()
    sc64, info = api.leverage(Xd.double(), "osnap", s, k, 17, 27, compute="f64", nnz=z)
    assert info["rank"] == sv["rank"]
    assert _max_rel(sc64.cpu().numpy(), want) < 1e-9
    sc32, _ = api.leverage(Xd, "osnap", s, k, 17, 27, compute="f32", nnz=z)
    assert _max_rel(sc32.cpu().numpy(), want) < 1e-4


def test_osnap_one_nonzero_is_not_countsketch():
    X = inputs.lognormal_rows(2000, 16, seed=4, dtype=torch.float64)
    Xd = X.cuda()
    sc_o, _ = api.leverage(Xd, "osnap", 256, 0, 5, 0, compute="f64", nnz=1)
    sc_c, _ = api.leverage(Xd, "countsketch", 256, 0, 5, 0, compute="f64")
    assert not torch.equal(sc_o, sc_c)
    want, _, _ = O.scores_from_sketch(X.numpy(), O.sketch(X.numpy(), "osnap", 256, 5, nnz=1), None, None, qr="lapack")
    assert _max_rel(sc_o.cpu().numpy(), want) < 1e-9


@pytest.mark.parametrize("z,s", [(3, 256), (65, 4160), (-1, 256)])
def test_osnap_invalid_nnz_refused(z, s):
    X = torch.ones(100, 4, dtype=torch.float32, device="cuda")
    with pytest.raises(SlsoError):
        api.leverage(X, "osnap", s, 0, 1, 0, nnz=z)
