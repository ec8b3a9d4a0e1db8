"""GPU parity of the sampling policies (Algorithm 4 step 4: "dec", "dec, swr", "dec, swor").

Both sides order the GPU's own float32 scores with the same seeded uniforms.  swor: the GPU's
order must be a permutation whose oracle keys log(u_i)/l_i are non-increasing (ties by index);
it equals the oracle's order unless two keys agree to float64 rounding (CUDA's and numpy's log
may differ in the last bit).  swr: every draw equals the oracle's unless its target u_t * total
lies within float64 rounding of a cumulative boundary (the prefix sums are added in another order).
"""
import numpy as np
import pytest
import torch

from oracle import slso_oracle as O
from paper_1812_07903_gb300 import api, inputs

pytestmark = pytest.mark.gpu


def _scores(n, d=48, seed=11):
    X = inputs.lognormal_rows(n, d, seed=seed, dtype=torch.float32)
    sc, _ = api.leverage(X.cuda(), "countsketch", 512, 16, 3, 4, compute="f32")
    return sc


def _keys(scores, seed):
    u = O.sample_uniforms(scores.size, seed)
    w = np.where(np.isfinite(scores) & (scores > 0), scores, 0.0)
    with np.errstate(divide="ignore"):
        return np.where(w > 0, np.log(u) / np.where(w > 0, w, 1.0), -np.inf)


@pytest.mark.parametrize("n", [1, 2, 33, 4097, 100003])
def test_swor_matches_oracle(n):
    sc = _scores(n)
    got = api.sample_order(sc, "swor", seed=5).cpu().numpy()
    s64 = sc.cpu().numpy().astype(np.float64)
    want = O.order_swor(s64, 5)
    assert np.array_equal(np.sort(got), np.arange(n))
    if not np.array_equal(got, want):
        k = _keys(s64, 5)[got]
        fin = np.isfinite(k)
        d = np.diff(k[fin])
        assert np.all(d <= 1e-13 * np.abs(k[fin][1:]))
        assert np.mean(got == want) > 0.9999


@pytest.mark.parametrize("n", [1, 2, 33, 4097, 100003])
def test_swr_matches_oracle(n):
    sc = _scores(n)
    got = api.sample_order(sc, "swr", seed=9).cpu().numpy()
    s64 = sc.cpu().numpy().astype(np.float64)
    want = O.order_swr(s64, 9)
    bad = np.nonzero(got != want)[0]
    if bad.size:
        C = np.cumsum(np.where(s64 > 0, s64, 0.0))
        tgt = O.sample_uniforms(n, 9)[bad] * C[-1]
        edge = C[np.minimum(got[bad], want[bad])]
        assert np.all(np.abs(tgt - edge) <= 1e-12 * C[-1])
    assert got.min() >= 0 and got.max() < n


def test_dec_policy_is_slso_order_and_seeds_matter():
    sc = _scores(5000)
    np.testing.assert_array_equal(api.sample_order(sc, "dec").cpu().numpy(), api.order(sc).cpu().numpy())
    a = api.sample_order(sc, "swor", seed=1).cpu().numpy()
    np.testing.assert_array_equal(a, api.sample_order(sc, "swor", seed=1).cpu().numpy())
    assert not np.array_equal(a, api.sample_order(sc, "swor", seed=2).cpu().numpy())


def test_zero_and_nan_weights():
    sc = torch.tensor([0.0, 2.0, float("nan"), 0.0, 1.0, 3.0], device="cuda", dtype=torch.float64)
    for seed in range(20):
        o = api.sample_order(sc, "swor", seed=seed).cpu().numpy()
        assert sorted(o[:3].tolist()) == [1, 4, 5] and o[3:].tolist() == [0, 3, 2]
        np.testing.assert_array_equal(o, O.order_swor(sc.cpu().numpy(), seed))
        r = api.sample_order(sc, "swr", seed=seed).cpu().numpy()
        assert set(r.tolist()) <= {1, 4, 5}
    z = torch.zeros(7, device="cuda", dtype=torch.float32)
    assert api.sample_order(z, "swr", seed=3).cpu().numpy().tolist() == [-1] * 7
    assert api.sample_order(z, "swor", seed=3).cpu().numpy().tolist() == list(range(7))
