"""GPU parity: every entry point of the C ABI against the FP64 CPU oracle on the same inputs.

Inputs are seeded and synthetic (paper_1812_07903_gb300.inputs), drawn on the CPU and copied to
the device; the oracle never sees anything the CUDA path produced, except where a test checks
a property of the GPU's own output (the ordering of the GPU's scores).

Tolerances (stated per test):
* float64 path: 1e-9 relative (float64 rounding amplified by the conditioning of SX);
* float32 path: 1e-4 relative, the parity bound set for the float32 scores;
* sketches: float32 butterflies / dot products against float64 sums, relative to max |SX|.
"""
import math

import numpy as np
import pytest
import torch

from oracle import slso_oracle as O
from paper_1812_07903_gb300 import api, inputs

pytestmark = pytest.mark.gpu


def _dev(X):
    return X.to("cuda")


def _np(X):
    return X.double().numpy() if X.dtype != torch.bfloat16 else X.float().double().numpy()


def _rel_to_max(a, b):
    return float(np.max(np.abs(a - b)) / max(np.max(np.abs(b)), 1e-300))


def _max_rel(a, b, floor=0.0):
    mask = np.abs(b) > floor
    return float(np.max(np.abs(a[mask] - b[mask]) / np.abs(b[mask]))) if mask.any() else 0.0


# ------------------------------------------------------------------ sketches
CS_CASES = [(1, 1, 1), (33, 7, 5), (5000, 64, 256), (4097, 300, 1024), (20000, 784, 2048)]


@pytest.mark.parametrize("n,d,s", CS_CASES)
@pytest.mark.parametrize("dtype", [torch.float32, torch.bfloat16, torch.float64])
def test_countsketch_matches_oracle(n, d, s, dtype):
    X = inputs.lognormal_rows(n, d, seed=n + d, dtype=dtype)
    SX = api.sketch(_dev(X), "countsketch", s, 77).cpu().numpy()
    want = O.sketch(_np(X), "countsketch", s, 77)
    # compensated float32 (float64 for F64 X) against float64 sums
    assert _rel_to_max(SX, want) < 1e-12


def test_countsketch_ragged_leading_dimension():
    Xf = inputs.lognormal_rows(3000, 70, seed=5, dtype=torch.float32)
    Xd = _dev(Xf)[:, :67]  # ldx = 70, d = 67
    SX = api.sketch(Xd, "countsketch", 512, 9).cpu().numpy()
    want = O.sketch(_np(Xf)[:, :67], "countsketch", 512, 9)
    assert _rel_to_max(SX, want) < 1e-12


# padded heights 1 (shared-memory kernel), 64, 128, 512 (register kernel, R = 1, 2, 8) and 4096-row
# chunks (R = 64) with 1, 2, 5 and 18 chunks; ragged 8-column slabs (d = 5, 9, 17, 100)
SRHT_CASES = [(1, 3, 1), (64, 8, 16), (100, 5, 64), (300, 9, 40), (2049, 17, 100), (5000, 64, 512),
              (20000, 100, 2048), (70000, 24, 1024)]


@pytest.mark.parametrize("n,d,s", SRHT_CASES)
@pytest.mark.parametrize("dtype", [torch.float32, torch.float64, torch.bfloat16])
def test_srht_matches_oracle(n, d, s, dtype):
    X = inputs.lognormal_rows(n, d, seed=3 * n + d, dtype=dtype)
    SX = api.sketch(_dev(X), "srht", s, 31).cpu().numpy()
    want = O.sketch(_np(X), "srht", s, 31)
    tol = 1e-12 if dtype == torch.float64 else 5e-6  # float32 butterflies, log2(n) levels
    assert _rel_to_max(SX, want) < tol


GAUSS_CASES = [(1, 2, 3), (100, 5, 64), (4096, 64, 256), (9000, 130, 200), (33000, 16, 130)]


@pytest.mark.parametrize("n,d,s", GAUSS_CASES)
@pytest.mark.parametrize("dtype", [torch.float32, torch.float64, torch.bfloat16])
def test_gaussian_matches_oracle(n, d, s, dtype):
    """float64 X: SIMT float64 sums.  float32 / bfloat16 X: tensor cores, exact bfloat16 products,
    float32 accumulation over sub-chunks of at most 32 MMA steps (error <= ~32 * 2^-24 of the
    partial sums), sub-chunk totals added in float32 and chunk totals in float64."""
    X = inputs.lognormal_rows(n, d, seed=7 * n + d, dtype=dtype)
    SX = api.sketch(_dev(X), "gaussian", s, 41).cpu().numpy()
    want = O.sketch(_np(X), "gaussian", s, 41)
    tol = 1e-12 if dtype == torch.float64 else 2e-6
    assert _rel_to_max(SX, want) < tol


@pytest.mark.parametrize("dtype", [torch.float32, torch.bfloat16])
def test_gaussian_tensor_core_several_chunks_ragged_tiles(dtype):
    """70001 rows = three chunks of 32768 rows (the last ragged), d = 300 (column tiles of 64 with a
    ragged last tile), s = 333 (row tiles of 128 with a ragged last tile)."""
    n, d, s = 70001, 300, 333
    X = inputs.lognormal_rows(n, d, seed=7 * n + d, dtype=dtype)
    SX = api.sketch(_dev(X), "gaussian", s, 41).cpu().numpy()
    want = O.sketch(_np(X), "gaussian", s, 41)
    assert _rel_to_max(SX, want) < 2e-6


@pytest.mark.parametrize("dtype", [torch.float32, torch.bfloat16])
def test_gaussian_sketch_of_identity_is_the_oracle_g_bit_for_bit(dtype):
    """X = I (4096 x 4096): SX = G / sqrt(s), one exact product per output, so every entry of G the
    GPU generated (four per Philox block, the near-midpoint ones rounded from the float64
    evaluation) must equal the oracle's bfloat16 G exactly; a one-ulp bfloat16 flip is a relative
    change of 2^-8 and would show."""
    n, s, seed = 4096, 1000, 41
    X = torch.eye(n, dtype=dtype)
    SX = api.sketch(_dev(X), "gaussian", s, seed).cpu().numpy()
    G = O.gaussian_block(np.arange(s), np.arange(n), seed)
    got = SX * math.sqrt(s)
    assert np.max(np.abs(got - G) / np.maximum(np.abs(G), 1e-30)) < 1e-12


# ------------------------------------------------------------------ small solve
@pytest.mark.parametrize("s,d", [(1, 1), (7, 3), (256, 64), (1000, 257), (4096, 700), (6000, 300),
                                 (9001, 200), (12000, 160), (14000, 96), (16384, 64)])
def test_sketched_svd_matches_oracle(s, d):
    """QR + SVD of SX; the s values cover every rows-per-thread instance of the left-looking QR
    (256 threads x 2 .. 64 rows, odd s included)."""
    rng = np.random.default_rng(s + d)
    SX = rng.standard_normal((s, d)) * np.exp(rng.standard_normal(d))
    sigma, V, R, info = api.sketched_svd(torch.from_numpy(SX).cuda())
    sv = O.sketched_svd(SX)
    np.testing.assert_allclose(R.cpu().numpy(), sv["R"], rtol=0, atol=1e-10 * np.abs(sv["R"]).max())
    np.testing.assert_allclose(sigma.cpu().numpy(), sv["sigma"], rtol=1e-10, atol=1e-12 * sv["sigma"][0])
    assert info["rank"] == sv["rank"] == d
    # right singular vectors up to sign: |V_gpu^T V_oracle| = I
    G = np.abs(V.cpu().numpy().T @ sv["V"])
    np.testing.assert_allclose(np.diag(G), 1.0, atol=1e-8)


def test_sketched_svd_zero_columns_and_rank():
    rng = np.random.default_rng(3)
    SX = rng.standard_normal((600, 40))
    SX[:, [0, 7, 39]] = 0.0
    sigma, V, R, info = api.sketched_svd(torch.from_numpy(SX).cuda())
    sv = O.sketched_svd(SX)
    assert info["rank"] == sv["rank"] == 37
    np.testing.assert_allclose(R.cpu().numpy(), sv["R"], atol=1e-11 * np.abs(sv["R"]).max())
    assert np.all(sigma.cpu().numpy()[-3:] == 0.0)


# ------------------------------------------------------------------ leverage scores
def test_plain_method_float64_lognormal_rows():
    """Plain method in float64: 4096 x 64 lognormal-scaled rows, Gaussian s=256, k=32 and k=0."""
    X = inputs.lognormal_rows(4096, 64, seed=1001)
    for k in (32, 0):
        sc, info = api.leverage(_dev(X), "gaussian", 256, k, 2001, 3001, compute="f64")
        want, oinfo = O.sketched_leverage(X.numpy(), "gaussian", 256, k, 2001, 3001)
        assert info["rank"] == oinfo["rank"] == 64
        assert info["svd_route"] == 0
        assert _max_rel(sc.cpu().numpy(), want) < 1e-9
        assert abs(info["score_sum"] - want.sum()) < 1e-9 * want.sum()


@pytest.mark.parametrize("kind,s", [("countsketch", 2048), ("srht", 1024), ("gaussian", 1024)])
def test_float32_path_image_like_rank_deficient(kind, s):
    """Image-like data with 68 zero columns: SVD route, rank 716, float32 scores within 1e-4."""
    X, _ = inputs.image_like(n=6000, seed=1001)
    sc, info = api.leverage(_dev(X), kind, s, 64, 2002, 3002, compute="f32")
    want, oinfo = O.sketched_leverage(_np(X), kind, s, 64, 2002, 3002)
    assert info["rank"] == oinfo["rank"] == 716
    assert info["svd_route"] == 1
    assert _max_rel(sc.cpu().numpy().astype(np.float64), want) < 1e-4


@pytest.mark.parametrize("n,d,s,k", [(20000, 256, 4096, 128), (3001, 100, 400, 0), (777, 33, 64, 16)])
def test_float32_path_snr_student_t(n, d, s, k):
    X = inputs.snr_student_t(n, d, rank=min(50, d // 2), seed=1003)
    sc, info = api.leverage(_dev(X), "countsketch", s, k, 2003, 3003, compute="f32")
    want, oinfo = O.sketched_leverage(_np(X), "countsketch", s, k, 2003, 3003)
    assert info["rank"] == oinfo["rank"] == d
    assert _max_rel(sc.cpu().numpy().astype(np.float64), want) < 1e-4


def test_bf16_path_median_error_against_float64():
    X = inputs.snr_student_t(20000, 256, rank=50, seed=1003)
    sc, info = api.leverage(_dev(X), "countsketch", 4096, 128, 2003, 3003, compute="bf16")
    want, _ = O.sketched_leverage(_np(X), "countsketch", 4096, 128, 2003, 3003)
    rel = np.abs(sc.cpu().numpy().astype(np.float64) - want) / want
    assert np.median(rel) < 0.02


def test_all_zero_matrix_gives_rank_zero_and_zero_scores():
    X = torch.zeros(500, 8, dtype=torch.float32)
    sc, info = api.leverage(_dev(X), "countsketch", 64, 4, 1, 2, compute="f32")
    assert info["rank"] == 0 and info["svd_route"] == 1
    assert torch.all(sc == 0)


def test_nonfinite_input_is_reported():
    X = inputs.lognormal_rows(300, 6, seed=1, dtype=torch.float32)
    X[17, 3] = float("nan")
    with pytest.raises(RuntimeError, match="NONFINITE"):
        api.leverage(_dev(X), "countsketch", 64, 0, 1, 2, compute="f32")


# ------------------------------------------------------------------ ordering
@pytest.mark.parametrize("n", [1, 2, 31, 4096, 4097, 100003])
@pytest.mark.parametrize("dtype", [torch.float32, torch.float64])
def test_order_is_stable_sort_of_gpu_scores(n, dtype):
    g = torch.Generator().manual_seed(n)
    sc = torch.rand(n, generator=g, dtype=torch.float64)
    # many ties, signed zeros and NaNs
    sc = torch.floor(sc * 50) / 50
    if n > 10:
        sc[::7] = 0.0
        sc[1::11] = -0.0
        sc[2::13] = float("nan")
    sc = sc.to(dtype)
    o = api.order(sc.cuda()).cpu().numpy()
    want = O.order_dec(sc.double().numpy())
    np.testing.assert_array_equal(o, want)


def test_order_of_leverage_scores_end_to_end():
    X = inputs.lognormal_rows(10000, 32, seed=12, dtype=torch.float32)
    sc, _ = api.leverage(_dev(X), "countsketch", 1024, 0, 4, 5, compute="f32")
    o = api.order(sc).cpu().numpy()
    np.testing.assert_array_equal(o, O.order_dec(sc.cpu().numpy().astype(np.float64)))


def test_host_entry_point_matches_device_entry_points():
    X = inputs.lognormal_rows(5000, 48, seed=13, dtype=torch.float32)
    sc_d, _ = api.leverage(_dev(X), "countsketch", 512, 16, 7, 8, compute="f32")
    o_d = api.order(sc_d)
    sc_h, o_h, info = api.rank_rows_host(X.pin_memory(), "countsketch", 512, 16, 7, 8, compute="f32")
    assert torch.equal(sc_h, sc_d.cpu()) and torch.equal(o_h, o_d.cpu())
    assert info["rank"] == 48


@pytest.mark.parametrize("count", [1, 2, 5])
def test_host_batch_entry_point_matches_item_by_item(count):
    """The pipelined host batch gives, item by item, what the device entry points give (same
    kernels on one stream), including a host row stride larger than d and per-item info."""
    Xs = [inputs.lognormal_rows(3000, 50, seed=100 + i, dtype=torch.float32) for i in range(count)]
    Xh = [X.pin_memory()[:, :47] for X in Xs]  # ldx = 50, d = 47
    scs, ods, infos = api.rank_rows_host_batch(Xh, "countsketch", 512, 16, 7, 8, compute="f32")
    for i in range(count):
        sc_d, info = api.leverage(_dev(Xs[i])[:, :47], "countsketch", 512, 16, 7, 8, compute="f32")
        assert torch.equal(scs[i], sc_d.cpu())
        assert torch.equal(ods[i], api.order(sc_d).cpu())
        assert infos[i]["rank"] == info["rank"] == 47
        assert infos[i]["score_sum"] == info["score_sum"]


# ------------------------------------------------------------------ tensor-core scores
@pytest.mark.parametrize("n,d,k", [(70, 16, 256), (1000, 100, 48), (12345, 320, 128), (4096, 1024, 16)])
def test_tensor_core_float32_scores_match_oracle(n, d, k):
    """3xTF32 tensor-core path: partial tiles, ragged K-blocks, N from 16 to 256."""
    X = inputs.lognormal_rows(n, d, seed=n + k, dtype=torch.float32)
    s = max(2 * d, 256)
    sc, info = api.leverage(_dev(X), "countsketch", s, k, 5, 6, compute="f32")
    want, oinfo = O.sketched_leverage(_np(X), "countsketch", s, k, 5, 6)
    assert info["rank"] == oinfo["rank"] == d
    assert _max_rel(sc.cpu().numpy().astype(np.float64), want) < 1e-4


@pytest.mark.parametrize("form", ["mixed", "tf32x3", "tf32x3_smem"])
@pytest.mark.parametrize("n,d,k", [(1000, 100, 48), (777, 33, 100), (12345, 320, 128), (4096, 1024, 16),
                                   (70000, 200, 128), (6000, 2600, 64)])
def test_float32_score_forms_match_oracle(form, n, d, k):
    """Every operand form of the float32 score product for k <= 128 (X's pieces in tensor memory,
    mixed tf32/bfloat16 or 3xTF32 products, or in shared memory) within the float32 bound: ragged
    row tiles and K-blocks, N from 32 to 128, several work items per CTA, rows longer than 2048
    (one tile per work item, K summed in chunks of 512 with a ragged last chunk), row pitch not a
    multiple of 16 bytes (d = 33: X staged with a padded pitch)."""
    X = inputs.lognormal_rows(n, d, seed=n + k + 1, dtype=torch.float32)
    s = max(2 * d, 256)
    h = api.Handle(0)
    api.set_score_form(form, handle=h)
    sc, info = api.leverage(_dev(X), "countsketch", s, k, 5, 6, compute="f32", handle=h)
    want, oinfo = O.sketched_leverage(_np(X), "countsketch", s, k, 5, 6)
    assert info["rank"] == oinfo["rank"] == d
    assert _max_rel(sc.cpu().numpy().astype(np.float64), want) < 1e-4


def test_score_forms_agree_with_each_other():
    """The mixed form against 3xTF32 on one matrix: both within a few 2^-20 of each other."""
    X = _dev(inputs.snr_student_t(50000, 512, seed=77))
    out = {}
    for form in ("mixed", "tf32x3"):
        h = api.Handle(0)
        api.set_score_form(form, handle=h)
        out[form], _ = api.leverage(X, "countsketch", 4096, 128, 8, 9, compute="f32", handle=h)
    a = out["mixed"].cpu().numpy().astype(np.float64)
    b = out["tf32x3"].cpu().numpy().astype(np.float64)
    assert _max_rel(a, b) < 2e-5


def test_unknown_score_form_is_rejected():
    h = api.Handle(0)
    with pytest.raises(api.L.SlsoError):
        api.L.check(api.L.load().slso_set_score_form(h.ptr, 7))


@pytest.mark.parametrize("n,d,k", [(70, 16, 256), (1000, 100, 48), (12345, 320, 128), (4096, 1024, 16),
                                   (20000, 3072, 256)])
def test_tensor_core_float32_scores_of_bfloat16_x_match_oracle(n, d, k):
    """bfloat16 X, float32-accurate scores: X loaded directly, M as three bfloat16 pieces (24
    significant bits), exact products, float32 accumulation; same 1e-4 bound as the float32 path."""
    X = inputs.lognormal_rows(n, d, seed=n + k, dtype=torch.bfloat16)
    s = max(2 * d, 256)
    sc, info = api.leverage(_dev(X), "countsketch", s, k, 5, 6, compute="f32")
    want, oinfo = O.sketched_leverage(_np(X), "countsketch", s, k, 5, 6, qr="lapack")
    assert info["rank"] == oinfo["rank"] == d
    assert _max_rel(sc.cpu().numpy().astype(np.float64), want) < 1e-4


@pytest.mark.parametrize("xdtype", [torch.float32, torch.bfloat16])
def test_tensor_core_bf16_scores_close_to_oracle(xdtype):
    """BF16 tensor-core paths (float32 X rounded in shared memory, or bfloat16 X loaded directly)."""
    X = inputs.snr_student_t(9000, 512, rank=64, seed=7, dtype=xdtype)
    sc, _ = api.leverage(_dev(X), "countsketch", 2048, 128, 8, 9, compute="bf16")
    want, _ = O.sketched_leverage(_np(X), "countsketch", 2048, 128, 8, 9)
    rel = np.abs(sc.cpu().numpy().astype(np.float64) - want) / want
    assert np.median(rel) < 0.01 and np.max(rel) < 0.2


def test_bf16_correction_pass_rescores_top_rows_in_float32():
    """Precision pattern: BF16 scores, then the top 2% rows rescored in float32 (a7)."""
    n = 20000
    X = inputs.snr_student_t(n, 256, rank=50, seed=1003)
    sc, _ = api.leverage(_dev(X), "countsketch", 4096, 128, 2003, 3003, compute="bf16", correct_frac=0.02)
    want, _ = O.sketched_leverage(_np(X), "countsketch", 4096, 128, 2003, 3003)
    g = sc.cpu().numpy().astype(np.float64)
    top = O.order_dec(g)[: n // 100]
    assert np.max(np.abs(g[top] - want[top]) / want[top]) < 1e-4
    overlap = len(set(top.tolist()) & set(O.order_dec(want)[: n // 100].tolist())) / (n // 100)
    assert overlap >= 0.99
    rest = O.order_dec(g)[n // 10:]
    assert np.median(np.abs(g[rest] - want[rest]) / want[rest]) < 0.01  # untouched rows keep BF16 scores


@pytest.mark.parametrize("xdtype", [torch.float32, torch.bfloat16])
def test_fp8_scores_with_column_scaling_close_to_oracle(xdtype):
    """FP8 e4m3 tensor-core path with per-column X scales folded into M."""
    n = 12000
    X = inputs.snr_student_t(n, 384, rank=64, seed=17, dtype=xdtype)
    X[:, 5] *= 1000.0  # a column on another scale: per-column scaling keeps it representable
    want, _ = O.sketched_leverage(_np(X), "countsketch", 2048, 128, 8, 9)
    sc, _ = api.leverage(_dev(X), "countsketch", 2048, 128, 8, 9, compute="fp8")
    rel = np.abs(sc.cpu().numpy().astype(np.float64) - want) / want
    assert np.median(rel) < 0.03
    sc, _ = api.leverage(_dev(X), "countsketch", 2048, 128, 8, 9, compute="fp8", correct_frac=0.02)
    g = sc.cpu().numpy().astype(np.float64)
    top = O.order_dec(g)[: n // 100]
    assert np.max(np.abs(g[top] - want[top]) / want[top]) < 1e-4
    assert len(set(top.tolist()) & set(O.order_dec(want)[: n // 100].tolist())) >= 0.97 * (n // 100)


def test_large_bf16_matrix_precision_ladder():
    """Outlier-subspace bf16 matrix (reduced n): FP32, BF16 and FP8 score error and top-1% overlap."""
    n, d, s, k = 60000, 3072, 6144, 256
    X, _ = inputs.outlier_subspace(n, d, seed=1005)
    want, oinfo = O.sketched_leverage(_np(X), "countsketch", s, k, 2005, 3005, qr="lapack")
    top_w = set(O.order_dec(want)[: n // 100].tolist())
    res = {}
    for comp in ("f32", "bf16", "fp8"):
        sc, info = api.leverage(_dev(X), "countsketch", s, k, 2005, 3005, compute=comp)
        assert info["rank"] == oinfo["rank"] == d
        g = sc.cpu().numpy().astype(np.float64)
        rel = np.abs(g - want) / want
        res[comp] = (np.median(rel), np.max(rel), len(set(O.order_dec(g)[: n // 100].tolist()) & top_w) / (n // 100))
    print(res)
    assert res["f32"][1] < 1e-4
    assert res["bf16"][0] < 0.02
    assert res["fp8"][0] < 0.05
