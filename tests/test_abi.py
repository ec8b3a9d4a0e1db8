"""The C-ABI library builds, loads and exports every entry point include/slso.h declares.

No compute call is made here (no GPU on this host); argument checks that fail before any
CUDA work are exercised where they cannot touch a device.
"""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    src = open(os.path.join(ROOT, "include", "slso.h")).read()
    return sorted(set(re.findall(r"^\s*(?:const char\*|slso_status)\s+(slso_\w+)\s*\(", src, re.M)))


@pytest.fixture(scope="module")
def lib():
    from paper_1812_07903_gb300 import build, _lib
    build.build()
    return _lib.load()


def test_header_declares_the_boundary():
    names = _declared()
    for n in ("slso_sketch", "slso_sketched_svd", "slso_leverage", "slso_order"):
        assert n in names


def test_library_exports_every_declared_symbol(lib):
    from paper_1812_07903_gb300 import _lib
    for name in _declared():
        assert hasattr(lib, name), name
    assert set(_declared()) <= set(_lib.EXPORTS)


def test_version_and_workspace_sizing_without_gpu(lib):
    from paper_1812_07903_gb300 import _lib as L
    assert b"sm_103a" in lib.slso_version()
    p = L.Params(kind=L.COUNTSKETCH, compute=L.F32, s=16384, k=128, seed_S=1, seed_Pi=2, tau=-1.0, correct_frac=0.0)
    nbytes = ctypes.c_size_t(0)
    assert lib.slso_workspace_size(ctypes.byref(p), 1_000_000, 1024, ctypes.byref(nbytes)) == L.SLSO_OK
    # dominated by SX (s x d float64), the QR copy of it and the Gram route's float32 split of it
    assert 3 * 16384 * 1024 * 8 <= nbytes.value < 4 * 16384 * 1024 * 8 + 200 * 2**20


def test_factor_choice_sizes_the_gram_route_and_rejects_unknown_values(lib):
    from paper_1812_07903_gb300 import _lib as L
    def size(compute, factor):
        p = L.Params(kind=L.COUNTSKETCH, compute=compute, s=4096, k=64, seed_S=1, seed_Pi=2, tau=-1.0,
                     correct_frac=0.0, nnz=0, factor=factor)
        nbytes = ctypes.c_size_t(0)
        st = lib.slso_workspace_size(ctypes.byref(p), 100_000, 256, ctypes.byref(nbytes))
        return st, nbytes.value
    st_auto, auto = size(L.F32, 0)
    st_hh, hh = size(L.F32, 1)
    assert st_auto == st_hh == L.SLSO_OK
    # the Gram route's buffers: the split SX (2 x s x d float32) at least
    assert auto - hh >= 2 * 4096 * 256 * 4
    # compute = F64 never tries the Gram route
    assert size(L.F64, 0) == size(L.F64, 1)
    st, _ = size(L.F32, 2)
    assert st == 1 and b"factor" in lib.slso_last_error()  # INVALID_ARG


def test_shape_errors_are_reported_before_any_device_work(lib):
    from paper_1812_07903_gb300 import _lib as L
    nbytes = ctypes.c_size_t(0)
    bad = L.Params(kind=L.COUNTSKETCH, compute=L.F32, s=8, k=0, seed_S=1, seed_Pi=2, tau=-1.0, correct_frac=0.0)
    assert lib.slso_workspace_size(ctypes.byref(bad), 1000, 16, ctypes.byref(nbytes)) == 2  # s < d
    assert b"s >= d" in lib.slso_last_error()
    bad.s, bad.k = 64, 5000
    assert lib.slso_workspace_size(ctypes.byref(bad), 1000, 16, ctypes.byref(nbytes)) == 2  # k > 4096
    bad.k, bad.kind = 0, 7
    assert lib.slso_workspace_size(ctypes.byref(bad), 1000, 16, ctypes.byref(nbytes)) == 1
    bad.kind, bad.s = L.SRHT, 2048
    assert lib.slso_workspace_size(ctypes.byref(bad), 1000, 16, ctypes.byref(nbytes)) == 2  # s > n_pad


def test_handle_calls_reject_null_handle(lib):
    from paper_1812_07903_gb300 import _lib as L
    assert lib.slso_order(None, None, L.F32, 10, None, None) == 1  # INVALID_ARG: NULL handle
    assert lib.slso_destroy(None) == L.SLSO_OK


def test_binding_maps_the_factor_choice():
    from paper_1812_07903_gb300 import api
    assert api.make_params(s=64, factor="auto").factor == 0
    assert api.make_params(s=64, factor="householder").factor == 1
    with pytest.raises(ValueError, match="factor"):
        api.make_params(s=64, factor="cholesky")
