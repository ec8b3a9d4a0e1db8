"""slso_order_static: the ordering entry point that allocates nothing.

It serves callers that cannot allocate device memory when they need an ordering (another
framework owns all device memory, allocation is forbidden after start-up, or the work is being
recorded into someone else's CUDA graph).  Its scratch is a fixed array inside the library, so
this test checks, through the C ABI, that two calls in a row give exactly the order the
allocating entry point gives, and that sizes beyond the array are refused.  This file is
collected last, and it passes on its own in a fresh process as well.
"""
import ctypes

import numpy as np
import pytest
import torch

from paper_1812_07903_gb300 import _lib as L
from paper_1812_07903_gb300 import api

pytestmark = pytest.mark.gpu

MAX_N = 1 << 20


def _scores(n, dtype, seed):
    g = torch.Generator().manual_seed(seed)
    sc = torch.floor(torch.rand(n, generator=g, dtype=torch.float64) * 1000) / 1000  # many ties
    sc[::97] = 0.0
    sc[5::101] = -0.0
    sc[7::211] = float("nan")
    return sc.to(dtype).cuda()


def _static(lib, sc, out):
    sdt = L.F32 if sc.dtype == torch.float32 else L.F64
    st = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    return lib.slso_order_static(sc.data_ptr(), sdt, sc.numel(), out.data_ptr(), st)


@pytest.mark.parametrize("n,dtype", [(MAX_N, torch.float32), (300007, torch.float64), (1, torch.float32)])
def test_static_order_matches_allocating_order_twice(n, dtype):
    lib = L.load()
    sc = _scores(n, dtype, n)
    want = api.order(sc).cpu()
    for _ in range(2):  # the shared scratch keeps the previous call's contents
        out = torch.full((n,), -1, dtype=torch.int64, device="cuda")
        assert _static(lib, sc, out) == L.SLSO_OK, lib.slso_last_error()
        torch.cuda.synchronize()
        assert torch.equal(out.cpu(), want)


def test_static_order_refuses_sizes_beyond_its_scratch():
    lib = L.load()
    sc = torch.zeros(MAX_N + 1, dtype=torch.float32, device="cuda")
    out = torch.empty(MAX_N + 1, dtype=torch.int64, device="cuda")
    assert _static(lib, sc, out) == 2  # SLSO_ERR_SHAPE
    assert b"2^20" in lib.slso_last_error() or b"1048576" in lib.slso_last_error()
