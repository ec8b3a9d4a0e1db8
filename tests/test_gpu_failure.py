"""Failure detection without a GPU fault.

* The bounded device waits (the QR's ready-flag wait, the tensor-core kernels' mbarrier wait)
  run on something nothing ever signals: each gives up after its short limit, the host gets
  SLSO_ERR_TIMEOUT, and the same handle then computes normally (the context is intact).
* Forced allocation failure: a pool cap below a call's scratch gives SLSO_ERR_OOM before
  anything is launched; lifting the cap lets the same call run.
* A queued serving job is cancelled: poll reports CANCELLED; running or finished jobs cannot be
  cancelled; the jobs around it finish normally.
"""
import time

import numpy as np
import pytest
import torch

from oracle import slso_oracle as O
from paper_1812_07903_gb300 import _lib as L
from paper_1812_07903_gb300 import api, inputs

pytestmark = pytest.mark.gpu


def _small_leverage(handle):
    X = inputs.lognormal_rows(2000, 24, seed=3, dtype=torch.float32).cuda()
    sc, info = api.leverage(X, "countsketch", 256, 8, 1, 2, compute="f32", handle=handle)
    want, _ = O.sketched_leverage(X.cpu().double().numpy(), "countsketch", 256, 8, 1, 2)
    assert info["rank"] == 24
    assert float(np.max(np.abs(sc.cpu().numpy() - want) / want)) < 1e-4


@pytest.mark.parametrize("what", ["flag", "mbarrier"])
def test_bounded_wait_times_out_and_context_stays_usable(what):
    h = api.Handle()
    t0 = time.perf_counter()
    with pytest.raises(L.SlsoError) as e:
        api.selftest_wait(what, limit_us=20000, handle=h)
    assert e.value.status == 7  # SLSO_ERR_TIMEOUT
    assert time.perf_counter() - t0 < 5.0
    _small_leverage(h)
    h.close()


def test_forced_allocation_failure_then_recovery():
    h = api.Handle()
    X = inputs.lognormal_rows(50000, 64, seed=4, dtype=torch.float32).cuda()
    api.set_pool_limit(1 << 20, handle=h)
    with pytest.raises(L.SlsoError) as e:
        api.leverage(X, "countsketch", 1024, 16, 1, 2, handle=h)
    assert e.value.status == 4  # SLSO_ERR_OOM
    api.set_pool_limit(0, handle=h)
    sc, info = api.leverage(X, "countsketch", 1024, 16, 1, 2, handle=h)
    assert info["rank"] == 64 and torch.isfinite(sc).all()
    h.close()


def test_cancel_a_queued_serving_job():
    srv = api.Server(slots=1, mem_budget_bytes=8 << 30)
    big = inputs.gaussian_mixture(1 << 20, 256, seed=1, device="cuda")
    small = inputs.gaussian_mixture(4096, 64, seed=2, device="cuda")
    t_big = srv.submit_leverage(big, "gaussian", 1024, 64, 1, 2)
    t_mid = srv.submit_leverage(small, "countsketch", 512, 16, 3, 4)
    t_cut = srv.submit_leverage(small, "countsketch", 512, 16, 5, 6)
    srv.cancel(t_cut)  # one slot: the big job runs, the other two wait
    # submit returns before the worker admits the big job; cancel it only once it has left the queue
    deadline = time.perf_counter() + 30.0
    while srv.counters()["admitted"] < 1 and time.perf_counter() < deadline:
        time.sleep(0.001)
    assert srv.counters()["admitted"] >= 1
    with pytest.raises(L.SlsoError) as e:
        srv.cancel(t_big)
    assert e.value.status == 8  # BUSY: already running
    st_cut, _, _, _ = srv.poll(t_cut)
    assert st_cut == 10  # SLSO_ERR_CANCELLED
    st_big, info_big, _, _ = srv.poll(t_big)
    st_mid, info_mid, _, _ = srv.poll(t_mid)
    assert st_big == 0 and st_mid == 0 and info_mid["rank"] == 64
    with pytest.raises(L.SlsoError) as e:
        srv.cancel(t_mid)
    assert e.value.status == 9  # NOT_FOUND: collected
    srv.close()
