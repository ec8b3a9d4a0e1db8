"""Python binding of the C ABI: the same entry points, taking torch CUDA tensors.

Only argument marshalling happens here; every step of the path runs in libslso's kernels.
PyTorch provides device memory and the current stream.  There is no CPU fallback: without
a CUDA device, or without the built library, these functions raise.
"""
from __future__ import annotations

import ctypes

import torch

from . import _lib as L

_XDT = {torch.float64: L.F64, torch.float32: L.F32, torch.bfloat16: L.BF16}


def _stream(t=None):
    return ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)


def _require_cuda(*ts):
    for t in ts:
        if not (isinstance(t, torch.Tensor) and t.is_cuda):
            raise TypeError("slso needs CUDA tensors (there is no CPU path)")


class Handle:
    """Owns an slso_handle (device scratch pool) on one device."""

    def __init__(self, device=None):
        lib = L.load()
        if not torch.cuda.is_available():
            raise RuntimeError("slso needs a CUDA device")
        dev = torch.cuda.current_device() if device is None else int(device)
        self._h = ctypes.c_void_p()
        L.check(lib.slso_create(ctypes.byref(self._h), dev))
        self.device = dev

    def close(self):
        if self._h:
            L.load().slso_destroy(self._h)
            self._h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    @property
    def ptr(self):
        return self._h


_default = {}


def default_handle():
    dev = torch.cuda.current_device()
    if dev not in _default:
        _default[dev] = Handle(dev)
    return _default[dev]


def _x_args(X):
    _require_cuda(X)
    if X.dim() != 2 or X.dtype not in _XDT:
        raise TypeError("X must be a 2-D float64/float32/bfloat16 CUDA tensor")
    if X.stride(1) != 1:
        raise ValueError("X rows must be contiguous (stride(1) == 1)")
    n, d = X.shape
    return n, d, X.stride(0), _XDT[X.dtype]


def sketch(X, kind, s, seed, handle=None):
    """slso_sketch: SX = S X as an s x d float64 tensor."""
    h = handle or default_handle()
    n, d, ldx, xdt = _x_args(X)
    SX = torch.empty(s, d, dtype=torch.float64, device=X.device)
    L.check(L.load().slso_sketch(h.ptr, X.data_ptr(), n, d, ldx, xdt, L.KIND[kind], s, seed,
                                 SX.data_ptr(), _stream()))
    return SX


def sketched_svd(SX, tau=-1.0, want_r=True, handle=None):
    """slso_sketched_svd: (sigma, V, R, info) of the s x d float64 sketch."""
    h = handle or default_handle()
    _require_cuda(SX)
    if SX.dtype != torch.float64 or not SX.is_contiguous():
        raise TypeError("SX must be a contiguous float64 CUDA tensor")
    s, d = SX.shape
    sigma = torch.empty(d, dtype=torch.float64, device=SX.device)
    V = torch.empty(d, d, dtype=torch.float64, device=SX.device)
    R = torch.empty(d, d, dtype=torch.float64, device=SX.device) if want_r else None
    info = L.Info()
    L.check(L.load().slso_sketched_svd(h.ptr, SX.data_ptr(), s, d, float(tau), sigma.data_ptr(),
                                       V.data_ptr(), R.data_ptr() if R is not None else None,
                                       ctypes.byref(info), _stream()))
    return sigma, V, R, info.as_dict()


def gram(SX, handle=None):
    """slso_gram: G = SX^T SX (d x d float64) as the float32 path's Gram route forms it."""
    h = handle or default_handle()
    _require_cuda(SX)
    if SX.dtype != torch.float64 or not SX.is_contiguous():
        raise TypeError("SX must be a contiguous float64 CUDA tensor")
    s, d = SX.shape
    G = torch.empty(d, d, dtype=torch.float64, device=SX.device)
    L.check(L.load().slso_gram(h.ptr, SX.data_ptr(), s, d, G.data_ptr(), _stream()))
    return G


FACTOR = {"auto": 0, "householder": 1}


def make_params(kind="countsketch", s=None, k=0, seed_S=0, seed_Pi=0, tau=-1.0, compute="f32",
                correct_frac=0.0, nnz=0, factor="auto"):
    """factor: how R of SX is formed; 'auto' tries the probe-checked Gram route (R = chol(SX^T SX))
    when compute != 'f64', 'householder' always takes Householder QR."""
    p = L.Params()
    p.kind = L.KIND[kind]
    p.compute = L.DTYPE[compute]
    p.s = int(s)
    p.k = int(k)
    p.seed_S = int(seed_S)
    p.seed_Pi = int(seed_Pi)
    p.tau = float(tau)
    p.correct_frac = float(correct_frac)
    p.nnz = int(nnz)
    if factor not in FACTOR:
        raise ValueError(f"factor must be one of {sorted(FACTOR)}, not {factor!r}")
    p.factor = FACTOR[factor]
    return p


def leverage(X, kind="countsketch", s=None, k=0, seed_S=0, seed_Pi=0, tau=-1.0, compute="f32",
             correct_frac=0.0, out=None, want_info=True, handle=None, nnz=0, factor="auto"):
    """slso_leverage: approximate leverage scores (float64 for compute='f64', else float32).
    nnz: OSNAP nonzeros per column of S (0: the default 4); factor: see make_params."""
    h = handle or default_handle()
    n, d, ldx, xdt = _x_args(X)
    p = make_params(kind, s, k, seed_S, seed_Pi, tau, compute, correct_frac, nnz, factor)
    sdt = torch.float64 if compute == "f64" else torch.float32
    scores = out if out is not None else torch.empty(n, dtype=sdt, device=X.device)
    info = L.Info()
    st = L.load().slso_leverage(h.ptr, X.data_ptr(), n, d, ldx, xdt, ctypes.byref(p), scores.data_ptr(),
                                ctypes.byref(info) if want_info else None, _stream())
    L.check(st)
    return scores, (info.as_dict() if want_info else None)


def approx_u(X, kind="countsketch", s=None, seed_S=0, tau=-1.0, out=None, handle=None, nnz=0):
    """slso_approx_u: U = X V_r Sigma_r^-1 from the sketched SVD (n x d; columns >= rank are zero)."""
    h = handle or default_handle()
    n, d, ldx, xdt = _x_args(X)
    p = make_params(kind, s, 0, seed_S, 0, tau, "f32", 0.0, nnz)
    udt = torch.float64 if X.dtype == torch.float64 else torch.float32
    U = out if out is not None else torch.empty(n, d, dtype=udt, device=X.device)
    if U.dtype != udt or U.dim() != 2 or U.shape != (n, d) or U.stride(1) != 1:
        raise TypeError(f"out must be a row-contiguous {udt} tensor of shape ({n}, {d})")
    info = L.Info()
    L.check(L.load().slso_approx_u(h.ptr, X.data_ptr(), n, d, ldx, xdt, ctypes.byref(p), U.data_ptr(), U.stride(0),
                                   ctypes.byref(info), _stream()))
    return U, info.as_dict()


def order(scores, out=None, handle=None):
    """slso_order: the "dec" ordering (int64 row indices) of a float32/float64 score vector."""
    h = handle or default_handle()
    _require_cuda(scores)
    if scores.dtype not in (torch.float32, torch.float64) or not scores.is_contiguous():
        raise TypeError("scores must be a contiguous float32/float64 CUDA tensor")
    n = scores.numel()
    o = out if out is not None else torch.empty(n, dtype=torch.int64, device=scores.device)
    sdt = L.F32 if scores.dtype == torch.float32 else L.F64
    L.check(L.load().slso_order(h.ptr, scores.data_ptr(), sdt, n, o.data_ptr(), _stream()))
    return o


def sample_order(scores, policy="swor", seed=0, out=None, handle=None):
    """slso_sample_order: the "dec", "swr" or "swor" ordering (Algorithm 4 step 4) of a score vector."""
    h = handle or default_handle()
    _require_cuda(scores)
    if scores.dtype not in (torch.float32, torch.float64) or not scores.is_contiguous():
        raise TypeError("scores must be a contiguous float32/float64 CUDA tensor")
    if policy not in L.POLICY:
        raise ValueError(f"policy must be one of {sorted(L.POLICY)}")
    n = scores.numel()
    o = out if out is not None else torch.empty(n, dtype=torch.int64, device=scores.device)
    sdt = L.F32 if scores.dtype == torch.float32 else L.F64
    L.check(L.load().slso_sample_order(h.ptr, scores.data_ptr(), sdt, n, L.POLICY[policy], seed, o.data_ptr(),
                                       _stream()))
    return o


def rank_rows_host(X_host, kind="countsketch", s=None, k=0, seed_S=0, seed_Pi=0, tau=-1.0,
                   compute="f32", correct_frac=0.0, scores_out=None, order_out=None, handle=None, nnz=0):
    """slso_rank_rows_host: scores and order from a HOST matrix (copies inside the call)."""
    h = handle or default_handle()
    if X_host.is_cuda or X_host.dim() != 2 or X_host.dtype not in _XDT or X_host.stride(1) != 1:
        raise TypeError("X_host must be a 2-D row-contiguous host tensor (float64/float32/bfloat16)")
    n, d = X_host.shape
    p = make_params(kind, s, k, seed_S, seed_Pi, tau, compute, correct_frac, nnz)
    sdt = torch.float64 if compute == "f64" else torch.float32
    sc = scores_out if scores_out is not None else torch.empty(n, dtype=sdt)
    od = order_out if order_out is not None else torch.empty(n, dtype=torch.int64)
    info = L.Info()
    L.check(L.load().slso_rank_rows_host(h.ptr, X_host.data_ptr(), n, d, X_host.stride(0), _XDT[X_host.dtype],
                                         ctypes.byref(p), sc.data_ptr(), od.data_ptr(), ctypes.byref(info),
                                         _stream()))
    return sc, od, info.as_dict()


def rank_rows_streamed(X_host, kind="countsketch", s=None, k=0, seed_S=0, seed_Pi=0, tau=-1.0, compute="f32",
                       block_rows=0, scores_out=None, order_out=None, handle=None, nnz=0, factor="auto"):
    """slso_rank_rows_streamed: scores and order of a HOST matrix streamed through the device in
    blocks of rows (out-of-core X: device memory independent of n x d)."""
    h = handle or default_handle()
    if X_host.is_cuda or X_host.dim() != 2 or X_host.dtype not in _XDT or X_host.stride(1) != 1:
        raise TypeError("X_host must be a 2-D row-contiguous host tensor (float64/float32/bfloat16)")
    n, d = X_host.shape
    p = make_params(kind, s, k, seed_S, seed_Pi, tau, compute, 0.0, nnz, factor)
    sdt = torch.float64 if compute == "f64" else torch.float32
    sc = scores_out if scores_out is not None else torch.empty(n, dtype=sdt)
    od = order_out if order_out is not None else torch.empty(n, dtype=torch.int64)
    info = L.Info()
    L.check(L.load().slso_rank_rows_streamed(h.ptr, X_host.data_ptr(), n, d, X_host.stride(0), _XDT[X_host.dtype],
                                             ctypes.byref(p), int(block_rows), sc.data_ptr(), od.data_ptr(),
                                             ctypes.byref(info), _stream()))
    return sc, od, info.as_dict()


def rank_rows_host_batch(X_hosts, kind="countsketch", s=None, k=0, seed_S=0, seed_Pi=0, tau=-1.0,
                         compute="f32", correct_frac=0.0, scores_out=None, order_out=None, handle=None,
                         nnz=0):
    """slso_rank_rows_host_batch: rank_rows_host over a list of same-shaped HOST matrices, with the
    copies of one item overlapped with the computation of its neighbours.  Returns lists of
    (scores, order) host tensors and the per-item info dicts."""
    h = handle or default_handle()
    if not X_hosts:
        raise ValueError("X_hosts must hold at least one matrix")
    X0 = X_hosts[0]
    for X in X_hosts:
        if (X.is_cuda or X.dim() != 2 or X.dtype not in _XDT or X.stride(1) != 1 or X.shape != X0.shape
                or X.dtype != X0.dtype or X.stride(0) != X0.stride(0)):
            raise TypeError("X_hosts must be 2-D row-contiguous host tensors of one shape, dtype and row stride")
    cnt = len(X_hosts)
    n, d = X0.shape
    p = make_params(kind, s, k, seed_S, seed_Pi, tau, compute, correct_frac, nnz)
    sdt = torch.float64 if compute == "f64" else torch.float32
    sc = scores_out or [torch.empty(n, dtype=sdt) for _ in range(cnt)]
    od = order_out or [torch.empty(n, dtype=torch.int64) for _ in range(cnt)]
    xs = (ctypes.c_void_p * cnt)(*[X.data_ptr() for X in X_hosts])
    ss = (ctypes.c_void_p * cnt)(*[t.data_ptr() for t in sc])
    os_ = (ctypes.c_void_p * cnt)(*[t.data_ptr() for t in od])
    infos = (L.Info * cnt)()
    L.check(L.load().slso_rank_rows_host_batch(h.ptr, cnt, xs, n, d, X0.stride(0), _XDT[X0.dtype], ctypes.byref(p),
                                               ss, os_, infos, _stream()))
    return sc, od, [i.as_dict() for i in infos]


def set_pool_limit(nbytes, handle=None):
    """slso_set_pool_limit: cap the handle's device pool (0: no cap); larger calls fail with OOM."""
    h = handle or default_handle()
    L.check(L.load().slso_set_pool_limit(h.ptr, int(nbytes)))


SCORE_FORMS = {"mixed": 0, "tf32x3": 1, "tf32x3_smem": 2}


def set_score_form(form, handle=None):
    """slso_set_score_form: operand form of the float32 score product for k <= 128 ("mixed",
    "tf32x3", "tf32x3_smem")."""
    h = handle or default_handle()
    L.check(L.load().slso_set_score_form(h.ptr, SCORE_FORMS[form]))


def selftest_wait(what="flag", limit_us=2000, handle=None):
    """slso_selftest_wait: run a bounded device wait that nothing signals; raises SlsoError(TIMEOUT)."""
    h = handle or default_handle()
    code = {"flag": 0, "mbarrier": 1}[what]
    L.check(L.load().slso_selftest_wait(h.ptr, code, int(limit_us), _stream()))


def profile(enable=True, handle=None):
    """slso_profile: start (or stop) per-stage event timing on the handle."""
    h = handle or default_handle()
    L.check(L.load().slso_profile(h.ptr, 1 if enable else 0))


def profile_read(handle=None):
    """slso_profile_read: {stage: (total ms, calls)} and the kernel launch count."""
    h = handle or default_handle()
    ms = (ctypes.c_double * len(L.STAGES))()
    calls = (ctypes.c_int64 * len(L.STAGES))()
    launches = ctypes.c_int64(0)
    L.check(L.load().slso_profile_read(h.ptr, ms, calls, ctypes.byref(launches)))
    return {name: (ms[i], calls[i]) for i, name in enumerate(L.STAGES)}, launches.value


class Server:
    """slso_server_*: continuous batching of leverage and sketched-SVD jobs on one device.

    Tensors referenced by a job are kept alive by the Server until the job is polled.
    """

    def __init__(self, slots=4, mem_budget_bytes=8 << 30, device=None):
        lib = L.load()
        dev = torch.cuda.current_device() if device is None else int(device)
        self._s = ctypes.c_void_p()
        L.check(lib.slso_server_create(ctypes.byref(self._s), dev, int(slots), int(mem_budget_bytes)))
        self._keep = {}

    def submit_leverage(self, X, kind="countsketch", s=None, k=0, seed_S=0, seed_Pi=0, tau=-1.0,
                        compute="f32", correct_frac=0.0, with_order=True, nnz=0):
        n, d, ldx, xdt = _x_args(X)
        j = L.Job()
        j.job, j.xdt, j.X, j.n, j.d, j.ldx = L.JOB_LEVERAGE, xdt, X.data_ptr(), n, d, ldx
        j.params = make_params(kind, s, k, seed_S, seed_Pi, tau, compute, correct_frac, nnz)
        sdt = torch.float64 if compute == "f64" else torch.float32
        scores = torch.empty(n, dtype=sdt, device=X.device)
        order = torch.empty(n, dtype=torch.int64, device=X.device) if with_order else None
        j.scores = scores.data_ptr()
        j.order = order.data_ptr() if order is not None else None
        t = ctypes.c_int64(0)
        L.check(L.load().slso_server_submit(self._s, ctypes.byref(j), ctypes.byref(t)))
        self._keep[t.value] = (X, scores, order)
        return t.value

    def submit_sketched_svd(self, SX, tau=-1.0):
        _require_cuda(SX)
        s, d = SX.shape
        j = L.Job()
        j.job, j.xdt, j.X, j.n, j.d, j.ldx = L.JOB_SKETCHED_SVD, L.F64, SX.data_ptr(), s, d, d
        j.params = make_params("countsketch", s, 0, 0, 0, tau, "f64", 0.0)
        sigma = torch.empty(d, dtype=torch.float64, device=SX.device)
        V = torch.empty(d, d, dtype=torch.float64, device=SX.device)
        R = torch.empty(d, d, dtype=torch.float64, device=SX.device)
        j.sigma, j.V, j.R = sigma.data_ptr(), V.data_ptr(), R.data_ptr()
        t = ctypes.c_int64(0)
        L.check(L.load().slso_server_submit(self._s, ctypes.byref(j), ctypes.byref(t)))
        self._keep[t.value] = (SX, sigma, V, R)
        return t.value

    def poll(self, ticket, timeout_ms=60000):
        """(status, info dict, times_ms [queued, running, total], outputs) of a finished job."""
        st = ctypes.c_int32(0)
        info = L.Info()
        times = (ctypes.c_double * 3)()
        L.check(L.load().slso_server_poll(self._s, int(ticket), int(timeout_ms), ctypes.byref(st),
                                          ctypes.byref(info), times))
        outs = self._keep.pop(ticket)
        return st.value, info.as_dict(), list(times), outs[1:]

    def cancel(self, ticket):
        """slso_server_cancel: cancel a job still waiting for admission (poll then reports CANCELLED)."""
        L.check(L.load().slso_server_cancel(self._s, int(ticket)))

    def stats(self):
        c = (ctypes.c_int64 * 4)()
        mem = ctypes.c_size_t(0)
        L.check(L.load().slso_server_stats(self._s, c, ctypes.byref(mem)))
        return {"submitted": c[0], "admitted": c[1], "completed": c[2], "queued": c[3], "mem_in_use": mem.value}

    def counters(self):
        """slso_server_counters: job counts, scratch in use, the graph-capture counters and the
        grouped score launches with the jobs they ran."""
        names = ("submitted", "admitted", "completed", "queued", "mem_in_use", "graphs_new", "graphs_updated",
                 "direct", "group_launches", "grouped_jobs")
        c = (ctypes.c_int64 * len(names))()
        L.check(L.load().slso_server_counters(self._s, c, len(names)))
        return dict(zip(names, list(c)))

    def close(self):
        if self._s:
            L.load().slso_server_destroy(self._s)
            self._s = ctypes.c_void_p()
            self._keep.clear()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def default_tau(s, d):
    return max(s, d) * 2.0**-52

