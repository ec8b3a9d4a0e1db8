// C ABI entry points of libslso (declared in include/slso.h).
//
// Each entry point validates its arguments on the host, sizes its scratch by running its plan
// against a measuring Arena, grows the handle's pool if needed, and then enqueues the plan on
// the caller's stream.  Only an `info` request synchronises.
#include <algorithm>
#include <cmath>
#include <cstring>

#include <vector>

#include "common.cuh"

using namespace slso;

namespace slso {

// Streamed entry point: rows per block (a power of two; a multiple of SRHT's 8192-row chunks and of
// the Gaussian generator's 4-column Philox blocks).
constexpr int64_t kStreamMinBlock = 65536;
constexpr int64_t kStreamDefaultBlock = 262144;

double default_tau(int64_t s, int64_t d) { return static_cast<double>(std::max(s, d)) * std::ldexp(1.0, -52); }

int64_t next_pow2(int64_t n) {
  int64_t p = 1;
  while (p < n) p <<= 1;
  return p;
}

slso_status check_x(const void* X, int64_t n, int64_t d, int64_t ldx, int32_t xdt) {
  if (!X) return fail(SLSO_ERR_INVALID_ARG, "X is NULL");
  if (n < 1 || d < 1) return fail(SLSO_ERR_SHAPE, "need n >= 1 and d >= 1 (n=%lld, d=%lld)", (long long)n, (long long)d);
  if (ldx < d) return fail(SLSO_ERR_SHAPE, "ldx=%lld < d=%lld", (long long)ldx, (long long)d);
  if (n >= (int64_t(1) << 31)) return fail(SLSO_ERR_SHAPE, "n=%lld must be < 2^31", (long long)n);
  if (xdt != SLSO_F64 && xdt != SLSO_F32 && xdt != SLSO_BF16)
    return fail(SLSO_ERR_DTYPE, "X dtype %d not supported (F64, F32, BF16)", xdt);
  return SLSO_OK;
}

slso_status check_sketch(int32_t kind, int64_t n, int64_t d, int64_t s, int32_t nnz) {
  if (kind != SLSO_COUNTSKETCH && kind != SLSO_SRHT && kind != SLSO_GAUSSIAN && kind != SLSO_OSNAP)
    return fail(SLSO_ERR_INVALID_ARG, "unknown sketch kind %d", kind);
  if (kind == SLSO_OSNAP) {
    const int64_t z = nnz > 0 ? nnz : kOsnapDefaultNnz;
    if (nnz < 0 || z > 64) return fail(SLSO_ERR_INVALID_ARG, "OSNAP nnz=%d must be in 0 .. 64", nnz);
    if (s % z != 0) return fail(SLSO_ERR_SHAPE, "OSNAP needs s=%lld divisible by nnz=%lld", (long long)s, (long long)z);
    if (n * z >= (int64_t(1) << 31)) return fail(SLSO_ERR_SHAPE, "OSNAP needs n * nnz < 2^31");
  }
  if (s < 1) return fail(SLSO_ERR_SHAPE, "s=%lld must be >= 1", (long long)s);
  if (s >= (int64_t(1) << 31)) return fail(SLSO_ERR_SHAPE, "s=%lld must be < 2^31", (long long)s);
  if (kind == SLSO_SRHT && s > next_pow2(n))
    return fail(SLSO_ERR_SHAPE, "SRHT needs s <= n_pad=%lld (s=%lld)", (long long)next_pow2(n), (long long)s);
  (void)d;
  return SLSO_OK;
}

slso_status check_params(const slso_params* p, int64_t n, int64_t d) {
  if (!p) return fail(SLSO_ERR_INVALID_ARG, "params is NULL");
  SLSO_TRY(check_sketch(p->kind, n, d, p->s, p->nnz));
  if (p->s < d) return fail(SLSO_ERR_SHAPE, "need s >= d for the d x d factor R (s=%lld, d=%lld)", (long long)p->s, (long long)d);
  if (p->k < 0 || p->k > 4096) return fail(SLSO_ERR_SHAPE, "k=%lld must be in [0, 4096]", (long long)p->k);
  if (p->compute != SLSO_F64 && p->compute != SLSO_F32 && p->compute != SLSO_BF16 && p->compute != SLSO_FP8_E4M3)
    return fail(SLSO_ERR_DTYPE, "unknown compute dtype %d", p->compute);
  if (!(p->correct_frac >= 0.0 && p->correct_frac <= 1.0))
    return fail(SLSO_ERR_INVALID_ARG, "correct_frac must be in [0, 1]");
  if (std::isnan(p->tau)) return fail(SLSO_ERR_INVALID_ARG, "tau is NaN");
  if (d > kMaxD) return fail(SLSO_ERR_SHAPE, "d=%lld exceeds %lld", (long long)d, (long long)kMaxD);
  if (p->factor != SLSO_FACTOR_AUTO && p->factor != SLSO_FACTOR_HOUSEHOLDER)
    return fail(SLSO_ERR_INVALID_ARG, "unknown factor %d", p->factor);
  return SLSO_OK;
}

bool use_gram(const slso_params* p) { return p->factor == SLSO_FACTOR_AUTO && p->compute != SLSO_F64; }

void info_from_state(const DevState& d, slso_info* info) {
  info->rank = d.rank;
  info->sigma_max = d.sigma_max;
  info->sigma_min_kept = d.sigma_min_kept;
  info->score_sum = d.score_sum;
  info->tau = d.tau;
  info->nonfinite = d.nonfinite;
  info->svd_route = d.need_svd;
  info->svd_sweeps = d.sweeps;
  info->gram_route = d.gram_ok;
  info->gram_resid = d.gram_tried ? d.gram_resid : std::nan("");
}

}  // namespace slso

namespace {

template <class Plan>
slso_status run_plan(Handle& h, Plan&& plan) {
  Arena m(nullptr, ~size_t(0), true);
  SLSO_TRY(plan(m));
  SLSO_TRY(ensure_pool(h, m.used()));
  Arena real(h.pool, h.pool_cap, false);
  SLSO_TRY(plan(real));
  if (real.overflow()) return fail(SLSO_ERR_OOM, "internal: scratch plan overflowed the pool");
  return SLSO_OK;
}

slso_status fill_info(Handle& h, cudaStream_t st, slso_info* info) {
  SLSO_CHECK_CUDA(cudaMemcpyAsync(h.state_host, h.state, sizeof(DevState), cudaMemcpyDeviceToHost, st));
  SLSO_CHECK_CUDA(cudaStreamSynchronize(st));
  const DevState& d = *h.state_host;
  info_from_state(d, info);
  if (d.timeout) return fail(SLSO_ERR_TIMEOUT, "a bounded device wait gave up (kernel %d)", d.timeout);
  if (d.nonfinite) return fail(SLSO_ERR_NONFINITE, "X holds NaN or Inf");
  return SLSO_OK;
}

}  // namespace

namespace slso {

slso_status leverage_solve(Handle& h, Arena& ar, const void* X, int64_t n, int64_t d, int64_t ldx,
                           int32_t xdt, const slso_params* p, cudaStream_t st, const double** M, int64_t* kk,
                           const unsigned int** colmax_out) {
  const double tau = p->tau < 0 ? default_tau(p->s, d) : p->tau;
  double* SX = ar.take<double>(static_cast<size_t>(p->s) * d);
  // FP8 scores of float32 / bfloat16 X after a CountSketch or OSNAP: the column maxima of |X| come
  // out of the sketch's pass over X, so X is read twice in all
  const bool fuse_max = p->compute == SLSO_FP8_E4M3 && xdt != SLSO_F64 &&
                        (p->kind == SLSO_COUNTSKETCH || p->kind == SLSO_OSNAP);
  unsigned int* colmax = fuse_max ? ar.take<unsigned int>(d) : nullptr;
  SketchBlock blk;
  blk.colmax = colmax;
  if (colmax && !ar.measure()) SLSO_CHECK_CUDA(cudaMemsetAsync(colmax, 0, sizeof(unsigned int) * d, st));
  prof_begin(h, ar, ST_SKETCH, st);
  SLSO_TRY(run_sketch(h, ar, X, n, d, ldx, xdt, p->kind, p->s, p->seed_S, p->nnz, SX, st, &blk));
  prof_end(h, ar, st);
  SolveOut so;
  SLSO_TRY(run_solve(h, ar, SX, p->s, d, tau, p->k, p->seed_Pi, 0, &so, st, use_gram(p)));
  *M = so.M;
  *kk = p->k > 0 ? p->k : d;
  *colmax_out = colmax;
  return SLSO_OK;
}

slso_status leverage_plan(Handle& h, Arena& ar, const void* X, int64_t n, int64_t d, int64_t ldx,
                          int32_t xdt, const slso_params* p, void* scores, cudaStream_t st) {
  const double* M = nullptr;
  int64_t kk = 0;
  const unsigned int* colmax = nullptr;
  SLSO_TRY(leverage_solve(h, ar, X, n, d, ldx, xdt, p, st, &M, &kk, &colmax));
  prof_begin(h, ar, ST_SCORES, st);
  SLSO_TRY(run_scores(h, ar, X, n, d, ldx, xdt, M, kk, p->compute, scores, p->correct_frac, st, colmax));
  prof_end(h, ar, st);
  return SLSO_OK;
}

}  // namespace slso

extern "C" slso_status slso_workspace_size(const slso_params* params, int64_t n, int64_t d, size_t* bytes) {
  if (!bytes) return fail(SLSO_ERR_INVALID_ARG, "bytes is NULL");
  SLSO_TRY(check_params(params, n, d));
  Handle h;
  h.num_sms = 148;
  Arena m(nullptr, ~size_t(0), true);
  const int32_t sdt = params->compute == SLSO_F64 ? SLSO_F64 : SLSO_F32;
  SLSO_TRY(leverage_plan(h, m, reinterpret_cast<const void*>(16), n, d, d, SLSO_F32, params,
                         reinterpret_cast<void*>(16), nullptr));
  SLSO_TRY(order_scores(h, m, reinterpret_cast<const void*>(16), sdt, n, reinterpret_cast<int64_t*>(16), nullptr));
  *bytes = m.used();
  return SLSO_OK;
}

extern "C" slso_status slso_sketch(slso_handle* handle, const void* X, int64_t n, int64_t d, int64_t ldx,
                                   int32_t xdt, int32_t kind, int64_t s, uint64_t seed_S, double* SX,
                                   void* stream) {
  Handle* h = nullptr;
  SLSO_TRY(check_handle(handle, &h));
  SLSO_TRY(check_x(X, n, d, ldx, xdt));
  SLSO_TRY(check_sketch(kind, n, d, s, 0));
  if (!SX) return fail(SLSO_ERR_INVALID_ARG, "SX is NULL");
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  SLSO_CHECK_CUDA(cudaMemsetAsync(h->state, 0, sizeof(DevState), st));
  return run_plan(*h, [&](Arena& ar) {
    prof_begin(*h, ar, ST_SKETCH, st);
    SLSO_TRY(run_sketch(*h, ar, X, n, d, ldx, xdt, kind, s, seed_S, 0, SX, st));
    prof_end(*h, ar, st);
    return SLSO_OK;
  });
}

extern "C" slso_status slso_sketched_svd(slso_handle* handle, const double* SX, int64_t s, int64_t d,
                                         double tau, double* sigma, double* V, double* R, slso_info* info,
                                         void* stream) {
  Handle* h = nullptr;
  SLSO_TRY(check_handle(handle, &h));
  if (!SX || !sigma || !V) return fail(SLSO_ERR_INVALID_ARG, "SX, sigma and V must be non-NULL");
  if (d < 1 || s < d) return fail(SLSO_ERR_SHAPE, "need 1 <= d <= s (s=%lld, d=%lld)", (long long)s, (long long)d);
  if (d > kMaxD || s >= (int64_t(1) << 31)) return fail(SLSO_ERR_SHAPE, "d <= %lld and s < 2^31 required", (long long)kMaxD);
  if (std::isnan(tau)) return fail(SLSO_ERR_INVALID_ARG, "tau is NaN");
  const double t = tau < 0 ? default_tau(s, d) : tau;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  SLSO_CHECK_CUDA(cudaMemsetAsync(h->state, 0, sizeof(DevState), st));
  SolveOut so;
  SLSO_TRY(run_plan(*h, [&](Arena& ar) { return run_solve(*h, ar, SX, s, d, t, 0, 0, 1, &so, st); }));
  SLSO_CHECK_CUDA(cudaMemcpyAsync(sigma, so.sigma, sizeof(double) * d, cudaMemcpyDeviceToDevice, st));
  SLSO_CHECK_CUDA(cudaMemcpyAsync(V, so.V, sizeof(double) * d * d, cudaMemcpyDeviceToDevice, st));
  if (R) SLSO_CHECK_CUDA(cudaMemcpyAsync(R, so.R, sizeof(double) * d * d, cudaMemcpyDeviceToDevice, st));
  if (info) return fill_info(*h, st, info);
  return SLSO_OK;
}

extern "C" slso_status slso_gram(slso_handle* handle, const double* SX, int64_t s, int64_t d, double* G,
                                 void* stream) {
  Handle* h = nullptr;
  SLSO_TRY(check_handle(handle, &h));
  if (!SX || !G) return fail(SLSO_ERR_INVALID_ARG, "SX and G must be non-NULL");
  if (d < 1 || d > kMaxD || s < 1 || s >= (int64_t(1) << 31))
    return fail(SLSO_ERR_SHAPE, "need 1 <= d <= %lld and 1 <= s < 2^31 (s=%lld, d=%lld)", (long long)kMaxD, (long long)s,
                (long long)d);
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  return run_plan(*h, [&](Arena& ar) {
    GramWork g = gram_take(*h, ar, s, d);
    double* L = ar.take<double>(static_cast<size_t>(d) * d);
    if (ar.measure()) return SLSO_OK;
    return run_gram_full(*h, ar, g, SX, s, d, L, G, st);
  });
}

extern "C" slso_status slso_leverage(slso_handle* handle, const void* X, int64_t n, int64_t d, int64_t ldx,
                                     int32_t xdt, const slso_params* params, void* scores, slso_info* info,
                                     void* stream) {
  Handle* h = nullptr;
  SLSO_TRY(check_handle(handle, &h));
  SLSO_TRY(check_x(X, n, d, ldx, xdt));
  SLSO_TRY(check_params(params, n, d));
  if (!scores) return fail(SLSO_ERR_INVALID_ARG, "scores is NULL");
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  SLSO_CHECK_CUDA(cudaMemsetAsync(h->state, 0, sizeof(DevState), st));
  SLSO_TRY(run_plan(*h, [&](Arena& ar) { return leverage_plan(*h, ar, X, n, d, ldx, xdt, params, scores, st); }));
  if (info) return fill_info(*h, st, info);
  return SLSO_OK;
}

extern "C" slso_status slso_approx_u(slso_handle* handle, const void* X, int64_t n, int64_t d, int64_t ldx,
                                     int32_t xdt, const slso_params* params, void* U, int64_t ldu, slso_info* info,
                                     void* stream) {
  Handle* h = nullptr;
  SLSO_TRY(check_handle(handle, &h));
  SLSO_TRY(check_x(X, n, d, ldx, xdt));
  SLSO_TRY(check_params(params, n, d));
  if (!U) return fail(SLSO_ERR_INVALID_ARG, "U is NULL");
  if (ldu < d) return fail(SLSO_ERR_SHAPE, "ldu=%lld must be >= d=%lld", (long long)ldu, (long long)d);
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  SLSO_CHECK_CUDA(cudaMemsetAsync(h->state, 0, sizeof(DevState), st));
  SLSO_TRY(run_plan(*h, [&](Arena& ar) { return approx_u_plan(*h, ar, X, n, d, ldx, xdt, params, U, ldu, st); }));
  if (info) return fill_info(*h, st, info);
  return SLSO_OK;
}

extern "C" slso_status slso_order(slso_handle* handle, const void* scores, int32_t sdt, int64_t n,
                                  int64_t* order, void* stream) {
  Handle* h = nullptr;
  SLSO_TRY(check_handle(handle, &h));
  if (!scores || !order) return fail(SLSO_ERR_INVALID_ARG, "scores and order must be non-NULL");
  if (n < 1 || n >= (int64_t(1) << 31)) return fail(SLSO_ERR_SHAPE, "need 1 <= n < 2^31");
  if (sdt != SLSO_F32 && sdt != SLSO_F64) return fail(SLSO_ERR_DTYPE, "scores must be F32 or F64");
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  return run_plan(*h, [&](Arena& ar) {
    prof_begin(*h, ar, ST_ORDER, st);
    SLSO_TRY(order_scores(*h, ar, scores, sdt, n, order, st));
    prof_end(*h, ar, st);
    return SLSO_OK;
  });
}

extern "C" slso_status slso_rank_rows_host_batch(slso_handle* handle, int64_t count, const void* const* X_host,
                                                 int64_t n, int64_t d, int64_t ldx, int32_t xdt,
                                                 const slso_params* params, void* const* scores_host,
                                                 int64_t* const* order_host, slso_info* info, void* stream) {
  Handle* h = nullptr;
  SLSO_TRY(check_handle(handle, &h));
  if (count < 1 || !X_host || !scores_host || !order_host)
    return fail(SLSO_ERR_INVALID_ARG, "need count >= 1 and non-NULL pointer arrays");
  for (int64_t i = 0; i < count; ++i) {
    SLSO_TRY(check_x(X_host[i], n, d, ldx, xdt));
    if (!scores_host[i] || !order_host[i]) return fail(SLSO_ERR_INVALID_ARG, "item %lld: NULL output", (long long)i);
  }
  SLSO_TRY(check_params(params, n, d));
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  const size_t esz = dtype_size(xdt);
  const int32_t sdt = params->compute == SLSO_F64 ? SLSO_F64 : SLSO_F32;
  const size_t ssz = dtype_size(sdt);
  const size_t xbytes = static_cast<size_t>(n) * d * esz;

  // fixed buffers (two of each: item i uses set i % 2) and one scratch region reused per item
  char* Xd[2] = {};
  char* sc[2] = {};
  int64_t* od[2] = {};
  DevState* states = nullptr;
  auto take_fixed = [&](Arena& ar) {
    for (int b = 0; b < 2; ++b) {
      Xd[b] = ar.take<char>(xbytes);
      sc[b] = ar.take<char>(static_cast<size_t>(n) * ssz);
      od[b] = ar.take<int64_t>(n);
    }
    states = ar.take<DevState>(count);
  };
  auto item = [&](Arena& ar, int b) -> slso_status {
    SLSO_TRY(leverage_plan(*h, ar, Xd[b], n, d, d, xdt, params, sc[b], st));
    prof_begin(*h, ar, ST_ORDER, st);
    SLSO_TRY(order_scores(*h, ar, sc[b], sdt, n, od[b], st));
    prof_end(*h, ar, st);
    return SLSO_OK;
  };
  Arena mf(nullptr, ~size_t(0), true);
  take_fixed(mf);
  const size_t scratch_off = (mf.used() + 255) & ~size_t(255);
  Arena mi(nullptr, ~size_t(0), true);
  SLSO_TRY(item(mi, 0));
  SLSO_TRY(ensure_pool(*h, scratch_off + mi.used()));
  Arena real(h->pool, h->pool_cap, false);
  take_fixed(real);

  cudaStream_t h2d = nullptr, d2h = nullptr;
  cudaEvent_t ev[9] = {};  // start, xready[2], xfree[2], oready[2], ofree[2]
  auto cleanup = [&]() {
    for (cudaEvent_t e : ev)
      if (e) cudaEventDestroy(e);
    if (h2d) cudaStreamDestroy(h2d);
    if (d2h) cudaStreamDestroy(d2h);
  };
  auto go = [&]() -> slso_status {
    SLSO_CHECK_CUDA(cudaStreamCreateWithFlags(&h2d, cudaStreamNonBlocking));
    SLSO_CHECK_CUDA(cudaStreamCreateWithFlags(&d2h, cudaStreamNonBlocking));
    for (cudaEvent_t& e : ev) SLSO_CHECK_CUDA(cudaEventCreateWithFlags(&e, cudaEventDisableTiming));
    cudaEvent_t start = ev[0], *xready = ev + 1, *xfree = ev + 3, *oready = ev + 5, *ofree = ev + 7;
    // the copies may not start before earlier work on the caller's stream (it may use the pool)
    SLSO_CHECK_CUDA(cudaEventRecord(start, st));
    SLSO_CHECK_CUDA(cudaStreamWaitEvent(h2d, start, 0));
    SLSO_CHECK_CUDA(cudaStreamWaitEvent(d2h, start, 0));
    auto copy_in = [&](int64_t i) -> slso_status {
      const int b = static_cast<int>(i & 1);
      if (ldx == d) SLSO_CHECK_CUDA(cudaMemcpyAsync(Xd[b], X_host[i], xbytes, cudaMemcpyHostToDevice, h2d));
      else
        SLSO_CHECK_CUDA(cudaMemcpy2DAsync(Xd[b], d * esz, X_host[i], ldx * esz, d * esz, n, cudaMemcpyHostToDevice, h2d));
      SLSO_CHECK_CUDA(cudaEventRecord(xready[b], h2d));
      return SLSO_OK;
    };
    SLSO_TRY(copy_in(0));
    if (count > 1) SLSO_TRY(copy_in(1));
    for (int64_t i = 0; i < count; ++i) {
      const int b = static_cast<int>(i & 1);
      SLSO_CHECK_CUDA(cudaStreamWaitEvent(st, xready[b], 0));
      if (i >= 2) SLSO_CHECK_CUDA(cudaStreamWaitEvent(st, ofree[b], 0));
      SLSO_CHECK_CUDA(cudaMemsetAsync(h->state, 0, sizeof(DevState), st));
      Arena sub(h->pool + scratch_off, h->pool_cap - scratch_off, false);
      SLSO_TRY(item(sub, b));
      if (sub.overflow()) return fail(SLSO_ERR_OOM, "internal: scratch plan overflowed the pool");
      SLSO_CHECK_CUDA(cudaMemcpyAsync(states + i, h->state, sizeof(DevState), cudaMemcpyDeviceToDevice, st));
      SLSO_CHECK_CUDA(cudaEventRecord(xfree[b], st));
      SLSO_CHECK_CUDA(cudaEventRecord(oready[b], st));
      if (i + 2 < count) {
        SLSO_CHECK_CUDA(cudaStreamWaitEvent(h2d, xfree[b], 0));
        SLSO_TRY(copy_in(i + 2));
      }
      SLSO_CHECK_CUDA(cudaStreamWaitEvent(d2h, oready[b], 0));
      SLSO_CHECK_CUDA(cudaMemcpyAsync(scores_host[i], sc[b], static_cast<size_t>(n) * ssz, cudaMemcpyDeviceToHost, d2h));
      SLSO_CHECK_CUDA(cudaMemcpyAsync(order_host[i], od[b], static_cast<size_t>(n) * sizeof(int64_t),
                                      cudaMemcpyDeviceToHost, d2h));
      SLSO_CHECK_CUDA(cudaEventRecord(ofree[b], d2h));
    }
    // the caller's stream completes after the last copy out
    SLSO_CHECK_CUDA(cudaEventRecord(start, d2h));
    SLSO_CHECK_CUDA(cudaStreamWaitEvent(st, start, 0));
    SLSO_CHECK_CUDA(cudaStreamSynchronize(st));
    std::vector<DevState> hs(static_cast<size_t>(count));
    SLSO_CHECK_CUDA(cudaMemcpy(hs.data(), states, sizeof(DevState) * count, cudaMemcpyDeviceToHost));
    slso_status first_err = SLSO_OK;
    for (int64_t i = 0; i < count; ++i) {
      const DevState& ds = hs[static_cast<size_t>(i)];
      if (info) info_from_state(ds, info + i);
      if (first_err == SLSO_OK && ds.timeout)
        first_err = fail(SLSO_ERR_TIMEOUT, "item %lld: a bounded device wait gave up (kernel %d)", (long long)i, ds.timeout);
      if (first_err == SLSO_OK && ds.nonfinite)
        first_err = fail(SLSO_ERR_NONFINITE, "item %lld: X holds NaN or Inf", (long long)i);
    }
    return first_err;
  };
  const slso_status r = go();
  if (r != SLSO_OK) {  // nothing issued may still use the pool, the host buffers or the events
    cudaStreamSynchronize(st);
    if (h2d) cudaStreamSynchronize(h2d);
    if (d2h) cudaStreamSynchronize(d2h);
  }
  cleanup();
  return r;
}

// Out-of-core X: two passes over blocks of rows copied from the host (see include/slso.h).
// Device layout: fixed buffers (two blocks, SX, the SRHT sample, scores and order of all n rows),
// then one scratch region R reused by every phase: the SRHT sample draw, each block's sketch, the
// solve (whose M stays at the start of R during pass 2), each block's scores after it, and the
// final score sum and ordering.
extern "C" slso_status slso_rank_rows_streamed(slso_handle* handle, const void* X_host, int64_t n, int64_t d,
                                               int64_t ldx, int32_t xdt, const slso_params* params,
                                               int64_t block_rows, void* scores_host, int64_t* order_host,
                                               slso_info* info, void* stream) {
  Handle* h = nullptr;
  SLSO_TRY(check_handle(handle, &h));
  SLSO_TRY(check_x(X_host, n, d, ldx, xdt));
  SLSO_TRY(check_params(params, n, d));
  if (!scores_host || !order_host) return fail(SLSO_ERR_INVALID_ARG, "scores_host and order_host must be non-NULL");
  if (params->correct_frac != 0.0)
    return fail(SLSO_ERR_INVALID_ARG, "correct_frac must be 0 for the streamed entry point");
  if (block_rows < 0) return fail(SLSO_ERR_INVALID_ARG, "block_rows must be >= 0");
  int64_t B = block_rows > 0 ? std::max<int64_t>(block_rows, kStreamMinBlock) : kStreamDefaultBlock;
  while (B & (B - 1)) B &= B - 1;  // round down to a power of two
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  const int64_t nb = ceil_div(n, B);
  const int64_t Bm = std::min(B, n);
  const size_t esz = dtype_size(xdt);
  const int32_t sdt = params->compute == SLSO_F64 ? SLSO_F64 : SLSO_F32;
  const size_t ssz = dtype_size(sdt);
  const size_t xbytes = static_cast<size_t>(Bm) * d * esz;
  const double tau = params->tau < 0 ? default_tau(params->s, d) : params->tau;
  const int64_t kk = params->k > 0 ? params->k : d;
  auto rows_of = [&](int64_t b) { return std::min(B, n - b * B); };

  char* Xb[2] = {};
  double* SX = nullptr;
  uint32_t* sample = nullptr;
  char* scd = nullptr;
  int64_t* odd = nullptr;
  auto take_fixed = [&](Arena& ar) {
    Xb[0] = ar.take<char>(xbytes);
    Xb[1] = nb > 1 ? ar.take<char>(xbytes) : nullptr;
    SX = ar.take<double>(static_cast<size_t>(params->s) * d);
    sample = params->kind == SLSO_SRHT ? ar.take<uint32_t>(params->s) : nullptr;
    scd = ar.take<char>(static_cast<size_t>(n) * ssz);
    odd = ar.take<int64_t>(n);
  };
  SketchBlock blk{};
  blk.n_total = n;
  SolveOut so;
  auto draw_sample = [&](Arena& ar) -> slso_status {
    if (params->kind != SLSO_SRHT) return SLSO_OK;
    const uint32_t* rows = nullptr;
    SLSO_TRY(srht_sample_rows(*h, ar, n, params->s, params->seed_S, &rows, st));
    if (!ar.measure())
      SLSO_CHECK_CUDA(cudaMemcpyAsync(sample, rows, sizeof(uint32_t) * params->s, cudaMemcpyDeviceToDevice, st));
    return SLSO_OK;
  };
  auto sketch_block = [&](Arena& ar, int64_t b) -> slso_status {
    blk.row0 = b * B;
    blk.accumulate = b > 0;
    blk.srht_rows = sample;
    prof_begin(*h, ar, ST_SKETCH, st);
    SLSO_TRY(run_sketch(*h, ar, Xb[b & 1], rows_of(b), d, d, xdt, params->kind, params->s, params->seed_S,
                        params->nnz, SX, st, &blk));
    prof_end(*h, ar, st);
    return SLSO_OK;
  };
  auto solve = [&](Arena& ar) {
    return run_solve(*h, ar, SX, params->s, d, tau, params->k, params->seed_Pi, 0, &so, st, use_gram(params));
  };
  auto score_block = [&](Arena& ar, int64_t b) -> slso_status {
    prof_begin(*h, ar, ST_SCORES, st);
    SLSO_TRY(run_scores(*h, ar, Xb[b & 1], rows_of(b), d, d, xdt, so.M, kk, params->compute,
                        scd + static_cast<size_t>(b * B) * ssz, 0.0, st));
    prof_end(*h, ar, st);
    return SLSO_OK;
  };
  auto finish = [&](Arena& ar) -> slso_status {
    SLSO_TRY(score_sum(*h, ar, scd, sdt, n, st));
    prof_begin(*h, ar, ST_ORDER, st);
    SLSO_TRY(order_scores(*h, ar, scd, sdt, n, odd, st));
    prof_end(*h, ar, st);
    return SLSO_OK;
  };

  // footprint: fixed + max(sample, block sketch, solve + block scores, finish), blocks of Bm rows
  auto aligned = [](size_t v) { return (v + 255) & ~size_t(255); };
  Arena mf(nullptr, ~size_t(0), true);
  take_fixed(mf);
  const size_t off_R = aligned(mf.used());
  size_t need = 0, solve_used = 0;
  {
    Arena m0(nullptr, ~size_t(0), true);
    SLSO_TRY(draw_sample(m0));
    need = std::max(need, m0.used());
    Arena m1(nullptr, ~size_t(0), true);
    SLSO_TRY(sketch_block(m1, 0));
    need = std::max(need, m1.used());
    Arena m2(nullptr, ~size_t(0), true);
    SLSO_TRY(solve(m2));
    solve_used = aligned(m2.used());
    Arena m3(nullptr, ~size_t(0), true);
    SLSO_TRY(score_block(m3, 0));
    need = std::max(need, solve_used + m3.used());
    Arena m4(nullptr, ~size_t(0), true);
    SLSO_TRY(finish(m4));
    need = std::max(need, m4.used());
  }
  SLSO_TRY(ensure_pool(*h, off_R + need));
  Arena real(h->pool, h->pool_cap, false);
  take_fixed(real);
  auto region = [&](size_t off) { return Arena(h->pool + off_R + off, h->pool_cap - off_R - off, false); };

  // steps: pass 1 over blocks 0 .. nb-1, pass 2 over nb-1 .. 0; block b lives in buffer b & 1, so
  // pass 2's first two blocks are still on the device
  struct Step { int pass; int64_t b; };
  std::vector<Step> steps;
  for (int64_t b = 0; b < nb; ++b) steps.push_back({1, b});
  for (int64_t b = nb - 1; b >= 0; --b) steps.push_back({2, b});
  auto needs_load = [&](size_t j) { return steps[j].pass == 1 || steps[j].b < nb - 2; };

  cudaStream_t h2d = nullptr;
  cudaEvent_t ev[5] = {};  // start, xready[2], xfree[2]
  auto go = [&]() -> slso_status {
    SLSO_CHECK_CUDA(cudaStreamCreateWithFlags(&h2d, cudaStreamNonBlocking));
    for (cudaEvent_t& e : ev) SLSO_CHECK_CUDA(cudaEventCreateWithFlags(&e, cudaEventDisableTiming));
    cudaEvent_t start = ev[0], *xready = ev + 1, *xfree = ev + 3;
    SLSO_CHECK_CUDA(cudaMemsetAsync(h->state, 0, sizeof(DevState), st));
    SLSO_CHECK_CUDA(cudaEventRecord(start, st));
    SLSO_CHECK_CUDA(cudaStreamWaitEvent(h2d, start, 0));
    auto copy_in = [&](size_t j) -> slso_status {
      const int64_t b = steps[j].b;
      const char* src = static_cast<const char*>(X_host) + static_cast<size_t>(b * B) * ldx * esz;
      if (ldx == d)
        SLSO_CHECK_CUDA(cudaMemcpyAsync(Xb[b & 1], src, static_cast<size_t>(rows_of(b)) * d * esz,
                                        cudaMemcpyHostToDevice, h2d));
      else
        SLSO_CHECK_CUDA(cudaMemcpy2DAsync(Xb[b & 1], d * esz, src, ldx * esz, d * esz, rows_of(b),
                                          cudaMemcpyHostToDevice, h2d));
      SLSO_CHECK_CUDA(cudaEventRecord(xready[b & 1], h2d));
      return SLSO_OK;
    };
    {
      Arena r = region(0);
      SLSO_TRY(draw_sample(r));
    }
    for (size_t j = 0; j < 2 && j < steps.size(); ++j)
      if (needs_load(j)) SLSO_TRY(copy_in(j));
    for (size_t j = 0; j < steps.size(); ++j) {
      const int64_t b = steps[j].b;
      if (needs_load(j)) SLSO_CHECK_CUDA(cudaStreamWaitEvent(st, xready[b & 1], 0));
      if (steps[j].pass == 1) {
        Arena r = region(0);
        SLSO_TRY(sketch_block(r, b));
        if (r.overflow()) return fail(SLSO_ERR_OOM, "internal: scratch plan overflowed the pool");
      } else {
        if (j == static_cast<size_t>(nb)) {
          Arena r = region(0);
          SLSO_TRY(solve(r));
          if (r.overflow()) return fail(SLSO_ERR_OOM, "internal: scratch plan overflowed the pool");
        }
        Arena r = region(solve_used);
        SLSO_TRY(score_block(r, b));
        if (r.overflow()) return fail(SLSO_ERR_OOM, "internal: scratch plan overflowed the pool");
      }
      SLSO_CHECK_CUDA(cudaEventRecord(xfree[b & 1], st));
      if (j + 2 < steps.size() && needs_load(j + 2)) {
        SLSO_CHECK_CUDA(cudaStreamWaitEvent(h2d, xfree[steps[j + 2].b & 1], 0));
        SLSO_TRY(copy_in(j + 2));
      }
    }
    {
      Arena r = region(0);
      SLSO_TRY(finish(r));
      if (r.overflow()) return fail(SLSO_ERR_OOM, "internal: scratch plan overflowed the pool");
    }
    prof_begin(*h, real, ST_COPY, st);
    SLSO_CHECK_CUDA(cudaMemcpyAsync(scores_host, scd, static_cast<size_t>(n) * ssz, cudaMemcpyDeviceToHost, st));
    SLSO_CHECK_CUDA(cudaMemcpyAsync(order_host, odd, static_cast<size_t>(n) * sizeof(int64_t), cudaMemcpyDeviceToHost, st));
    prof_end(*h, real, st);
    slso_info tmp{};
    return fill_info(*h, st, info ? info : &tmp);
  };
  const slso_status r = go();
  if (r != SLSO_OK) {  // nothing issued may still use the pool, the host buffer or the events
    cudaStreamSynchronize(st);
    if (h2d) cudaStreamSynchronize(h2d);
  }
  for (cudaEvent_t e : ev)
    if (e) cudaEventDestroy(e);
  if (h2d) cudaStreamDestroy(h2d);
  return r;
}

extern "C" slso_status slso_sample_order(slso_handle* handle, const void* scores, int32_t sdt, int64_t n,
                                         int32_t policy, uint64_t seed, int64_t* order, void* stream) {
  Handle* h = nullptr;
  SLSO_TRY(check_handle(handle, &h));
  if (!scores || !order) return fail(SLSO_ERR_INVALID_ARG, "scores and order must be non-NULL");
  if (n < 1 || n >= (int64_t(1) << 31)) return fail(SLSO_ERR_SHAPE, "need 1 <= n < 2^31");
  if (sdt != SLSO_F32 && sdt != SLSO_F64) return fail(SLSO_ERR_DTYPE, "scores must be F32 or F64");
  if (policy != SLSO_POLICY_DEC && policy != SLSO_POLICY_SWR && policy != SLSO_POLICY_SWOR)
    return fail(SLSO_ERR_INVALID_ARG, "unknown sampling policy %d", policy);
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  return run_plan(*h, [&](Arena& ar) {
    prof_begin(*h, ar, ST_ORDER, st);
    SLSO_TRY(sample_order(*h, ar, scores, sdt, n, policy, seed, order, st));
    prof_end(*h, ar, st);
    return SLSO_OK;
  });
}

extern "C" slso_status slso_rank_rows_host(slso_handle* handle, const void* X_host, int64_t n, int64_t d,
                                           int64_t ldx, int32_t xdt, const slso_params* params,
                                           void* scores_host, int64_t* order_host, slso_info* info,
                                           void* stream) {
  Handle* h = nullptr;
  SLSO_TRY(check_handle(handle, &h));
  SLSO_TRY(check_x(X_host, n, d, ldx, xdt));
  SLSO_TRY(check_params(params, n, d));
  if (!scores_host || !order_host) return fail(SLSO_ERR_INVALID_ARG, "scores_host and order_host must be non-NULL");
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  const size_t esz = dtype_size(xdt);
  const int32_t sdt = params->compute == SLSO_F64 ? SLSO_F64 : SLSO_F32;
  const size_t ssz = dtype_size(sdt);
  char* Xd = nullptr;
  void* sc = nullptr;
  int64_t* od = nullptr;
  SLSO_CHECK_CUDA(cudaMemsetAsync(h->state, 0, sizeof(DevState), st));
  SLSO_TRY(run_plan(*h, [&](Arena& ar) {
    Xd = ar.take<char>(static_cast<size_t>(n) * d * esz);
    sc = ar.take<char>(static_cast<size_t>(n) * ssz);
    od = ar.take<int64_t>(n);
    prof_begin(*h, ar, ST_COPY, st);
    if (!ar.measure()) {
      if (ldx == d) {
        SLSO_CHECK_CUDA(cudaMemcpyAsync(Xd, X_host, static_cast<size_t>(n) * d * esz, cudaMemcpyHostToDevice, st));
      } else {
        SLSO_CHECK_CUDA(cudaMemcpy2DAsync(Xd, d * esz, X_host, ldx * esz, d * esz, n, cudaMemcpyHostToDevice, st));
      }
    }
    prof_end(*h, ar, st);
    SLSO_TRY(leverage_plan(*h, ar, Xd, n, d, d, xdt, params, sc, st));
    prof_begin(*h, ar, ST_ORDER, st);
    SLSO_TRY(order_scores(*h, ar, sc, sdt, n, od, st));
    prof_end(*h, ar, st);
    prof_begin(*h, ar, ST_COPY, st);
    if (!ar.measure()) {
      SLSO_CHECK_CUDA(cudaMemcpyAsync(scores_host, sc, static_cast<size_t>(n) * ssz, cudaMemcpyDeviceToHost, st));
      SLSO_CHECK_CUDA(cudaMemcpyAsync(order_host, od, static_cast<size_t>(n) * sizeof(int64_t), cudaMemcpyDeviceToHost, st));
    }
    prof_end(*h, ar, st);
    return SLSO_OK;
  }));
  if (info) return fill_info(*h, st, info);
  SLSO_CHECK_CUDA(cudaStreamSynchronize(st));
  return SLSO_OK;
}
