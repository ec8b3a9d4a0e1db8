// Handle, device pool and error reporting of libslso.
#include <atomic>
#include <map>
#include <mutex>
#include <utility>
#include <cstdarg>
#include <cstdio>
#include <cstring>

#include "common.cuh"

namespace slso {

static thread_local char g_last_error[1024] = "";
static std::atomic<long long> g_launches{0};

void note_launch() { g_launches.fetch_add(1, std::memory_order_relaxed); }

void prof_begin(Handle& h, const Arena& ar, int stage, cudaStream_t st) {
  if (!h.prof || ar.measure() || h.nrec >= kProfCap) return;
  ProfRecord& r = h.recs[h.nrec];
  if (!r.a) {
    cudaEventCreate(&r.a);
    cudaEventCreate(&r.b);
  }
  r.stage = stage;
  cudaEventRecord(r.a, st);
  h.open_rec = h.nrec++;
}

void prof_end(Handle& h, const Arena& ar, cudaStream_t st) {
  if (!h.prof || ar.measure() || h.open_rec < 0) return;
  cudaEventRecord(h.recs[h.open_rec].b, st);
  h.open_rec = -1;
}

slso_status fail(slso_status st, const char* fmt, ...) {
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(g_last_error, sizeof(g_last_error), fmt, ap);
  va_end(ap);
  return st;
}

slso_status raise_smem_limit(const void* fn, size_t bytes) {
  static std::mutex mu;
  static std::map<std::pair<int, const void*>, size_t> limits;
  int dev = 0;
  SLSO_CHECK_CUDA(cudaGetDevice(&dev));
  std::lock_guard<std::mutex> lock(mu);
  auto key = std::make_pair(dev, fn);
  auto it = limits.find(key);
  if (it == limits.end()) {
    // A function starts with a dynamic limit of 48 KB minus its own static __shared__ bytes, so
    // the starting value is read from the function, not assumed.
    cudaFuncAttributes a{};
    SLSO_CHECK_CUDA(cudaFuncGetAttributes(&a, fn));
    it = limits.emplace(key, static_cast<size_t>(a.maxDynamicSharedSizeBytes)).first;
  }
  size_t& cur = it->second;
  if (bytes <= cur) return SLSO_OK;
  SLSO_CHECK_CUDA(cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, static_cast<int>(bytes)));
  cur = bytes;
  return SLSO_OK;
}

slso_status ensure_pool(Handle& h, size_t bytes) {
  if (bytes <= h.pool_cap) return SLSO_OK;
  if (h.pool_limit && bytes > h.pool_limit)
    return fail(SLSO_ERR_OOM, "scratch of %zu bytes exceeds the pool limit of %zu bytes", bytes, h.pool_limit);
  // Growing frees the old block; cudaFree waits for work in flight on the device.
  if (h.pool) {
    SLSO_CHECK_CUDA(cudaFree(h.pool));
    h.pool = nullptr;
    h.pool_cap = 0;
  }
  const size_t cap = (bytes + (size_t(2) << 20) - 1) & ~((size_t(2) << 20) - 1);
  cudaError_t e = cudaMalloc(reinterpret_cast<void**>(&h.pool), cap);
  if (e != cudaSuccess) {
    cudaGetLastError();
    h.pool = nullptr;
    return fail(SLSO_ERR_OOM, "device pool of %zu bytes could not be allocated: %s", cap,
                cudaGetErrorString(e));
  }
  h.pool_cap = cap;
  return SLSO_OK;
}

slso_status check_handle(slso_handle* hp, Handle** out) {
  if (!hp) return fail(SLSO_ERR_INVALID_ARG, "handle is NULL");
  Handle* h = reinterpret_cast<Handle*>(hp);
  SLSO_CHECK_CUDA(cudaSetDevice(h->device));
  *out = h;
  return SLSO_OK;
}

}  // namespace slso

using namespace slso;

extern "C" const char* slso_version(void) { return "slso-gb300 0.1 (sm_103a)"; }

extern "C" const char* slso_last_error(void) { return g_last_error; }

namespace slso {

cudaError_t side_stream_create(Handle& h) {
  if (h.side) return cudaSuccess;
  cudaError_t e = cudaStreamCreateWithFlags(&h.side, cudaStreamNonBlocking);
  if (e == cudaSuccess) e = cudaEventCreateWithFlags(&h.ev_fork, cudaEventDisableTiming);
  for (int i = 0; i < 2 && e == cudaSuccess; ++i) {
    e = cudaEventCreateWithFlags(&h.ev_ready[i], cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&h.ev_free[i], cudaEventDisableTiming);
  }
  if (e != cudaSuccess) side_stream_release(h);
  return e;
}

void side_stream_release(Handle& h) {
  if (h.side) cudaStreamDestroy(h.side);
  if (h.ev_fork) cudaEventDestroy(h.ev_fork);
  for (int i = 0; i < 2; ++i) {
    if (h.ev_ready[i]) cudaEventDestroy(h.ev_ready[i]);
    if (h.ev_free[i]) cudaEventDestroy(h.ev_free[i]);
    h.ev_ready[i] = h.ev_free[i] = nullptr;
  }
  h.side = nullptr;
  h.ev_fork = nullptr;
}

}  // namespace slso

extern "C" slso_status slso_create(slso_handle** handle, int device) {
  if (!handle) return fail(SLSO_ERR_INVALID_ARG, "handle out-pointer is NULL");
  *handle = nullptr;
  int count = 0;
  SLSO_CHECK_CUDA(cudaGetDeviceCount(&count));
  if (device < 0 || device >= count)
    return fail(SLSO_ERR_INVALID_ARG, "device %d out of range (%d devices)", device, count);
  SLSO_CHECK_CUDA(cudaSetDevice(device));
  Handle* h = new Handle();
  h->device = device;
  cudaError_t e = cudaDeviceGetAttribute(&h->num_sms, cudaDevAttrMultiProcessorCount, device);
  if (e == cudaSuccess) e = cudaMalloc(reinterpret_cast<void**>(&h->state), sizeof(DevState));
  if (e == cudaSuccess) e = cudaMallocHost(reinterpret_cast<void**>(&h->state_host), sizeof(DevState));
  if (e == cudaSuccess) e = cudaMemset(h->state, 0, sizeof(DevState));
  if (e == cudaSuccess) e = side_stream_create(*h);
  if (e != cudaSuccess) {
    side_stream_release(*h);
    if (h->state) cudaFree(h->state);
    if (h->state_host) cudaFreeHost(h->state_host);
    delete h;
    return fail(SLSO_ERR_CUDA, "slso_create: %s", cudaGetErrorString(e));
  }
  *handle = reinterpret_cast<slso_handle*>(h);
  return SLSO_OK;
}

extern "C" slso_status slso_destroy(slso_handle* handle) {
  if (!handle) return SLSO_OK;
  Handle* h = reinterpret_cast<Handle*>(handle);
  cudaSetDevice(h->device);
  cudaDeviceSynchronize();
  if (h->pool) cudaFree(h->pool);
  if (h->recs) {
    for (int i = 0; i < kProfCap; ++i)
      if (h->recs[i].a) {
        cudaEventDestroy(h->recs[i].a);
        cudaEventDestroy(h->recs[i].b);
      }
    delete[] h->recs;
  }
  side_stream_release(*h);
  if (h->state) cudaFree(h->state);
  if (h->state_host) cudaFreeHost(h->state_host);
  delete h;
  return SLSO_OK;
}

extern "C" slso_status slso_set_pool_limit(slso_handle* handle, size_t bytes) {
  Handle* h = nullptr;
  SLSO_TRY(check_handle(handle, &h));
  h->pool_limit = bytes;
  return SLSO_OK;
}

extern "C" slso_status slso_set_score_form(slso_handle* handle, int32_t form) {
  Handle* h = nullptr;
  SLSO_TRY(check_handle(handle, &h));
  if (form < SLSO_SCORE_FORM_MIXED || form > SLSO_SCORE_FORM_TF32X3_SMEM)
    return fail(SLSO_ERR_INVALID_ARG, "unknown score form");
  h->score_form = form;
  return SLSO_OK;
}

extern "C" slso_status slso_profile(slso_handle* handle, int enable) {
  Handle* h = nullptr;
  SLSO_TRY(check_handle(handle, &h));
  if (!h->recs) {
    h->recs = new ProfRecord[kProfCap];
    for (int i = 0; i < kProfCap; ++i) h->recs[i] = ProfRecord{0, nullptr, nullptr};
  }
  h->prof = enable != 0;
  h->nrec = 0;
  h->open_rec = -1;
  h->launches_at_enable = g_launches.load();
  return SLSO_OK;
}

extern "C" slso_status slso_profile_read(slso_handle* handle, double* stage_ms, int64_t* stage_calls,
                                         int64_t* launches) {
  Handle* h = nullptr;
  SLSO_TRY(check_handle(handle, &h));
  if (!stage_ms || !stage_calls || !launches) return fail(SLSO_ERR_INVALID_ARG, "NULL output");
  for (int i = 0; i < SLSO_STAGES; ++i) {
    stage_ms[i] = 0.0;
    stage_calls[i] = 0;
  }
  for (int i = 0; i < h->nrec; ++i) {
    const ProfRecord& r = h->recs[i];
    SLSO_CHECK_CUDA(cudaEventSynchronize(r.b));
    float ms = 0.f;
    SLSO_CHECK_CUDA(cudaEventElapsedTime(&ms, r.a, r.b));
    stage_ms[r.stage] += ms;
    stage_calls[r.stage] += 1;
  }
  *launches = g_launches.load() - h->launches_at_enable;
  return SLSO_OK;
}
