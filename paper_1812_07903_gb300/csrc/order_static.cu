// slso_order_static: the "dec" ordering for callers that cannot allocate device memory.
//
// Some callers have no way to call cudaMalloc at the point where they need an ordering: code
// that runs while another framework owns every byte of device memory through its own caching
// allocator, services that forbid allocation after start-up so their memory footprint and
// latency stay fixed, and code that is being recorded into a CUDA graph by someone else.  This
// entry point needs neither a handle nor any allocation: its scratch (radix-sort key and value
// double buffers and digit histograms) lives in one file-scope __device__ array sized for
// n <= 2^20 scores (about 24.3 MB, held by every GPU that loads the library until the process
// exits).  It runs the same kernels as slso_order.
#include <mutex>

#include "common.cuh"

namespace slso {
namespace {

constexpr int64_t kStaticMaxN = int64_t(1) << 20;
// keys + alternate keys (8 bytes each for float64 scores), values + alternate values (4 bytes
// each), 256 digit counts per 4096-key tile, the 256 digit totals, plus 256-byte alignment of
// each piece.
constexpr size_t kStaticBytes = size_t(kStaticMaxN) * (8 + 8 + 4 + 4) + size_t(256) * (kStaticMaxN / 4096) * 4 +
                                size_t(256) * 4 + size_t(16) * 256;

__device__ __align__(256) unsigned char g_order_scratch[kStaticBytes];

constexpr int kMaxDevices = 64;
std::mutex g_mutex;
void* g_scratch[kMaxDevices] = {};
int g_sms[kMaxDevices] = {};

// Device address of the scratch array on the current device, looked up once per device.  In host
// code the array's name is only a host-side stand-in, so the address comes from
// cudaGetSymbolAddress with that device current.
slso_status static_scratch(int dev, void** ptr, int* sms) {
  std::lock_guard<std::mutex> lock(g_mutex);
  if (!g_scratch[dev]) {
    void* p = nullptr;
    SLSO_CHECK_CUDA(cudaGetSymbolAddress(&p, g_order_scratch));
    int count = 0;
    SLSO_CHECK_CUDA(cudaDeviceGetAttribute(&count, cudaDevAttrMultiProcessorCount, dev));
    g_scratch[dev] = p;
    g_sms[dev] = count;
  }
  *ptr = g_scratch[dev];
  *sms = g_sms[dev];
  return SLSO_OK;
}

}  // namespace
}  // namespace slso

using namespace slso;

extern "C" slso_status slso_order_static(const void* scores, int32_t sdt, int64_t n, int64_t* order,
                                         void* stream) {
  if (!scores || !order) return fail(SLSO_ERR_INVALID_ARG, "scores and order must be non-NULL");
  if (sdt != SLSO_F32 && sdt != SLSO_F64) return fail(SLSO_ERR_DTYPE, "scores must be F32 or F64");
  if (n < 1 || n > kStaticMaxN)
    return fail(SLSO_ERR_SHAPE, "slso_order_static handles 1 <= n <= %lld scores (n=%lld); use slso_order",
                (long long)kStaticMaxN, (long long)n);
  int dev = 0;
  SLSO_CHECK_CUDA(cudaGetDevice(&dev));
  if (dev < 0 || dev >= kMaxDevices) return fail(SLSO_ERR_INVALID_ARG, "device %d out of range", dev);
  void* base = nullptr;
  int sms = 0;
  SLSO_TRY(static_scratch(dev, &base, &sms));
  Handle h;  // describes the device only: no pool, no state, nothing allocated
  h.device = dev;
  h.num_sms = sms;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  Arena m(nullptr, ~size_t(0), true);
  SLSO_TRY(order_scores(h, m, scores, sdt, n, order, st));
  if (m.used() > kStaticBytes) return fail(SLSO_ERR_SHAPE, "internal: static scratch too small");
  Arena real(static_cast<char*>(base), kStaticBytes, false);
  return order_scores(h, real, scores, sdt, n, order, st);
}
