// slso_selftest_wait: runs one of the library's bounded device-side waits on something that is
// never signalled, so that the timeout path (error word in DevState, SLSO_ERR_TIMEOUT on the
// host, context still usable) can be tested without faulting or hanging a GPU.
#include "common.cuh"
#include "tc.cuh"

namespace slso {
namespace {

constexpr int32_t kTimeoutSelftestFlag = 9, kTimeoutSelftestMbar = 10;

// The QR's ready-flag wait (polls with a 64 ns sleep) on a flag nothing sets.
__global__ void selftest_flag_kernel(const int* flag, long long polls, DevState* state) {
  if (threadIdx.x == 0 && !wait_flag_geq(reinterpret_cast<const volatile int*>(flag), 1, polls))
    atomicExch(&state->timeout, kTimeoutSelftestFlag);
}

// The tensor-core kernels' mbarrier wait (bounded by %globaltimer) on a barrier nobody arrives on.
__global__ void selftest_mbar_kernel(unsigned long long limit_ns, DevState* state) {
  __shared__ __align__(8) uint64_t bar;
  if (threadIdx.x == 0) {
    tc::mbar_init(&bar, 1);
    tc::fence_mbar_init();
  }
  __syncthreads();
  if (threadIdx.x == 0 && !tc::mbar_wait(&bar, 0u, nullptr, limit_ns)) atomicExch(&state->timeout, kTimeoutSelftestMbar);
}

}  // namespace
}  // namespace slso

using namespace slso;

extern "C" slso_status slso_selftest_wait(slso_handle* handle, int32_t what, int64_t limit_us, void* stream) {
  Handle* h = nullptr;
  SLSO_TRY(check_handle(handle, &h));
  if (what != 0 && what != 1) return fail(SLSO_ERR_INVALID_ARG, "what must be 0 (flag) or 1 (mbarrier)");
  if (limit_us < 1 || limit_us > 10000000) return fail(SLSO_ERR_INVALID_ARG, "limit_us must be in 1 .. 10^7");
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  SLSO_TRY(ensure_pool(*h, 256));
  int* flag = reinterpret_cast<int*>(h->pool);
  SLSO_CHECK_CUDA(cudaMemsetAsync(h->state, 0, sizeof(DevState), st));
  if (what == 0) {
    SLSO_CHECK_CUDA(cudaMemsetAsync(flag, 0, sizeof(int), st));
    const long long polls = limit_us * 1000 / 64 + 1;  // every poll sleeps at least 64 ns
    selftest_flag_kernel<<<1, 32, 0, st>>>(flag, polls, h->state);
  } else {
    selftest_mbar_kernel<<<1, 32, 0, st>>>(static_cast<unsigned long long>(limit_us) * 1000ull, h->state);
  }
  SLSO_CHECK_LAUNCH();
  SLSO_CHECK_CUDA(cudaMemcpyAsync(h->state_host, h->state, sizeof(DevState), cudaMemcpyDeviceToHost, st));
  SLSO_CHECK_CUDA(cudaStreamSynchronize(st));
  if (h->state_host->timeout)
    return fail(SLSO_ERR_TIMEOUT, "a bounded device wait gave up (self-test %d)", h->state_host->timeout);
  return SLSO_OK;
}
