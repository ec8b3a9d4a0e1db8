// Sampling policies of Algorithm 4 step 4 (Sec. 5.2) on the GPU: "dec, swor" and "dec, swr"
// from P = l / sum l.
//
//   swor  the order of n successive weighted draws without replacement.  Point i gets the key
//         log(u_i) / l_i (Efraimidis and Spirakis's u^(1/P) on a log scale; P is l times a
//         positive constant), and the existing stable radix argsort orders the float64 keys
//         decreasingly: weight-0 points (key -inf) follow all others in increasing index, NaN
//         scores last.
//   swr   n draws with replacement: the inclusive prefix sums C of the weights (float64, fixed
//         summation order), then draw t = the smallest i with C_i > u_t C_{n-1} (binary search).
//         When no score is positive and finite every draw is -1.
// u_t = (m + 1/2) 2^-52 with m = w0 2^20 + (w1 >> 12) from the Philox block (lo t, hi t, 0, 6).
#include <math_constants.h>

#include <cmath>

#include "common.cuh"

namespace slso {

namespace {

constexpr uint32_t TAG_SAMPLE = 6;
constexpr int kScanThreads = 256;
constexpr int kScanPerThread = 8;
constexpr int kScanChunk = kScanThreads * kScanPerThread;  // elements per scan block

__device__ __forceinline__ double sample_uniform(uint64_t seed, uint64_t t) {
  const U32x4 w = philox(static_cast<uint32_t>(t), static_cast<uint32_t>(t >> 32), 0u, TAG_SAMPLE, seed);
  const uint64_t m = (static_cast<uint64_t>(w.x) << 20) | (w.y >> 12);
  return (static_cast<double>(m) + 0.5) * 0x1p-52;
}

template <typename T>
__device__ __forceinline__ double sampling_weight(T v) {
  const double x = static_cast<double>(v);
  return (isfinite(x) && x > 0.0) ? x : 0.0;
}

template <typename T>
__global__ void swor_keys_kernel(const T* __restrict__ scores, int64_t n, uint64_t seed, double* __restrict__ keys) {
  for (int64_t i = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; i < n;
       i += static_cast<int64_t>(gridDim.x) * blockDim.x) {
    const double x = static_cast<double>(scores[i]);
    const double w = sampling_weight(scores[i]);
    double key = (w > 0.0) ? log(sample_uniform(seed, static_cast<uint64_t>(i))) / w : -CUDART_INF;
    if (isnan(x)) key = CUDART_NAN;
    keys[i] = key;
  }
}

// Inclusive block scan of 256 values (one per thread), warp shuffles then warp totals.
__device__ __forceinline__ double block_incl_scan(double v, double* warp_tot) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const double y = __shfl_up_sync(0xFFFFFFFFu, v, o);
    if (lane >= o) v += y;
  }
  if (lane == 31) warp_tot[warp] = v;
  __syncthreads();
  double off = 0.0;
  for (int w = 0; w < warp; ++w) off += warp_tot[w];
  __syncthreads();
  return v + off;
}

// Phase 1: per-chunk totals (thread sums of 8 consecutive weights, then the block scan's total).
template <typename T>
__global__ void __launch_bounds__(kScanThreads) scan_partials_kernel(const T* __restrict__ scores, int64_t n,
                                                                      double* __restrict__ part) {
  __shared__ double warp_tot[kScanThreads / 32];
  const int64_t base = static_cast<int64_t>(blockIdx.x) * kScanChunk + static_cast<int64_t>(threadIdx.x) * kScanPerThread;
  double t = 0.0;
#pragma unroll
  for (int e = 0; e < kScanPerThread; ++e)
    if (base + e < n) t += sampling_weight(scores[base + e]);
  const double incl = block_incl_scan(t, warp_tot);
  if (threadIdx.x == kScanThreads - 1) part[blockIdx.x] = incl;
}

// Phase 2: exclusive offsets of the chunks, summed in order by one thread (<= 2^20 chunks).
__global__ void scan_offsets_kernel(double* __restrict__ part, int64_t nblocks) {
  double acc = 0.0;
  for (int64_t b = 0; b < nblocks; ++b) {
    const double v = part[b];
    part[b] = acc;
    acc += v;
  }
}

// Phase 3: C_i for every element, in the same summation order as phase 1.
template <typename T>
__global__ void __launch_bounds__(kScanThreads) scan_final_kernel(const T* __restrict__ scores, int64_t n,
                                                                   const double* __restrict__ part,
                                                                   double* __restrict__ C) {
  __shared__ double warp_tot[kScanThreads / 32];
  const int64_t base = static_cast<int64_t>(blockIdx.x) * kScanChunk + static_cast<int64_t>(threadIdx.x) * kScanPerThread;
  double w[kScanPerThread];
  double t = 0.0;
#pragma unroll
  for (int e = 0; e < kScanPerThread; ++e) {
    w[e] = (base + e < n) ? sampling_weight(scores[base + e]) : 0.0;
    t += w[e];
  }
  const double incl = block_incl_scan(t, warp_tot);
  double run = part[blockIdx.x] + (incl - t);  // offset of this thread's first element
#pragma unroll
  for (int e = 0; e < kScanPerThread; ++e) {
    run += w[e];
    if (base + e < n) C[base + e] = run;
  }
}

__global__ void swr_draw_kernel(const double* __restrict__ C, int64_t n, uint64_t seed, int64_t* __restrict__ order) {
  const double total = C[n - 1];
  const bool ok = isfinite(total) && total > 0.0;
  for (int64_t t = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; t < n;
       t += static_cast<int64_t>(gridDim.x) * blockDim.x) {
    if (!ok) {
      order[t] = -1;
      continue;
    }
    const double target = sample_uniform(seed, static_cast<uint64_t>(t)) * total;
    int64_t lo = 0, hi = n - 1;  // smallest i with C[i] > target; C[n-1] = total > target
    while (lo < hi) {
      const int64_t mid = lo + ((hi - lo) >> 1);
      if (C[mid] > target) hi = mid;
      else lo = mid + 1;
    }
    order[t] = lo;
  }
}

template <typename T>
slso_status swr(Handle& h, Arena& ar, const T* scores, int64_t n, uint64_t seed, int64_t* order, cudaStream_t st) {
  const int64_t nb = ceil_div(n, kScanChunk);
  double* part = ar.take<double>(nb);
  double* C = ar.take<double>(n);
  if (ar.measure()) return SLSO_OK;
  scan_partials_kernel<T><<<static_cast<unsigned>(nb), kScanThreads, 0, st>>>(scores, n, part);
  SLSO_CHECK_LAUNCH();
  scan_offsets_kernel<<<1, 1, 0, st>>>(part, nb);
  SLSO_CHECK_LAUNCH();
  scan_final_kernel<T><<<static_cast<unsigned>(nb), kScanThreads, 0, st>>>(scores, n, part, C);
  SLSO_CHECK_LAUNCH();
  const unsigned g = static_cast<unsigned>(std::min<int64_t>(ceil_div(n, 256), int64_t(h.num_sms) * 8));
  swr_draw_kernel<<<g, 256, 0, st>>>(C, n, seed, order);
  SLSO_CHECK_LAUNCH();
  return SLSO_OK;
}

template <typename T>
slso_status swor(Handle& h, Arena& ar, const T* scores, int64_t n, uint64_t seed, int64_t* order, cudaStream_t st) {
  double* keys = ar.take<double>(n);
  if (!ar.measure()) {
    const unsigned g = static_cast<unsigned>(std::min<int64_t>(ceil_div(n, 256), int64_t(h.num_sms) * 8));
    swor_keys_kernel<T><<<g, 256, 0, st>>>(scores, n, seed, keys);
    SLSO_CHECK_LAUNCH();
  }
  return order_scores(h, ar, keys, SLSO_F64, n, order, st);
}

}  // namespace

slso_status sample_order(Handle& h, Arena& ar, const void* scores, int32_t sdt, int64_t n, int32_t policy,
                         uint64_t seed, int64_t* order, cudaStream_t st) {
  switch (policy) {
    case SLSO_POLICY_DEC:
      return order_scores(h, ar, scores, sdt, n, order, st);
    case SLSO_POLICY_SWOR:
      if (sdt == SLSO_F32) return swor(h, ar, static_cast<const float*>(scores), n, seed, order, st);
      return swor(h, ar, static_cast<const double*>(scores), n, seed, order, st);
    case SLSO_POLICY_SWR:
      if (sdt == SLSO_F32) return swr(h, ar, static_cast<const float*>(scores), n, seed, order, st);
      return swr(h, ar, static_cast<const double*>(scores), n, seed, order, st);
    default:
      return fail(SLSO_ERR_INVALID_ARG, "unknown sampling policy %d", policy);
  }
}

}  // namespace slso
