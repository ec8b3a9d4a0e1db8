// Row scores l_i = ||(X M)_i||^2 (Algorithm 3 steps 4-5): the product X M is never written;
// each tile reduces its squared entries per row in the epilogue.
//
// The tensor-core kernel (score_tc.cu) takes float32 and bfloat16 X whenever k <= 256; this
// SIMT kernel covers the rest (float64, k > 256, unaligned X): CTA tile of 64 rows x 64 columns of Y, K-steps of 16 through shared memory,
// 4x4 outputs per thread.  Per-row partial sums of squares of each 64-column block go to
// part[cb][i]; a second kernel adds the column blocks in ascending order.
//   compute F64: float64 products and sums.
//   compute F32: float32 products and sums.
//   compute BF16: X and M rounded to bfloat16, exact products, float32 sums.
#include <algorithm>
#include <cmath>

#include "common.cuh"

namespace slso {

namespace {

constexpr int kBm = 64, kBn = 64, kBk = 16;

template <class Acc, int ROUND>
__device__ __forceinline__ Acc quantise(Acc v) {
  if constexpr (ROUND == 1) return static_cast<Acc>(__bfloat162float(__float2bfloat16_rn(static_cast<float>(v))));
  return v;
}

template <class T> __device__ __forceinline__ double load_as_double(const T* p) { return static_cast<double>(to_float(*p)); }
template <> __device__ __forceinline__ double load_as_double<double>(const double* p) { return *p; }

// ROUND: 0 none, 1 bfloat16
template <class T, class Acc, int ROUND>
__global__ void __launch_bounds__(256) score_tile_kernel(const T* __restrict__ X, int64_t n, int64_t d,
                                                         int64_t ldx, const Acc* __restrict__ M, int64_t kk,
                                                         Acc* __restrict__ part) {
  __shared__ Acc Xs[kBk][kBm + 1];
  __shared__ Acc Ms[kBk][kBn];
  __shared__ Acc rowsum[kBm][17];
  const int tx = threadIdx.x % 16, ty = threadIdx.x / 16;
  const int64_t r0 = static_cast<int64_t>(blockIdx.x) * kBm, c0 = static_cast<int64_t>(blockIdx.y) * kBn;
  Acc acc[4][4];
#pragma unroll
  for (int a = 0; a < 4; ++a)
#pragma unroll
    for (int b = 0; b < 4; ++b) acc[a][b] = Acc(0);
  for (int64_t k0 = 0; k0 < d; k0 += kBk) {
    for (int t = threadIdx.x; t < kBm * kBk; t += 256) {
      const int rr = t / kBk, kc = t % kBk;
      const int64_t r = r0 + rr, k = k0 + kc;
      Xs[kc][rr] = (r < n && k < d) ? quantise<Acc, ROUND>(static_cast<Acc>(load_as_double(X + r * ldx + k))) : Acc(0);
    }
    for (int t = threadIdx.x; t < kBk * kBn; t += 256) {
      const int kc = t / kBn, cc = t % kBn;
      const int64_t k = k0 + kc, c = c0 + cc;
      Ms[kc][cc] = (k < d && c < kk) ? M[k * kk + c] : Acc(0);
    }
    __syncthreads();
#pragma unroll
    for (int kc = 0; kc < kBk; ++kc) {
      Acc xv[4], mv[4];
#pragma unroll
      for (int a = 0; a < 4; ++a) xv[a] = Xs[kc][ty * 4 + a];
#pragma unroll
      for (int b = 0; b < 4; ++b) mv[b] = Ms[kc][tx * 4 + b];
#pragma unroll
      for (int a = 0; a < 4; ++a)
#pragma unroll
        for (int b = 0; b < 4; ++b) acc[a][b] = fma(xv[a], mv[b], acc[a][b]);
    }
    __syncthreads();
  }
#pragma unroll
  for (int a = 0; a < 4; ++a) {
    Acc sq = Acc(0);
#pragma unroll
    for (int b = 0; b < 4; ++b) sq = fma(acc[a][b], acc[a][b], sq);
    rowsum[ty * 4 + a][tx] = sq;
  }
  __syncthreads();
  if (threadIdx.x < kBm) {
    const int rr = threadIdx.x;
    Acc t = Acc(0);
    for (int q = 0; q < 16; ++q) t += rowsum[rr][q];
    const int64_t r = r0 + rr;
    if (r < n) part[static_cast<int64_t>(blockIdx.y) * n + r] = t;
  }
}

template <class Acc, class Out>
__global__ void score_combine_kernel(const Acc* __restrict__ part, int64_t n, int64_t ncb,
                                     Out* __restrict__ scores) {
  for (int64_t i = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; i < n;
       i += static_cast<int64_t>(gridDim.x) * blockDim.x) {
    Acc t = Acc(0);
    for (int64_t cb = 0; cb < ncb; ++cb) t += part[cb * n + i];
    scores[i] = static_cast<Out>(t);
  }
}

// Sum of the scores (normaliser of P, Algorithm 4 step 3) in two fixed-order stages:
// kSumBlocks contiguous chunks, then one thread adds the chunk sums in order.
constexpr int kSumBlocks = 128;

template <class Out>
__global__ void score_sum_partial_kernel(const Out* __restrict__ scores, int64_t n, double* __restrict__ part) {
  __shared__ double red[32];
  const int64_t chunk = (n + gridDim.x - 1) / gridDim.x;
  const int64_t lo = blockIdx.x * chunk, hi = lo + chunk < n ? lo + chunk : n;
  double p = 0.0;
  for (int64_t i = lo + threadIdx.x; i < hi; i += blockDim.x) p += static_cast<double>(scores[i]);
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) p += __shfl_down_sync(0xFFFFFFFFu, p, o);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = p;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int w = 0; w < static_cast<int>(blockDim.x >> 5); ++w) t += red[w];
    part[blockIdx.x] = t;
  }
}

__global__ void score_sum_final_kernel(const double* __restrict__ part, DevState* __restrict__ st) {
  double t = 0.0;
  for (int b = 0; b < kSumBlocks; ++b) t += part[b];
  st->score_sum = t;
}

template <class Out>
slso_status launch_score_sum(Handle& h, const Out* scores, int64_t n, double* part, cudaStream_t st) {
  score_sum_partial_kernel<Out><<<kSumBlocks, 256, 0, st>>>(scores, n, part);
  SLSO_CHECK_LAUNCH();
  score_sum_final_kernel<<<1, 1, 0, st>>>(part, h.state);
  SLSO_CHECK_LAUNCH();
  return SLSO_OK;
}

// Correction pass: rescore the rows listed in order[0..T) (the top-T rows of the low-precision
// scores) in float32 from the float32 copy of M and overwrite their scores.  CTA = 64 gathered
// rows; the CTA walks all column blocks of M itself, so each row's sum is finished in-CTA.
template <class T>
__global__ void __launch_bounds__(256) rescore_rows_kernel(const T* __restrict__ X, int64_t d, int64_t ldx,
                                                           const float* __restrict__ M, int64_t kk,
                                                           const int64_t* __restrict__ order, int64_t T_rows,
                                                           float* __restrict__ scores) {
  __shared__ float Xs[kBk][kBm + 1];
  __shared__ float Ms[kBk][kBn];
  __shared__ float rowsum[kBm][17];
  __shared__ int64_t rows[kBm];
  const int tx = threadIdx.x % 16, ty = threadIdx.x / 16;
  const int64_t t0 = static_cast<int64_t>(blockIdx.x) * kBm;
  if (threadIdx.x < kBm) rows[threadIdx.x] = (t0 + threadIdx.x < T_rows) ? order[t0 + threadIdx.x] : -1;
  __syncthreads();
  float sq[4] = {0.f, 0.f, 0.f, 0.f};
  for (int64_t c0 = 0; c0 < kk; c0 += kBn) {
    float acc[4][4];
#pragma unroll
    for (int a = 0; a < 4; ++a)
#pragma unroll
      for (int b = 0; b < 4; ++b) acc[a][b] = 0.f;
    for (int64_t k0 = 0; k0 < d; k0 += kBk) {
      for (int t = threadIdx.x; t < kBm * kBk; t += 256) {
        const int rr = t / kBk, kc = t % kBk;
        const int64_t r = rows[rr], k = k0 + kc;
        Xs[kc][rr] = (r >= 0 && k < d) ? static_cast<float>(load_as_double(X + r * ldx + k)) : 0.f;
      }
      for (int t = threadIdx.x; t < kBk * kBn; t += 256) {
        const int kc = t / kBn, cc = t % kBn;
        const int64_t k = k0 + kc, c = c0 + cc;
        Ms[kc][cc] = (k < d && c < kk) ? M[k * kk + c] : 0.f;
      }
      __syncthreads();
#pragma unroll
      for (int kc = 0; kc < kBk; ++kc) {
        float xv[4], mv[4];
#pragma unroll
        for (int a = 0; a < 4; ++a) xv[a] = Xs[kc][ty * 4 + a];
#pragma unroll
        for (int b = 0; b < 4; ++b) mv[b] = Ms[kc][tx * 4 + b];
#pragma unroll
        for (int a = 0; a < 4; ++a)
#pragma unroll
          for (int b = 0; b < 4; ++b) acc[a][b] = fmaf(xv[a], mv[b], acc[a][b]);
      }
      __syncthreads();
    }
#pragma unroll
    for (int a = 0; a < 4; ++a)
#pragma unroll
      for (int b = 0; b < 4; ++b) sq[a] = fmaf(acc[a][b], acc[a][b], sq[a]);
  }
#pragma unroll
  for (int a = 0; a < 4; ++a) rowsum[ty * 4 + a][tx] = sq[a];
  __syncthreads();
  if (threadIdx.x < kBm && rows[threadIdx.x] >= 0) {
    float t = 0.f;
    for (int q = 0; q < 16; ++q) t += rowsum[threadIdx.x][q];
    scores[rows[threadIdx.x]] = t;
  }
}

__global__ void m_to_f32_kernel(const double* __restrict__ M, int64_t e, float* __restrict__ Mf) {
  for (int64_t i = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; i < e;
       i += static_cast<int64_t>(gridDim.x) * blockDim.x)
    Mf[i] = static_cast<float>(M[i]);
}

__global__ void m_to_bf16val_kernel(const double* __restrict__ M, int64_t e, float* __restrict__ Mf) {
  for (int64_t i = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; i < e;
       i += static_cast<int64_t>(gridDim.x) * blockDim.x)
    Mf[i] = __bfloat162float(__float2bfloat16_rn(static_cast<float>(M[i])));
}

int grid1d(int64_t n, const Handle& h) {
  return static_cast<int>(std::max<int64_t>(1, std::min<int64_t>(ceil_div(n, 256), 8LL * h.num_sms)));
}

// Correction pass (BF16 / FP8 compute with correct_frac > 0): order the low-precision scores,
// take the top ceil(frac n) rows and rescore them in float32.
template <class T>
slso_status correct_top_rows(Handle& h, Arena& ar, const T* X, int64_t n, int64_t d, int64_t ldx,
                             const double* M, int64_t kk, int32_t compute, double frac, float* scores,
                             cudaStream_t st) {
  if (!(frac > 0.0) || (compute != SLSO_BF16 && compute != SLSO_FP8_E4M3)) return SLSO_OK;
  const int64_t T_rows = std::min<int64_t>(n, static_cast<int64_t>(std::ceil(frac * static_cast<double>(n))));
  int64_t* order = ar.take<int64_t>(n);
  float* Mf = ar.take<float>(static_cast<size_t>(d) * kk);
  SLSO_TRY(order_scores(h, ar, scores, SLSO_F32, n, order, st));
  if (ar.measure()) return SLSO_OK;
  m_to_f32_kernel<<<grid1d(d * kk, h), 256, 0, st>>>(M, d * kk, Mf);
  SLSO_CHECK_LAUNCH();
  rescore_rows_kernel<T><<<static_cast<unsigned>(ceil_div(T_rows, kBm)), 256, 0, st>>>(X, d, ldx, Mf, kk, order,
                                                                                       T_rows, scores);
  SLSO_CHECK_LAUNCH();
  return SLSO_OK;
}

template <class T>
slso_status scores_typed(Handle& h, Arena& ar, const T* X, int64_t n, int64_t d, int64_t ldx,
                         const double* M, int64_t kk, int32_t compute, double correct_frac, void* scores,
                         cudaStream_t st, const unsigned int* colmax_pre) {
  const int64_t ncb = ceil_div(kk, kBn);
  dim3 grid(static_cast<unsigned>(ceil_div(n, kBm)), static_cast<unsigned>(ncb));
  double* sums = ar.take<double>(kSumBlocks);
  if (compute == SLSO_F64) {
    double* part = ar.take<double>(static_cast<size_t>(ncb) * n);
    if (ar.measure()) return SLSO_OK;
    score_tile_kernel<T, double, 0><<<grid, 256, 0, st>>>(X, n, d, ldx, M, kk, part);
    SLSO_CHECK_LAUNCH();
    score_combine_kernel<double, double><<<grid1d(n, h), 256, 0, st>>>(part, n, ncb, static_cast<double*>(scores));
    SLSO_CHECK_LAUNCH();
    return launch_score_sum<double>(h, static_cast<double*>(scores), n, sums, st);
  }
  bool used_tc = false;
  SLSO_TRY(run_scores_tc(h, ar, X, n, d, ldx, std::is_same<T, float>::value ? SLSO_F32
                                                : (std::is_same<T, double>::value ? SLSO_F64 : SLSO_BF16),
                         M, kk, compute, static_cast<float*>(scores), &used_tc, st, colmax_pre));
  if (used_tc) {
    SLSO_TRY(correct_top_rows(h, ar, X, n, d, ldx, M, kk, compute, correct_frac, static_cast<float*>(scores), st));
    if (ar.measure()) return SLSO_OK;
    return launch_score_sum<float>(h, static_cast<float*>(scores), n, sums, st);
  }
  float* Mf = ar.take<float>(static_cast<size_t>(d) * kk);
  float* part = ar.take<float>(static_cast<size_t>(ncb) * n);
  if (ar.measure()) return SLSO_OK;
  if (compute == SLSO_F32) {
    m_to_f32_kernel<<<grid1d(d * kk, h), 256, 0, st>>>(M, d * kk, Mf);
    SLSO_CHECK_LAUNCH();
    score_tile_kernel<T, float, 0><<<grid, 256, 0, st>>>(X, n, d, ldx, Mf, kk, part);
  } else {
    m_to_bf16val_kernel<<<grid1d(d * kk, h), 256, 0, st>>>(M, d * kk, Mf);
    SLSO_CHECK_LAUNCH();
    score_tile_kernel<T, float, 1><<<grid, 256, 0, st>>>(X, n, d, ldx, Mf, kk, part);
  }
  SLSO_CHECK_LAUNCH();
  score_combine_kernel<float, float><<<grid1d(n, h), 256, 0, st>>>(part, n, ncb, static_cast<float*>(scores));
  SLSO_CHECK_LAUNCH();
  SLSO_TRY(correct_top_rows(h, ar, X, n, d, ldx, M, kk, compute, correct_frac, static_cast<float*>(scores), st));
  return launch_score_sum<float>(h, static_cast<float*>(scores), n, sums, st);
}

}  // namespace

slso_status run_scores(Handle& h, Arena& ar, const void* X, int64_t n, int64_t d, int64_t ldx,
                       int32_t xdt, const double* M, int64_t kk, int32_t compute, void* scores,
                       double correct_frac, cudaStream_t st, const unsigned int* colmax_pre) {
  switch (xdt) {
    case SLSO_F64: return scores_typed(h, ar, static_cast<const double*>(X), n, d, ldx, M, kk, compute, correct_frac, scores, st, colmax_pre);
    case SLSO_F32: return scores_typed(h, ar, static_cast<const float*>(X), n, d, ldx, M, kk, compute, correct_frac, scores, st, colmax_pre);
    case SLSO_BF16: return scores_typed(h, ar, static_cast<const __nv_bfloat16*>(X), n, d, ldx, M, kk, compute, correct_frac, scores, st, colmax_pre);
    default: return fail(SLSO_ERR_DTYPE, "unsupported X dtype %d", xdt);
  }
}

}  // namespace slso

namespace slso {

slso_status score_sum(Handle& h, Arena& ar, const void* scores, int32_t sdt, int64_t n, cudaStream_t st) {
  double* sums = ar.take<double>(kSumBlocks);
  if (ar.measure()) return SLSO_OK;
  if (sdt == SLSO_F64) return launch_score_sum<double>(h, static_cast<const double*>(scores), n, sums, st);
  return launch_score_sum<float>(h, static_cast<const float*>(scores), n, sums, st);
}


slso_status score_group_add(Handle& h, Arena& ar, const void* X, int64_t n, int64_t d, int64_t ldx, const double* M,
                            int64_t kk, float* scores, ScoreGroupJob* job, double** sums, cudaStream_t st) {
  // scores_typed's scratch, in its order: the score-sum blocks, then the tensor-core product's
  *sums = ar.take<double>(kSumBlocks);
  bool used = false;
  SLSO_TRY(run_scores_tc(h, ar, X, n, d, ldx, SLSO_F32, M, kk, SLSO_F32, scores, &used, st, nullptr, job));
  if (!ar.measure() && !used) return fail(SLSO_ERR_SHAPE, "internal: grouped scores need the tensor-core product");
  return SLSO_OK;
}

slso_status score_group_sum(Handle& h, const float* scores, int64_t n, double* sums, cudaStream_t st) {
  return launch_score_sum<float>(h, scores, n, sums, st);
}
}  // namespace slso
