// Approximate left singular vectors U = X V_r Sigma_r^-1 (Algorithm 2 step 3; Algorithm 3
// step 4): the sketch SX, its sketched SVD (Householder QR + one-sided Jacobi SVD of R, float64,
// rank r = #{sigma_j > tau sigma_1} on the device), M = V diag(1/sigma) with columns >= r zero,
// then the product X M.  For float32 / bfloat16 X it runs on the tensor cores (the score kernel
// with a write-out epilogue, 256-column blocks of M, float32-accurate 3xTF32 / BF16X3 operands);
// for float64 X it is written tile by tile in float64 (CTA tile 64 rows x 64 columns, K-steps of
// 16 through shared memory, 4 x 4 outputs per thread).
#include <algorithm>
#include <type_traits>

#include "common.cuh"

namespace slso {

namespace {

constexpr int kUm = 64, kUn = 64, kUk = 16;

unsigned blocks_for(int64_t n, const Handle& h) {
  return static_cast<unsigned>(std::max<int64_t>(1, std::min<int64_t>(ceil_div(n, 256), int64_t(h.num_sms) * 8)));
}

template <class Acc>
__global__ void basis_m_kernel(const double* __restrict__ sigma, const double* __restrict__ V, int64_t d,
                               const DevState* __restrict__ state, Acc* __restrict__ M) {
  const int64_t r = state->rank;
  for (int64_t e = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; e < d * d;
       e += static_cast<int64_t>(gridDim.x) * blockDim.x) {
    const int64_t c = e % d;
    M[e] = (c < r) ? static_cast<Acc>(V[e] / sigma[c]) : Acc(0);
  }
}

template <class T> __device__ __forceinline__ double as_double(const T* p) { return static_cast<double>(to_float(*p)); }
template <> __device__ __forceinline__ double as_double<double>(const double* p) { return *p; }

template <class T, class Acc>
__global__ void __launch_bounds__(256) basis_tile_kernel(const T* __restrict__ X, int64_t n, int64_t d, int64_t ldx,
                                                         const Acc* __restrict__ M, Acc* __restrict__ U,
                                                         int64_t ldu) {
  __shared__ Acc Xs[kUk][kUm + 1];
  __shared__ Acc Ms[kUk][kUn];
  const int tx = threadIdx.x % 16, ty = threadIdx.x / 16;
  const int64_t r0 = static_cast<int64_t>(blockIdx.x) * kUm, c0 = static_cast<int64_t>(blockIdx.y) * kUn;
  Acc acc[4][4];
#pragma unroll
  for (int a = 0; a < 4; ++a)
#pragma unroll
    for (int b = 0; b < 4; ++b) acc[a][b] = Acc(0);
  for (int64_t k0 = 0; k0 < d; k0 += kUk) {
    for (int t = threadIdx.x; t < kUm * kUk; t += 256) {
      const int rr = t / kUk, kc = t % kUk;
      const int64_t r = r0 + rr, k = k0 + kc;
      Xs[kc][rr] = (r < n && k < d) ? static_cast<Acc>(as_double(X + r * ldx + k)) : Acc(0);
    }
    for (int t = threadIdx.x; t < kUk * kUn; t += 256) {
      const int kc = t / kUn, cc = t % kUn;
      const int64_t k = k0 + kc, c = c0 + cc;
      Ms[kc][cc] = (k < d && c < d) ? M[k * d + c] : Acc(0);
    }
    __syncthreads();
#pragma unroll
    for (int kc = 0; kc < kUk; ++kc) {
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
    const int64_t r = r0 + ty * 4 + a;
    if (r >= n) continue;
#pragma unroll
    for (int b = 0; b < 4; ++b) {
      const int64_t c = c0 + tx * 4 + b;
      if (c < d) U[r * ldu + c] = acc[a][b];
    }
  }
}

template <class T, class Acc>
slso_status basis_typed(Handle& h, Arena& ar, const T* X, int64_t n, int64_t d, int64_t ldx, const SolveOut& so,
                        Acc* U, int64_t ldu, cudaStream_t st) {
  if constexpr (!std::is_same<T, double>::value) {
    // float32 / bfloat16 X: the product on the tensor cores (float32-accurate split operands)
    double* M64 = ar.take<double>(static_cast<size_t>(d) * d);
    if (!ar.measure()) {
      basis_m_kernel<double><<<blocks_for(d * d, h), 256, 0, st>>>(so.sigma, so.V, d, h.state, M64);
      SLSO_CHECK_LAUNCH();
    }
    bool used = false;
    SLSO_TRY(run_product_tc(h, ar, X, n, d, ldx, std::is_same<T, float>::value ? SLSO_F32 : SLSO_BF16, M64, d, U,
                            ldu, &used, st));
    if (used) return SLSO_OK;
  }
  Acc* M = ar.take<Acc>(static_cast<size_t>(d) * d);
  if (ar.measure()) return SLSO_OK;
  basis_m_kernel<Acc><<<blocks_for(d * d, h), 256, 0, st>>>(so.sigma, so.V, d, h.state, M);
  SLSO_CHECK_LAUNCH();
  const dim3 g(static_cast<unsigned>(ceil_div(n, kUm)), static_cast<unsigned>(ceil_div(d, kUn)));
  basis_tile_kernel<T, Acc><<<g, 256, 0, st>>>(X, n, d, ldx, M, U, ldu);
  SLSO_CHECK_LAUNCH();
  return SLSO_OK;
}

}  // namespace

slso_status approx_u_plan(Handle& h, Arena& ar, const void* X, int64_t n, int64_t d, int64_t ldx, int32_t xdt,
                          const slso_params* p, void* U, int64_t ldu, cudaStream_t st) {
  const int64_t s = p->s;
  const double tau = p->tau < 0 ? default_tau(s, d) : p->tau;
  double* SX = ar.take<double>(static_cast<size_t>(s) * d);
  prof_begin(h, ar, ST_SKETCH, st);
  SLSO_TRY(run_sketch(h, ar, X, n, d, ldx, xdt, p->kind, s, p->seed_S, p->nnz, SX, st));
  prof_end(h, ar, st);
  SolveOut so;
  SLSO_TRY(run_solve(h, ar, SX, s, d, tau, 0, 0, 1, &so, st));
  prof_begin(h, ar, ST_SCORES, st);
  switch (xdt) {
    case SLSO_F64:
      SLSO_TRY(basis_typed(h, ar, static_cast<const double*>(X), n, d, ldx, so, static_cast<double*>(U), ldu, st));
      break;
    case SLSO_F32:
      SLSO_TRY(basis_typed(h, ar, static_cast<const float*>(X), n, d, ldx, so, static_cast<float*>(U), ldu, st));
      break;
    default:
      SLSO_TRY(basis_typed(h, ar, static_cast<const __nv_bfloat16*>(X), n, d, ldx, so, static_cast<float*>(U), ldu, st));
      break;
  }
  prof_end(h, ar, st);
  return SLSO_OK;
}

}  // namespace slso
