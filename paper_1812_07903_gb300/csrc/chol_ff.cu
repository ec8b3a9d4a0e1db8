// Cholesky factor of the Gram matrix and its inverse in float-float arithmetic on the float32 pipe,
// in one cooperative kernel (the Gram route's R = chol(SX^T SX) and R^-1; Algorithm 2/3 steps 2-4).
//
// On this part a float64 instruction that depends on the previous one costs ~64 clocks and the
// float64 pipe runs at 1/64 of the float32 pipe, so a float64 Cholesky of d = 1024 is bound by
// latency chains and launch gaps (32 panel + 31 update launches, then a column-by-column R^-1).
// Here every number is an unevaluated pair hi + lo of float32 values (about 2^-48 relative):
// products by FMA with their exact rounding error, sums by TwoSum (Knuth), square root and
// reciprocal by one Newton step from the correctly rounded float32 value.  The Gram matrix is taken
// as G' = D G D with D = diag(2^-e_j) (the column scales of SX), so that every entry of G' lies in
// float32's range; then L' = chol(G') = D L and L'^-1 = L^-1 D^-1 with L = R^T.
//
// Blocked right-looking Cholesky with 32-wide blocks that builds X = L'^-1 in the same elimination:
// the right-hand side B starts as the identity, and at step k
//   A  (every CTA, redundantly): L_kk = chol(A_kk) and Li = L_kk^-1 in shared memory (the
//      augmented column operations of the factorisation applied to an identity block);
//   B  (tasks over CTAs): the panel L_Ik = A_Ik Li^T (I > k) and the row block X_k = Li B_k;
//   C  (tasks over CTAs): A_IJ -= L_Ik L_Jk^T (k < J <= I) and B_I -= L_Ik X_k (I > k);
// with a grid barrier after B and after C (bounded waits: a timeout sets DevState::timeout).
// A non-positive or non-finite pivot closes the route (gram_ok = 0, gram_resid = NaN); every CTA
// factors the same block with the same arithmetic, so all of them take that exit at the same step.
// Outputs in float64: L (d x d row-major, lower triangle) = R^T, and Rinv (column-major R^-1, i.e.
// X row-major: (R^-1)_ic = X_ci).
#include <cmath>

#include <math_constants.h>

#include "common.cuh"

namespace slso {

namespace {

constexpr int kFb = 32;  // block edge
constexpr int kFThreads = 256;
constexpr long long kFWaitPolls = 1ll << 24;

struct ff {
  float h, l;
};

__device__ __forceinline__ void two_sum(float a, float b, float& s, float& e) {
  s = __fadd_rn(a, b);
  const float bb = __fsub_rn(s, a);
  e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
}
// |a| >= |b| (or a == 0)
__device__ __forceinline__ ff fast_two_sum(float a, float b) {
  const float s = __fadd_rn(a, b);
  return {s, __fsub_rn(b, __fsub_rn(s, a))};
}
__device__ __forceinline__ ff ff_add(ff x, ff y) {
  float s, e;
  two_sum(x.h, y.h, s, e);
  e = __fadd_rn(e, __fadd_rn(x.l, y.l));
  return fast_two_sum(s, e);
}
__device__ __forceinline__ ff ff_mul(ff x, ff y) {
  const float p = __fmul_rn(x.h, y.h);
  float e = __fmaf_rn(x.h, y.h, -p);
  e = __fmaf_rn(x.h, y.l, e);
  e = __fmaf_rn(x.l, y.h, e);
  return fast_two_sum(p, e);
}
// z - x y
__device__ __forceinline__ ff ff_fms(ff z, ff x, ff y) {
  const ff p = ff_mul(x, y);
  return ff_add(z, ff{-p.h, -p.l});
}
// sqrt(a), a > 0: y = fl(sqrt(a_h)), then y + (a - y^2) / (2y)
__device__ __forceinline__ ff ff_sqrt(ff a) {
  const float y = __fsqrt_rn(a.h);
  const float p = __fmul_rn(y, y);
  const float e = __fmaf_rn(y, y, -p);
  const float r = __fadd_rn(__fsub_rn(__fsub_rn(a.h, p), e), a.l);
  return fast_two_sum(y, __fmul_rn(r, __fdiv_rn(0.5f, y)));
}
// 1 / a: y = fl(1 / a_h), then y + y (1 - a y)
__device__ __forceinline__ ff ff_recip(ff a) {
  const float y = __frcp_rn(a.h);
  const float p = __fmul_rn(a.h, y);
  const float e = __fmaf_rn(a.h, y, -p);
  const float r = __fsub_rn(__fsub_rn(__fsub_rn(1.0f, p), e), __fmul_rn(a.l, y));
  return fast_two_sum(y, __fmul_rn(y, r));
}

// One term of a float-float dot product: (S, C) += (ah + al)(bh + bl), the product's rounding
// error by FMA, the sum's by TwoSum; (S, C) is folded into a pair every 16 terms by the caller.
__device__ __forceinline__ void dot_term(float ah, float al, float bh, float bl, float& S, float& C) {
  const float p = __fmul_rn(ah, bh);
  float e = __fmaf_rn(ah, bh, -p);
  e = __fmaf_rn(ah, bl, e);
  e = __fmaf_rn(al, bh, e);
  float t, err;
  two_sum(S, p, t, err);
  S = t;
  C = __fadd_rn(C, __fadd_rn(err, e));
}

__device__ bool grid_barrier_ff(unsigned int* count, volatile unsigned int* gen, int* abort_flag) {
  __syncthreads();
  __shared__ int s_ok;
  if (threadIdx.x == 0) {
    s_ok = 1;
    const unsigned int g = *gen;
    __threadfence();
    if (atomicAdd(count, 1u) == gridDim.x - 1) {
      *count = 0;
      __threadfence();
      atomicAdd(const_cast<unsigned int*>(gen), 1u);
    } else {
      long long it = 0;
      while (*gen == g) {
        if (++it > kFWaitPolls || *reinterpret_cast<volatile int*>(abort_flag)) {
          s_ok = 0;
          atomicExch(abort_flag, 1);
          break;
        }
        __nanosleep(64);
      }
    }
    __threadfence();
  }
  __syncthreads();
  return s_ok;
}

struct Smem {
  float Dh[kFb][kFb + 1], Dl[kFb][kFb + 1];  // A_kk -> L_kk
  float Ih[kFb][kFb + 1], Il[kFb][kFb + 1];  // identity -> L_kk^-1
  float Ph[kFb][kFb + 4], Pl[kFb][kFb + 4];  // task operands, [m][row]
  float Qh[kFb][kFb + 4], Ql[kFb][kFb + 4];  // [m][column]
  float rh, rl;
  int bad;
};

// C (32 x 32 tile at rows r0, columns c0 of a row-major float-float matrix Y with pitch d) =
// init + sign * sum_m P[m][i] Q[m][j]; init from Y (add = true) or zero.  Rows / columns beyond
// nrow / ncol are not written; lower = true writes only j <= i (global indices).
// Thread t: row i = t / 8, columns 4 (t % 8) .. + 4.
__device__ void tile_product(Smem& sm, float2* Y, int d, int r0, int c0, bool add, float sign, bool lower) {
  const int t = threadIdx.x, i = t >> 3, j0 = (t & 7) * 4;
  float S[4] = {0.f, 0.f, 0.f, 0.f}, C[4] = {0.f, 0.f, 0.f, 0.f};
  ff acc[4];
#pragma unroll
  for (int q = 0; q < 4; ++q) acc[q] = {0.f, 0.f};
#pragma unroll 4
  for (int m = 0; m < kFb; ++m) {
    const float ah = sm.Ph[m][i] * sign, al = sm.Pl[m][i] * sign;
    const float4 bh = *reinterpret_cast<const float4*>(&sm.Qh[m][j0]);
    const float4 bl = *reinterpret_cast<const float4*>(&sm.Ql[m][j0]);
    dot_term(ah, al, bh.x, bl.x, S[0], C[0]);
    dot_term(ah, al, bh.y, bl.y, S[1], C[1]);
    dot_term(ah, al, bh.z, bl.z, S[2], C[2]);
    dot_term(ah, al, bh.w, bl.w, S[3], C[3]);
    if ((m & 15) == 15) {
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        acc[q] = ff_add(acc[q], fast_two_sum(S[q], C[q]));
        S[q] = 0.f;
        C[q] = 0.f;
      }
    }
  }
  const int gi = r0 + i;
  if (gi >= d) return;
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    const int gj = c0 + j0 + q;
    if (gj >= d || (lower && gj > gi)) continue;
    float2* y = Y + static_cast<int64_t>(gi) * d + gj;
    ff v = acc[q];
    if (add) {
      const float2 o = *y;
      v = ff_add(ff{o.x, o.y}, v);
    }
    *y = make_float2(v.h, v.l);
  }
}

// P[m][i] = Y[r0 + i][c0 + m] (zero beyond d)
__device__ void load_rows_t(Smem& sm, const float2* Y, int d, int r0, int c0) {
  for (int e = threadIdx.x; e < kFb * kFb; e += kFThreads) {
    const int i = e >> 5, m = e & 31;
    float2 v = make_float2(0.f, 0.f);
    if (r0 + i < d && c0 + m < d) v = Y[static_cast<int64_t>(r0 + i) * d + c0 + m];
    sm.Ph[m][i] = v.x;
    sm.Pl[m][i] = v.y;
  }
}
// Q[m][j] = Y[r0 + j][c0 + m]
__device__ void load_q_rows_t(Smem& sm, const float2* Y, int d, int r0, int c0) {
  for (int e = threadIdx.x; e < kFb * kFb; e += kFThreads) {
    const int j = e >> 5, m = e & 31;
    float2 v = make_float2(0.f, 0.f);
    if (r0 + j < d && c0 + m < d) v = Y[static_cast<int64_t>(r0 + j) * d + c0 + m];
    sm.Qh[m][j] = v.x;
    sm.Ql[m][j] = v.y;
  }
}
// Q[m][j] = Y[r0 + m][c0 + j]
__device__ void load_q_rows(Smem& sm, const float2* Y, int d, int r0, int c0) {
  for (int e = threadIdx.x; e < kFb * kFb; e += kFThreads) {
    const int m = e >> 5, j = e & 31;
    float2 v = make_float2(0.f, 0.f);
    if (r0 + m < d && c0 + j < d) v = Y[static_cast<int64_t>(r0 + m) * d + c0 + j];
    sm.Qh[m][j] = v.x;
    sm.Ql[m][j] = v.y;
  }
}

// Step k, part A: L_kk and L_kk^-1 in shared memory (rows / columns beyond d: identity).
// Returns false (uniformly) on a non-positive or non-finite pivot.
__device__ bool factor_diag(Smem& sm, const float2* A, int d, int k0) {
  const int t = threadIdx.x;
  for (int e = t; e < kFb * kFb; e += kFThreads) {
    const int i = e >> 5, j = e & 31;
    float2 v = make_float2(i == j ? 1.f : 0.f, 0.f);
    if (k0 + i < d && k0 + j < d) v = j <= i ? A[static_cast<int64_t>(k0 + i) * d + k0 + j] : make_float2(0.f, 0.f);
    sm.Dh[i][j] = v.x;
    sm.Dl[i][j] = v.y;
    sm.Ih[i][j] = i == j ? 1.f : 0.f;
    sm.Il[i][j] = 0.f;
  }
  if (t == 0) sm.bad = 0;
  __syncthreads();
  for (int j = 0; j < kFb; ++j) {
    if (t == 0) {
      const ff piv{sm.Dh[j][j], sm.Dl[j][j]};
      if (!(piv.h > 0.f) || !isfinite(piv.h) || !isfinite(piv.l)) {
        sm.bad = 1;
      } else {
        const ff s = ff_sqrt(piv);
        const ff r = ff_recip(s);
        sm.Dh[j][j] = s.h;
        sm.Dl[j][j] = s.l;
        sm.rh = r.h;
        sm.rl = r.l;
      }
    }
    __syncthreads();
    if (sm.bad) return false;
    const ff r{sm.rh, sm.rl};
    if (t < kFb) {
      if (t > j) {
        const ff v = ff_mul(ff{sm.Dh[t][j], sm.Dl[t][j]}, r);
        sm.Dh[t][j] = v.h;
        sm.Dl[t][j] = v.l;
      }
    } else if (t < 2 * kFb) {
      const int c = t - kFb;
      if (c <= j) {
        const ff v = ff_mul(ff{sm.Ih[j][c], sm.Il[j][c]}, r);
        sm.Ih[j][c] = v.h;
        sm.Il[j][c] = v.l;
      }
    }
    __syncthreads();
    // rows i > j: D[i][m] -= L_ij L_mj (j < m <= i), I[i][c] -= L_ij I[j][c] (c <= j)
    const int rows = kFb - 1 - j;
    for (int e = t; e < rows * kFb; e += kFThreads) {
      const int i = j + 1 + e / kFb, m = e % kFb;
      const ff lij{sm.Dh[i][j], sm.Dl[i][j]};
      if (m > j && m <= i) {
        const ff v = ff_fms(ff{sm.Dh[i][m], sm.Dl[i][m]}, lij, ff{sm.Dh[m][j], sm.Dl[m][j]});
        sm.Dh[i][m] = v.h;
        sm.Dl[i][m] = v.l;
      } else if (m <= j) {
        const ff v = ff_fms(ff{sm.Ih[i][m], sm.Il[i][m]}, lij, ff{sm.Ih[j][m], sm.Il[j][m]});
        sm.Ih[i][m] = v.h;
        sm.Il[i][m] = v.l;
      }
    }
    __syncthreads();
  }
  return true;
}

// bar[0..1] grid barrier, bar[2] abort flag (zeroed by the host before the launch).
__global__ void __launch_bounds__(kFThreads, 1)
    chol_ff_kernel(double* __restrict__ L, const int* __restrict__ cexp, int d, float2* __restrict__ A,
                   float2* __restrict__ X, double* __restrict__ Rinv, unsigned int* bar, DevState* __restrict__ st) {
  if (*reinterpret_cast<volatile int32_t*>(&st->gram_ok) == 0) return;  // grid-uniform
  extern __shared__ __align__(16) unsigned char smem_raw[];
  Smem& sm = *reinterpret_cast<Smem*>(smem_raw);
  int* abort_flag = reinterpret_cast<int*>(bar + 2);
  const int64_t dd = static_cast<int64_t>(d) * d;
  const int64_t gtid = static_cast<int64_t>(blockIdx.x) * kFThreads + threadIdx.x;
  const int64_t gstride = static_cast<int64_t>(gridDim.x) * kFThreads;
  // G' = D G D as float-float (lower triangle), X = identity
  for (int64_t e = gtid; e < dd; e += gstride) {
    const int i = static_cast<int>(e / d), j = static_cast<int>(e % d);
    if (j <= i) {
      const double g = ldexp(L[e], -cexp[i] - cexp[j]);
      const float h = __double2float_rn(g);
      A[e] = make_float2(h, __double2float_rn(g - static_cast<double>(h)));
    }
    X[e] = make_float2(i == j ? 1.f : 0.f, 0.f);
  }
  auto sync_all = [&]() -> bool {
    if (grid_barrier_ff(bar, bar + 1, abort_flag)) return true;
    if (threadIdx.x == 0) atomicExch(&st->timeout, 7);
    return false;
  };
  if (!sync_all()) return;
  const int nb = (d + kFb - 1) / kFb;
  for (int k = 0; k < nb; ++k) {
    const int k0 = k * kFb;
    if (!factor_diag(sm, A, d, k0)) {
      if (blockIdx.x == 0 && threadIdx.x == 0) {
        st->gram_ok = 0;
        st->gram_resid = CUDART_NAN;
      }
      return;
    }
    // part B: tasks 0 .. nb-k-2 are the panel row blocks I = k+1.., then k+1 column tiles of X_k
    const int npanel = nb - k - 1;
    for (int task = blockIdx.x; task < nb; task += gridDim.x) {
      __syncthreads();
      if (task < npanel) {
        const int r0 = (k + 1 + task) * kFb;
        load_rows_t(sm, A, d, r0, k0);  // P[m][i] = A[r0+i][k0+m]
        for (int e = threadIdx.x; e < kFb * kFb; e += kFThreads) {
          const int m = e >> 5, j = e & 31;  // Q[m][j] = Li[j][m]
          sm.Qh[m][j] = sm.Ih[j][m];
          sm.Ql[m][j] = sm.Il[j][m];
        }
        __syncthreads();
        tile_product(sm, A, d, r0, k0, false, 1.f, false);
      } else {
        const int c0 = (task - npanel) * kFb;
        for (int e = threadIdx.x; e < kFb * kFb; e += kFThreads) {
          const int m = e >> 5, i = e & 31;  // P[m][i] = Li[i][m]
          sm.Ph[m][i] = sm.Ih[i][m];
          sm.Pl[m][i] = sm.Il[i][m];
        }
        load_q_rows(sm, X, d, k0, c0);  // Q[m][j] = B[k0+m][c0+j]
        __syncthreads();
        tile_product(sm, X, d, k0, c0, false, 1.f, false);
      }
    }
    if (!sync_all()) return;
    if (blockIdx.x == 0)  // L_kk into A: every CTA has read A_kk before the barrier above
      for (int e = threadIdx.x; e < kFb * kFb; e += kFThreads) {
        const int i = e >> 5, j = e & 31;
        if (k0 + i < d && j <= i) A[static_cast<int64_t>(k0 + i) * d + k0 + j] = make_float2(sm.Dh[i][j], sm.Dl[i][j]);
      }
    // part C: lower tiles (I, J) of the trailing matrix, then the (I, c) tiles of B
    const int ntri = npanel * (npanel + 1) / 2;
    const int ntask = ntri + npanel * (k + 1);
    for (int task = blockIdx.x; task < ntask; task += gridDim.x) {
      __syncthreads();
      if (task < ntri) {
        int a = static_cast<int>((sqrt(8.0 * task + 1.0) - 1.0) * 0.5);
        while ((a + 1) * (a + 2) / 2 <= task) ++a;
        while (a * (a + 1) / 2 > task) --a;
        const int b = task - a * (a + 1) / 2;
        const int r0 = (k + 1 + a) * kFb, c0 = (k + 1 + b) * kFb;
        load_rows_t(sm, A, d, r0, k0);    // P[m][i] = L[r0+i][k0+m]
        load_q_rows_t(sm, A, d, c0, k0);  // Q[m][j] = L[c0+j][k0+m]
        __syncthreads();
        tile_product(sm, A, d, r0, c0, true, -1.f, a == b);
      } else {
        const int u = task - ntri;
        const int a = u / (k + 1), c = u % (k + 1);
        const int r0 = (k + 1 + a) * kFb, c0 = c * kFb;
        load_rows_t(sm, A, d, r0, k0);  // P[m][i] = L[r0+i][k0+m]
        load_q_rows(sm, X, d, k0, c0);  // Q[m][j] = X[k0+m][c0+j]
        __syncthreads();
        tile_product(sm, X, d, r0, c0, true, -1.f, false);
      }
    }
    if (!sync_all()) return;
  }
  // L = D^-1 L' (row i times 2^e_i) and R^-1 = X^T with X = X' D (column i of X' times 2^-e_i)
  for (int64_t e = gtid; e < dd; e += gstride) {
    const int i = static_cast<int>(e / d), j = static_cast<int>(e % d);
    if (j <= i) {
      const float2 a = A[e];
      L[e] = ldexp(static_cast<double>(a.x) + static_cast<double>(a.y), cexp[i]);
    }
    const float2 x = X[e];  // X'[i][j]: (R^-1)_ji at Rinv[i d + j]
    Rinv[e] = j <= i ? ldexp(static_cast<double>(x.x) + static_cast<double>(x.y), -cexp[j]) : 0.0;
  }
}

}  // namespace

size_t chol_ff_smem() { return sizeof(Smem); }

bool chol_ff_applies(int64_t d) { return d >= 1 && d <= 8192; }

slso_status run_chol_ff(Handle& h, double* L, const int* cexp, int64_t d, float2* A, float2* X, double* Rinv,
                        unsigned int* bar, cudaStream_t st) {
  const size_t smem = sizeof(Smem);
  SLSO_TRY(raise_smem_limit(chol_ff_kernel, smem));
  int occ = 0;
  SLSO_CHECK_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, chol_ff_kernel, kFThreads, smem));
  if (occ < 1) return fail(SLSO_ERR_CUDA, "float-float Cholesky kernel cannot be resident (smem %zu)", smem);
  SLSO_CHECK_CUDA(cudaMemsetAsync(bar, 0, sizeof(unsigned int) * 4, st));
  int d_i = static_cast<int>(d);
  DevState* stp = h.state;
  void* args[] = {&L, &cexp, &d_i, &A, &X, &Rinv, &bar, &stp};
  SLSO_CHECK_CUDA(cudaLaunchCooperativeKernel(reinterpret_cast<void*>(chol_ff_kernel), dim3(h.num_sms), dim3(kFThreads),
                                              args, smem, st));
  note_launch();
  return SLSO_OK;
}

}  // namespace slso
