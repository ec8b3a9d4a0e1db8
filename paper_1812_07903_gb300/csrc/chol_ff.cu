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

// acc[q] += sum_m P[m][i] Q[m][j0 + q] for this thread's row i = t / 8, columns j0 = 4 (t % 8) .. + 4.
__device__ void tile_accumulate(const Smem& sm, ff* acc) {
  const int t = threadIdx.x, i = t >> 3, j0 = (t & 7) * 4;
  float S[4] = {0.f, 0.f, 0.f, 0.f}, C[4] = {0.f, 0.f, 0.f, 0.f};
#pragma unroll 4
  for (int m = 0; m < kFb; ++m) {
    const float ah = sm.Ph[m][i], al = sm.Pl[m][i];
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
}

// P[m][i] = Y[r0 + m][c0 + i] (zero beyond d)
__device__ void load_p_rows(Smem& sm, const float2* Y, int d, int r0, int c0) {
  for (int e = threadIdx.x; e < kFb * kFb; e += kFThreads) {
    const int m = e >> 5, i = e & 31;
    float2 v = make_float2(0.f, 0.f);
    if (r0 + m < d && c0 + i < d) v = Y[static_cast<int64_t>(r0 + m) * d + c0 + i];
    sm.Ph[m][i] = v.x;
    sm.Pl[m][i] = v.y;
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
// Right-hand sides after the factorisation (every CTA, tasks of 32 x 32 outputs): with the JL
// matrix Pi (d x k, k > 0) and the probes Z (d x 4), both float64 row-major, Out = X'^T [Pi | Z]
// (Out_ic = sum over m >= i of X'_mi [Pi | Z]_mc) gives M = R^-1 Pi = diag(2^-e) Out[:, :k] (float64,
// d x k row-major; st->m_ready = 1) and Y'' = X'^T Z (float-float, d x 4) for the probe check.
__global__ void __launch_bounds__(kFThreads, 1)
    chol_ff_kernel(double* __restrict__ L, const int* __restrict__ cexp, int d, float2* __restrict__ A,
                   float2* __restrict__ X, double* __restrict__ Rinv, const double* __restrict__ Pi, int k,
                   const double* __restrict__ Z, double* __restrict__ M, float2* __restrict__ Yff, unsigned int* bar,
                   DevState* __restrict__ st) {
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
  // Out = X'^T [Pi | Z]: output tiles (I, Cb), I over row blocks, Cb over 32-column blocks of [Pi | Z]
  {
    const int width = k + 4, ncb = (width + kFb - 1) / kFb;
    for (int task = blockIdx.x; task < nb * ncb; task += gridDim.x) {
      const int I = task / ncb, Cb = task % ncb;
      const int i0 = I * kFb, c0 = Cb * kFb;
      ff acc[4];
#pragma unroll
      for (int q = 0; q < 4; ++q) acc[q] = {0.f, 0.f};
      for (int mb = I; mb < nb; ++mb) {
        __syncthreads();
        load_p_rows(sm, X, d, mb * kFb, i0);  // P[m][i] = X'[mb 32 + m][i0 + i]
        for (int e = threadIdx.x; e < kFb * kFb; e += kFThreads) {
          const int m = e >> 5, j = e & 31;  // Q[m][j] = [Pi | Z][mb 32 + m][c0 + j]
          const int r = mb * kFb + m, c = c0 + j;
          double v = 0.0;
          if (r < d) v = c < k ? Pi[static_cast<int64_t>(r) * k + c] : (c < width ? Z[r * 4 + (c - k)] : 0.0);
          const float h = __double2float_rn(v);
          sm.Qh[m][j] = h;
          sm.Ql[m][j] = __double2float_rn(v - static_cast<double>(h));
        }
        __syncthreads();
        tile_accumulate(sm, acc);
      }
      const int i = i0 + (threadIdx.x >> 3), j0 = c0 + (threadIdx.x & 7) * 4;
      if (i < d)
#pragma unroll
        for (int q = 0; q < 4; ++q) {
          const int c = j0 + q;
          if (c < k) M[static_cast<int64_t>(i) * k + c] = ldexp(static_cast<double>(acc[q].h) + static_cast<double>(acc[q].l), -cexp[i]);
          else if (c < width) Yff[i * 4 + (c - k)] = make_float2(acc[q].h, acc[q].l);
        }
    }
    if (k > 0 && blockIdx.x == 0 && threadIdx.x == 0) st->m_ready = 1;
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

// ------------------------------------------------------------------ probe check in float-float
// With SX' = SX D (column j times 2^-e_j, every entry in (-1, 1)), X' = L'^-1 and Y'' = X'^T Z, the
// probe residual F Z = R^-T SX^T SX R^-1 Z - Z equals X' (SX'^T (SX' Y'')) - Z: every power of two
// cancels, so float32's range suffices.  SX is read in float64 and split exactly into a float pair
// with integer operations.

// a 2^-e as hi + lo (hi: the leading 24 bits rounded, lo: the remaining 29 bits rounded to 24).
__device__ __forceinline__ ff split_scaled(double a, int e) {
  const unsigned long long u = static_cast<unsigned long long>(__double_as_longlong(a));
  const int ex = static_cast<int>((u >> 52) & 0x7FFu);
  if (ex == 0x7FF) return {CUDART_NAN_F, 0.f};
  if (ex == 0) {  // zero or subnormal: the float64 path (rare)
    const double v = ldexp(a, -e);
    const float h = __double2float_rn(v);
    return {h, __double2float_rn(v - static_cast<double>(h))};
  }
  const long long m = static_cast<long long>((u & ((1ull << 52) - 1)) | (1ull << 52));
  const int E = ex - 1075 - e;  // |a 2^-e| = m 2^E
  const long long hi = (m + (1ll << 28)) >> 29;
  const long long lo = m - hi * (1ll << 29);
  float fh = ldexpf(static_cast<float>(hi), E + 29);
  float fl = ldexpf(static_cast<float>(lo), E);
  if (u >> 63) {
    fh = -fh;
    fl = -fl;
  }
  return {fh, fl};
}

// W[r] = SX'_r . Y'' (4 probes, float-float): one warp per row.
__global__ void __launch_bounds__(256) probe_w_ff_kernel(const double* __restrict__ SX, int64_t s, int d,
                                                         const int* __restrict__ cexp, const float2* __restrict__ Yff,
                                                         float2* __restrict__ Wff, const DevState* __restrict__ st) {
  if (*reinterpret_cast<const volatile int32_t*>(&st->gram_ok) == 0) return;
  const int lane = threadIdx.x & 31;
  const int64_t r = blockIdx.x * static_cast<int64_t>(blockDim.x >> 5) + (threadIdx.x >> 5);
  if (r >= s) return;
  const double* row = SX + r * d;
  float S[4] = {0.f, 0.f, 0.f, 0.f}, C[4] = {0.f, 0.f, 0.f, 0.f};
  ff acc[4] = {{0.f, 0.f}, {0.f, 0.f}, {0.f, 0.f}, {0.f, 0.f}};
  int cnt = 0;
  for (int j = lane; j < d; j += 32) {
    const ff a = split_scaled(row[j], cexp[j]);
    const float4 y0 = *reinterpret_cast<const float4*>(Yff + 4 * j);      // probes 0, 1
    const float4 y1 = *reinterpret_cast<const float4*>(Yff + 4 * j + 2);  // probes 2, 3
    dot_term(a.h, a.l, y0.x, y0.y, S[0], C[0]);
    dot_term(a.h, a.l, y0.z, y0.w, S[1], C[1]);
    dot_term(a.h, a.l, y1.x, y1.y, S[2], C[2]);
    dot_term(a.h, a.l, y1.z, y1.w, S[3], C[3]);
    if ((++cnt & 15) == 0)
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        acc[q] = ff_add(acc[q], fast_two_sum(S[q], C[q]));
        S[q] = C[q] = 0.f;
      }
  }
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    ff v = ff_add(acc[q], fast_two_sum(S[q], C[q]));
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      const ff w{__shfl_xor_sync(0xFFFFFFFFu, v.h, o), __shfl_xor_sync(0xFFFFFFFFu, v.l, o)};
      v = ff_add(v, w);
    }
    if (lane == 0) Wff[r * 4 + q] = make_float2(v.h, v.l);
  }
}

// vpart[b][j][q] = sum over the rows r of chunk b of SX'[r, j] W[r, q] (float-float).
__global__ void __launch_bounds__(256) probe_v_ff_kernel(const double* __restrict__ SX, int64_t s, int d,
                                                         const int* __restrict__ cexp, const float2* __restrict__ Wff,
                                                         int64_t rows_per_chunk, float2* __restrict__ vpart,
                                                         const DevState* __restrict__ st) {
  if (*reinterpret_cast<const volatile int32_t*>(&st->gram_ok) == 0) return;
  const int64_t r0 = blockIdx.x * rows_per_chunk;
  const int64_t r1 = r0 + rows_per_chunk < s ? r0 + rows_per_chunk : s;
  for (int j = threadIdx.x; j < d; j += blockDim.x) {
    const int e = cexp[j];
    float S[4] = {0.f, 0.f, 0.f, 0.f}, C[4] = {0.f, 0.f, 0.f, 0.f};
    ff acc[4] = {{0.f, 0.f}, {0.f, 0.f}, {0.f, 0.f}, {0.f, 0.f}};
    int cnt = 0;
    for (int64_t r = r0; r < r1; ++r) {
      const ff a = split_scaled(SX[r * d + j], e);
      const float4 w0 = *reinterpret_cast<const float4*>(Wff + 4 * r);
      const float4 w1 = *reinterpret_cast<const float4*>(Wff + 4 * r + 2);
      dot_term(a.h, a.l, w0.x, w0.y, S[0], C[0]);
      dot_term(a.h, a.l, w0.z, w0.w, S[1], C[1]);
      dot_term(a.h, a.l, w1.x, w1.y, S[2], C[2]);
      dot_term(a.h, a.l, w1.z, w1.w, S[3], C[3]);
      if ((++cnt & 15) == 0)
#pragma unroll
        for (int q = 0; q < 4; ++q) {
          acc[q] = ff_add(acc[q], fast_two_sum(S[q], C[q]));
          S[q] = C[q] = 0.f;
        }
    }
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const ff v = ff_add(acc[q], fast_two_sum(S[q], C[q]));
      vpart[(static_cast<int64_t>(blockIdx.x) * d + j) * 4 + q] = make_float2(v.h, v.l);
    }
  }
}

// V''[j][q] = the chunk partials added in chunk order.
__global__ void probe_vsum_ff_kernel(const float2* __restrict__ vpart, int chunks, int d, float2* __restrict__ V,
                                     const DevState* __restrict__ st) {
  if (*reinterpret_cast<const volatile int32_t*>(&st->gram_ok) == 0) return;
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= d * 4) return;
  ff v{0.f, 0.f};
  for (int b = 0; b < chunks; ++b) {
    const float2 p = vpart[static_cast<int64_t>(b) * d * 4 + e];
    v = ff_add(v, ff{p.x, p.y});
  }
  V[e] = make_float2(v.h, v.l);
}

// eres[c] = sum_q ((X' V'')_cq - Z_cq)^2 (float64 at the end): one CTA of 128 threads per row c.
__global__ void __launch_bounds__(128) probe_u_ff_kernel(const float2* __restrict__ X, int d,
                                                         const float2* __restrict__ V, const double* __restrict__ Z,
                                                         double* __restrict__ eres, const DevState* __restrict__ st) {
  if (*reinterpret_cast<const volatile int32_t*>(&st->gram_ok) == 0) return;
  __shared__ float2 red[4][4];
  const int c = blockIdx.x, lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  float S[4] = {0.f, 0.f, 0.f, 0.f}, C[4] = {0.f, 0.f, 0.f, 0.f};
  ff acc[4] = {{0.f, 0.f}, {0.f, 0.f}, {0.f, 0.f}, {0.f, 0.f}};
  int cnt = 0;
  for (int i = threadIdx.x; i <= c; i += blockDim.x) {
    const float2 x = X[static_cast<int64_t>(c) * d + i];
    const float4 v0 = *reinterpret_cast<const float4*>(V + 4 * i);
    const float4 v1 = *reinterpret_cast<const float4*>(V + 4 * i + 2);
    dot_term(x.x, x.y, v0.x, v0.y, S[0], C[0]);
    dot_term(x.x, x.y, v0.z, v0.w, S[1], C[1]);
    dot_term(x.x, x.y, v1.x, v1.y, S[2], C[2]);
    dot_term(x.x, x.y, v1.z, v1.w, S[3], C[3]);
    if ((++cnt & 15) == 0)
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        acc[q] = ff_add(acc[q], fast_two_sum(S[q], C[q]));
        S[q] = C[q] = 0.f;
      }
  }
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    ff v = ff_add(acc[q], fast_two_sum(S[q], C[q]));
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      const ff u{__shfl_xor_sync(0xFFFFFFFFu, v.h, o), __shfl_xor_sync(0xFFFFFFFFu, v.l, o)};
      v = ff_add(v, u);
    }
    if (lane == 0) red[w][q] = make_float2(v.h, v.l);
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    double e = 0.0;
    for (int q = 0; q < 4; ++q) {
      ff u{0.f, 0.f};
      for (int ww = 0; ww < 4; ++ww) u = ff_add(u, ff{red[ww][q].x, red[ww][q].y});
      const double diff = (static_cast<double>(u.h) + static_cast<double>(u.l)) - Z[c * 4 + q];
      e = fma(diff, diff, e);
    }
    eres[c] = e;
  }
}

}  // namespace

slso_status run_probe_ff(Handle& h, const double* SX, int64_t s, int64_t d, const int* cexp, const float2* X,
                         const float2* Yff, float2* Wff, float2* vpart, int chunks, float2* Vff, const double* Z,
                         double* eres, cudaStream_t st) {
  const int d_i = static_cast<int>(d);
  probe_w_ff_kernel<<<static_cast<unsigned>(ceil_div(s, 8)), 256, 0, st>>>(SX, s, d_i, cexp, Yff, Wff, h.state);
  SLSO_CHECK_LAUNCH();
  const int64_t rpc = ceil_div(s, chunks);
  const unsigned vb = static_cast<unsigned>(ceil_div(s, rpc));
  probe_v_ff_kernel<<<vb, 256, 0, st>>>(SX, s, d_i, cexp, Wff, rpc, vpart, h.state);
  SLSO_CHECK_LAUNCH();
  probe_vsum_ff_kernel<<<static_cast<unsigned>(ceil_div(d * 4, 256)), 256, 0, st>>>(vpart, static_cast<int>(vb), d_i,
                                                                                    Vff, h.state);
  SLSO_CHECK_LAUNCH();
  probe_u_ff_kernel<<<static_cast<unsigned>(d), 128, 0, st>>>(X, d_i, Vff, Z, eres, h.state);
  SLSO_CHECK_LAUNCH();
  return SLSO_OK;
}

size_t chol_ff_smem() { return sizeof(Smem); }

bool chol_ff_applies(int64_t d) { return d >= 1 && d <= 8192; }

slso_status run_chol_ff(Handle& h, double* L, const int* cexp, int64_t d, float2* A, float2* X, double* Rinv,
                        const double* Pi, int64_t k, const double* Z, double* M, float2* Yff, unsigned int* bar,
                        cudaStream_t st) {
  const size_t smem = sizeof(Smem);
  SLSO_TRY(raise_smem_limit(chol_ff_kernel, smem));
  int occ = 0;
  SLSO_CHECK_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, chol_ff_kernel, kFThreads, smem));
  if (occ < 1) return fail(SLSO_ERR_CUDA, "float-float Cholesky kernel cannot be resident (smem %zu)", smem);
  SLSO_CHECK_CUDA(cudaMemsetAsync(bar, 0, sizeof(unsigned int) * 4, st));
  int d_i = static_cast<int>(d);
  DevState* stp = h.state;
  int k_i = static_cast<int>(k);
  void* args[] = {&L, &cexp, &d_i, &A, &X, &Rinv, &Pi, &k_i, &Z, &M, &Yff, &bar, &stp};
  SLSO_CHECK_CUDA(cudaLaunchCooperativeKernel(reinterpret_cast<void*>(chol_ff_kernel), dim3(h.num_sms), dim3(kFThreads),
                                              args, smem, st));
  note_launch();
  return SLSO_OK;
}

}  // namespace slso
