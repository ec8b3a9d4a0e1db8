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

// x 2^k, the same correctly rounded value as ldexp(x, k), by one multiplication when 2^k is a
// normal float64
__device__ __forceinline__ double times_pow2(double x, int k) {
  if (k >= -1022 && k <= 1023) return x * __longlong_as_double(static_cast<long long>(k + 1023) << 52);
  return ldexp(x, k);
}

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

constexpr int kBarWords = 4;  // count, generation, abort, breakdown

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
  float rh[kFb], rl[kFb], r2h[kFb], r2l[kFb], sh[kFb], sl[kFb];  // pivots: 1/L_jj, 1/L_jj^2, L_jj
  int bad;
};

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

// 1 / sqrt(a), a > 0: y = rsqrtf(a_h) refined once in float32 and once in float-float (Newton for
// the inverse square root, y' = y + y (1 - a y^2) / 2, the residual 1 - a y^2 formed exactly).
__device__ __forceinline__ ff ff_rsqrt(ff a) {
  float y = rsqrtf(a.h);
  y = __fmul_rn(y, __fmaf_rn(-0.5f * a.h, __fmul_rn(y, y), 1.5f));
  const float p = __fmul_rn(y, y);
  const ff y2{p, __fmaf_rn(y, y, -p)};
  const ff ay2 = ff_mul(a, y2);
  const ff res = ff_add(ff{1.f, 0.f}, ff{-ay2.h, -ay2.l});
  return fast_two_sum(y, __fmul_rn(__fmul_rn(0.5f, y), res.h));
}

// 1 / a: y0 ~ 1 / a_h (the hardware's approximate reciprocal, relative error below 2^-22), one
// float32 Newton step y = y0 + y0 (1 - a_h y0) (error about 2^-24), then y + y (1 - a y) in
// float-float with the residual formed exactly (error about 2^-48).
__device__ __forceinline__ float rcp_approx(float x) {
  float y;
  asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}
__device__ __forceinline__ ff ff_recip(ff a) {
  const float y0 = rcp_approx(a.h);
  const float y = __fmaf_rn(y0, __fmaf_rn(-a.h, y0, 1.0f), y0);
  const float p = __fmul_rn(a.h, y);
  const float e = __fmaf_rn(a.h, y, -p);
  const float r = __fsub_rn(__fsub_rn(__fsub_rn(1.0f, p), e), __fmul_rn(a.l, y));
  return fast_two_sum(y, __fmul_rn(y, r));
}

// Pivot j of the diagonal block: r_j^2 = 1 / D_jj (all the column updates need); false on a
// non-positive or non-finite pivot.  r_j = 1 / sqrt(D_jj) and s_j = sqrt(D_jj) follow at the end.
__device__ __forceinline__ bool pivot(Smem& sm, int j, ff piv) {
  if (!(piv.h > 0.f) || !isfinite(piv.h) || !isfinite(piv.l)) return false;
  const ff r2 = ff_recip(piv);
  sm.r2h[j] = r2.h;
  sm.r2l[j] = r2.l;
  sm.sh[j] = piv.h;  // the pivot itself, for the final pass
  sm.sl[j] = piv.l;
  return true;
}

// Step k, part A: L_kk and L_kk^-1 in shared memory (rows / columns beyond d: identity).
// Right-looking over the 32 columns with the column and row scalings deferred: column j of D
// keeps its unscaled values D_ij = L_ij L_jj, row j of the identity block keeps B_j (before the
// division by L_jj), and the updates use r_j^2 = 1 / D_jj:
//   D_im -= D_ij D_mj r_j^2 (j < m <= i),   B_ic -= D_ij B_jc r_j^2 (c <= j)   for rows i > j.
// Warp 0 updates D_(j+1)(j+1) alone and forms pivot j + 1 at once while warps 1-7 do the rest, so
// one barrier per column suffices.  The scalings are applied in one pass at the end.
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
  __syncthreads();
  if (t == 0) sm.bad = pivot(sm, 0, ff{sm.Dh[0][0], sm.Dl[0][0]}) ? 0 : 1;
  __syncthreads();
  if (sm.bad) return false;
  // warps 1-7 own fixed positions (i, m), m <= i, of the 528 in the lower triangle (at most 3 each):
  // while j < m the position is D_im's update, while m <= j < i it is B_im's
  constexpr int kPos = kFb * (kFb + 1) / 2;
  int pi[3], pm[3];
#pragma unroll
  for (int q = 0; q < 3; ++q) {
    const int e = t - 32 + q * (kFThreads - 32);
    pi[q] = -1;
    pm[q] = 0;
    if (t >= 32 && e < kPos) {
      int a = static_cast<int>((sqrtf(8.f * e + 1.f) - 1.f) * 0.5f);
      while ((a + 1) * (a + 2) / 2 <= e) ++a;
      while (a * (a + 1) / 2 > e) --a;
      pi[q] = a;
      pm[q] = e - a * (a + 1) / 2;
    }
  }
  for (int j = 0; j < kFb - 1; ++j) {
    const ff r2{sm.r2h[j], sm.r2l[j]};
    if (t == 0) {
      const ff dij{sm.Dh[j + 1][j], sm.Dl[j + 1][j]};
      const ff v = ff_fms(ff{sm.Dh[j + 1][j + 1], sm.Dl[j + 1][j + 1]}, ff_mul(dij, dij), r2);
      sm.Dh[j + 1][j + 1] = v.h;
      sm.Dl[j + 1][j + 1] = v.l;
      if (!pivot(sm, j + 1, v)) sm.bad = 1;
    } else if (t >= 32) {
      // branch-free over the slots: target -= D_ij src r_j^2 with (target, src) = (D_im, D_mj)
      // while m > j, (B_im, B_jm) while m <= j; inactive slots compute on row 0 and store nothing.
      // Every slot's operands are loaded before any store, so that the three chains interleave
      // (a store through one slot's pointer could otherwise alias the next slot's loads).
      float ah[3], al[3], bh[3], bl[3], ch[3], cl[3];
      float* th[3];
      float* tl[3];
      bool on[3];
#pragma unroll
      for (int q = 0; q < 3; ++q) {
        const int i = pi[q], m = pm[q];
        on[q] = i > j && !(i == j + 1 && m == j + 1);
        const bool dpart = m > j;
        const int ii = on[q] ? i : 0;
        th[q] = dpart ? &sm.Dh[ii][m] : &sm.Ih[ii][m];
        tl[q] = dpart ? &sm.Dl[ii][m] : &sm.Il[ii][m];
        bh[q] = dpart ? sm.Dh[m][j] : sm.Ih[j][m];
        bl[q] = dpart ? sm.Dl[m][j] : sm.Il[j][m];
        ah[q] = sm.Dh[ii][j];
        al[q] = sm.Dl[ii][j];
        ch[q] = *th[q];
        cl[q] = *tl[q];
      }
#pragma unroll
      for (int q = 0; q < 3; ++q) {
        const ff v = ff_fms(ff{ch[q], cl[q]}, ff_mul(ff{ah[q], al[q]}, ff{bh[q], bl[q]}), r2);
        ch[q] = v.h;
        cl[q] = v.l;
      }
#pragma unroll
      for (int q = 0; q < 3; ++q)
        if (on[q]) {
          *th[q] = ch[q];
          *tl[q] = cl[q];
        }
    }
    __syncthreads();
    if (sm.bad) return false;
  }
  // r_j = 1 / sqrt(D_jj) and s_j = sqrt(D_jj) from the pivots (sh, sl hold D_jj)
  if (t < kFb) {
    const ff piv{sm.sh[t], sm.sl[t]};
    const ff r = ff_rsqrt(piv);
    const ff sq = ff_mul(piv, r);
    sm.rh[t] = r.h;
    sm.rl[t] = r.l;
    __syncwarp();
    sm.sh[t] = sq.h;
    sm.sl[t] = sq.l;
  }
  __syncthreads();
  // L_ij = D_ij r_j (i > j), L_jj = s_j; L_kk^-1 row j = B_j r_j
  for (int e = t; e < kFb * kFb; e += kFThreads) {
    const int i = e >> 5, j = e & 31;
    if (i > j) {
      const ff v = ff_mul(ff{sm.Dh[i][j], sm.Dl[i][j]}, ff{sm.rh[j], sm.rl[j]});
      sm.Dh[i][j] = v.h;
      sm.Dl[i][j] = v.l;
    } else if (i == j) {
      sm.Dh[i][j] = sm.sh[j];
      sm.Dl[i][j] = sm.sl[j];
    }
    if (j <= i) {
      const ff v = ff_mul(ff{sm.Ih[i][j], sm.Il[i][j]}, ff{sm.rh[i], sm.rl[i]});
      sm.Ih[i][j] = v.h;
      sm.Il[i][j] = v.l;
    }
  }
  __syncthreads();
  return true;
}

// bar[0..1] grid barrier (count, generation), bar[2] abort flag, bar[3] lookahead breakdown (all
// zeroed by the host before the launch).  Dbuf (2 x 32 x 32 float-float): the next diagonal block's inverse as CTA 0 publishes it.
// Right-hand sides: with the JL matrix Pi (d x k_rhs; none when k_rhs = 0) and the probes Z (d x 4),
// both float64 row-major, Out = X'^T [Pi | Z] (Out_ic = sum over m >= i of X'_mi [Pi | Z]_mc; d x
// (k_rhs + 4) float-float, accumulated row block by row block in part C of the step that finishes
// that block of X') gives M = R^-1 Pi = diag(2^-e) Out[:, :k_rhs] (float64, d x k_rhs row-major;
// st->m_ready = 1) and Y'' = X'^T Z (float-float, d x 4) for the probe check.
__global__ void __launch_bounds__(kFThreads, 1)
    chol_ff_kernel(double* __restrict__ L, const int* __restrict__ cexp, int d, float2* __restrict__ A,
                   float2* __restrict__ X, double* __restrict__ Rinv, const double* __restrict__ Pi, int k_rhs,
                   const double* __restrict__ Z, double* __restrict__ M, float2* __restrict__ Yff, unsigned int* bar,
                   float2* __restrict__ Dbuf, float2* __restrict__ Out, DevState* __restrict__ st) {
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
      const double g = times_pow2(L[e], -cexp[i] - cexp[j]);
      const float h = __double2float_rn(g);
      A[e] = make_float2(h, __double2float_rn(g - static_cast<double>(h)));
    }
    X[e] = make_float2(i == j ? 1.f : 0.f, 0.f);
  }
  for (int64_t e = gtid; e < static_cast<int64_t>(d) * (k_rhs + 4); e += gstride) Out[e] = make_float2(0.f, 0.f);
  auto sync_all = [&]() -> bool {
    if (grid_barrier_ff(bar, bar + 1, abort_flag)) return true;
    if (threadIdx.x == 0) atomicExch(&st->timeout, 7);
    return false;
  };
  if (!sync_all()) return;
  const int nb = (d + kFb - 1) / kFb;
  for (int k = 0; k < nb; ++k) {
    const int k0 = k * kFb;
    // part B's operand for this CTA's first task (panel rows of A, or the row block of B), fetched
    // before the diagonal factorisation so that its latency hides behind it
    const int npanel = nb - k - 1;
    float2 bv[4];
    auto fetch_b = [&](int task) {
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        const int e = threadIdx.x + u * kFThreads, hi = e >> 5, lo = e & 31;
        if (task < npanel) {  // P[lo][hi] = A[r0 + hi][k0 + lo]
          const int r0 = (k + 1 + task) * kFb;
          bv[u] = (r0 + hi < d && k0 + lo < d) ? A[static_cast<int64_t>(r0 + hi) * d + k0 + lo] : make_float2(0.f, 0.f);
        } else {  // Q[hi][lo] = B[k0 + hi][c0 + lo]
          const int c0 = (task - npanel) * kFb;
          bv[u] = (k0 + hi < d && c0 + lo < d) ? X[static_cast<int64_t>(k0 + hi) * d + c0 + lo] : make_float2(0.f, 0.f);
        }
      }
    };
    if (static_cast<int>(blockIdx.x) < nb) fetch_b(blockIdx.x);
    bool good = true;
    if (k == 0) {
      good = factor_diag(sm, A, d, k0);
    } else if (*reinterpret_cast<volatile int*>(bar + 3) != 0) {  // CTA 0's lookahead broke down
      good = false;
    } else if (blockIdx.x != 0) {  // L_kk^-1 as CTA 0 published it during the previous step
      for (int e = threadIdx.x; e < kFb * kFb; e += kFThreads) {
        const float2 v = Dbuf[kFb * kFb + e];
        sm.Ih[e >> 5][e & 31] = v.x;
        sm.Il[e >> 5][e & 31] = v.y;
      }
      __syncthreads();
    }
    if (!good) {
      if (blockIdx.x == 0 && threadIdx.x == 0) {
        st->gram_ok = 0;
        st->gram_resid = CUDART_NAN;
      }
      return;
    }
    // part B: tasks 0 .. nb-k-2 are the panel row blocks I = k+1.., then k+1 column tiles of X_k
    for (int task = blockIdx.x; task < nb; task += gridDim.x) {
      if (task != static_cast<int>(blockIdx.x)) fetch_b(task);
      __syncthreads();
      const bool panel = task < npanel;
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        const int e = threadIdx.x + u * kFThreads, hi = e >> 5, lo = e & 31;
        if (panel) {
          sm.Ph[lo][hi] = bv[u].x;  // P[m][i] = A[r0 + i][k0 + m]
          sm.Pl[lo][hi] = bv[u].y;
          sm.Qh[lo][hi] = sm.Ih[hi][lo];  // Q[m][j] = Li[j][m]
          sm.Ql[lo][hi] = sm.Il[hi][lo];
        } else {
          sm.Qh[hi][lo] = bv[u].x;  // Q[m][j] = B[k0 + m][c0 + j]
          sm.Ql[hi][lo] = bv[u].y;
          sm.Ph[lo][hi] = sm.Ih[hi][lo];  // P[m][i] = Li[i][m]
          sm.Pl[lo][hi] = sm.Il[hi][lo];
        }
      }
      __syncthreads();
      ff acc[4];
#pragma unroll
      for (int q = 0; q < 4; ++q) acc[q] = {0.f, 0.f};
      tile_accumulate(sm, acc);
      const int r0 = panel ? (k + 1 + task) * kFb : k0, c0 = panel ? k0 : (task - npanel) * kFb;
      float2* Y = panel ? A : X;
      const int gi = r0 + (threadIdx.x >> 3);
      if (gi < d)
#pragma unroll
        for (int q = 0; q < 4; ++q) {
          const int gj = c0 + (threadIdx.x & 7) * 4 + q;
          if (gj < d) Y[static_cast<int64_t>(gi) * d + gj] = make_float2(acc[q].h, acc[q].l);
        }
    }
    if (!sync_all()) return;
    if (k == 0 && blockIdx.x == 0)  // L_00 into A: every CTA has read A_00 before the barrier above
      for (int e = threadIdx.x; e < kFb * kFb; e += kFThreads) {
        const int i = e >> 5, j = e & 31;
        if (k0 + i < d && j <= i) A[static_cast<int64_t>(k0 + i) * d + k0 + j] = make_float2(sm.Dh[i][j], sm.Dl[i][j]);
      }
    // part C: lower tiles (I, J) of the trailing matrix, then the (I, c) tiles of B.  Software
    // pipelined: every thread fetches the next task's operand and output elements into registers
    // before it computes the current one, so the L2 latency hides behind the arithmetic.
    const int ntri = npanel * (npanel + 1) / 2;
    const int nbt = npanel * (k + 1);
    const int width = k_rhs + 4, ncb = (width + kFb - 1) / kFb;
    // the right-hand sides: row block k of X' is final after part B, so its share of
    // Out = X'^T [Pi | Z] goes into the tiles (I <= k, Cb) now
    const int ntask = ntri + nbt + (k + 1) * ncb;
    struct Task {
      int r0, c0;
      bool tri, diag, rhs;
    };
    auto decode = [&](int task) {
      Task tk;
      tk.rhs = false;
      if (task >= ntri + nbt) {  // Out tile (I, Cb) += X'[k0.., I block]^T [Pi | Z][k0.., Cb block]
        const int u = task - ntri - nbt;
        tk.r0 = (u / ncb) * kFb;
        tk.c0 = (u % ncb) * kFb;
        tk.tri = false;
        tk.diag = false;
        tk.rhs = true;
      } else if (task < ntri) {
        int a = static_cast<int>((sqrtf(8.f * static_cast<float>(task) + 1.f) - 1.f) * 0.5f);
        while ((a + 1) * (a + 2) / 2 <= task) ++a;
        while (a * (a + 1) / 2 > task) --a;
        const int b = task - a * (a + 1) / 2;
        tk.r0 = (k + 1 + a) * kFb;
        tk.c0 = (k + 1 + b) * kFb;
        tk.tri = true;
        tk.diag = a == b;
      } else {
        const int u = task - ntri;
        tk.r0 = (k + 1 + u / (k + 1)) * kFb;
        tk.c0 = (u % (k + 1)) * kFb;
        tk.tri = false;
        tk.diag = false;
      }
      return tk;
    };
    float2 pv[4], qv[4], ov[4];
    const int ti = threadIdx.x >> 3, tj0 = (threadIdx.x & 7) * 4;
    auto fetch = [&](const Task& tk) {
      if (tk.rhs) {
#pragma unroll
        for (int u = 0; u < 4; ++u) {
          const int e = threadIdx.x + u * kFThreads, hi = e >> 5, lo = e & 31;
          // P[hi][lo] = X'[k0 + hi][r0 + lo];  Q[hi][lo] = [Pi | Z][k0 + hi][c0 + lo] (float64 -> pair)
          pv[u] = (k0 + hi < d && tk.r0 + lo < d) ? X[static_cast<int64_t>(k0 + hi) * d + tk.r0 + lo]
                                                  : make_float2(0.f, 0.f);
          const int r = k0 + hi, c = tk.c0 + lo;
          double v = 0.0;
          if (r < d) v = c < k_rhs ? Pi[static_cast<int64_t>(r) * k_rhs + c] : (c < width ? Z[r * 4 + (c - k_rhs)] : 0.0);
          const float h = __double2float_rn(v);
          qv[u] = make_float2(h, __double2float_rn(v - static_cast<double>(h)));
          const int gi = tk.r0 + ti, gj = tk.c0 + tj0 + u;
          ov[u] = (gi < d && gj < width) ? Out[static_cast<int64_t>(gi) * width + gj] : make_float2(0.f, 0.f);
        }
        return;
      }
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        const int e = threadIdx.x + u * kFThreads, hi = e >> 5, lo = e & 31;
        // P[lo][hi] = L[r0 + hi][k0 + lo]
        pv[u] = (tk.r0 + hi < d && k0 + lo < d) ? A[static_cast<int64_t>(tk.r0 + hi) * d + k0 + lo] : make_float2(0.f, 0.f);
        if (tk.tri)  // Q[lo][hi] = L[c0 + hi][k0 + lo]
          qv[u] = (tk.c0 + hi < d && k0 + lo < d) ? A[static_cast<int64_t>(tk.c0 + hi) * d + k0 + lo] : make_float2(0.f, 0.f);
        else  // Q[hi][lo] = X[k0 + hi][c0 + lo]
          qv[u] = (k0 + hi < d && tk.c0 + lo < d) ? X[static_cast<int64_t>(k0 + hi) * d + tk.c0 + lo] : make_float2(0.f, 0.f);
        // this thread's output elements (row ti, columns tj0 + u)
        const int gi = tk.r0 + ti, gj = tk.c0 + tj0 + u;
        const float2* Y = tk.tri ? A : X;
        ov[u] = (gi < d && gj < d && !(tk.diag && gj > gi)) ? Y[static_cast<int64_t>(gi) * d + gj] : make_float2(0.f, 0.f);
      }
    };
    // CTA 0 takes only task 0, the update of the next diagonal tile, and then factors that block
    // (lookahead); the other CTAs share tasks 1.. round-robin.
    const int cstride = blockIdx.x == 0 ? ntask : static_cast<int>(gridDim.x) - 1;
    int task = blockIdx.x == 0 ? 0 : static_cast<int>(blockIdx.x);
    Task cur{};
    if (task < ntask) {
      cur = decode(task);
      fetch(cur);
    }
    while (task < ntask) {
      __syncthreads();  // the previous task is done with the shared operands
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        const int e = threadIdx.x + u * kFThreads, hi = e >> 5, lo = e & 31;
        if (cur.rhs) {
          sm.Ph[hi][lo] = pv[u].x;
          sm.Pl[hi][lo] = pv[u].y;
          sm.Qh[hi][lo] = qv[u].x;
          sm.Ql[hi][lo] = qv[u].y;
          continue;
        }
        sm.Ph[lo][hi] = pv[u].x;
        sm.Pl[lo][hi] = pv[u].y;
        if (cur.tri) {
          sm.Qh[lo][hi] = qv[u].x;
          sm.Ql[lo][hi] = qv[u].y;
        } else {
          sm.Qh[hi][lo] = qv[u].x;
          sm.Ql[hi][lo] = qv[u].y;
        }
      }
      float2 out[4];
#pragma unroll
      for (int u = 0; u < 4; ++u) out[u] = ov[u];
      __syncthreads();
      const Task now = cur;
      const int next = task + cstride;
      if (next < ntask) {
        cur = decode(next);
        fetch(cur);
      }
      ff acc[4];
#pragma unroll
      for (int q = 0; q < 4; ++q) acc[q] = {0.f, 0.f};
      tile_accumulate(sm, acc);
      const int gi = now.r0 + ti;
      if (now.rhs) {
        if (gi < d)
#pragma unroll
          for (int q = 0; q < 4; ++q) {
            const int gj = now.c0 + tj0 + q;
            if (gj >= width) continue;
            const ff v = ff_add(ff{out[q].x, out[q].y}, acc[q]);
            Out[static_cast<int64_t>(gi) * width + gj] = make_float2(v.h, v.l);
          }
        task = next;
        continue;
      }
      float2* Y = now.tri ? A : X;
      if (gi < d)
#pragma unroll
        for (int q = 0; q < 4; ++q) {
          const int gj = now.c0 + tj0 + q;
          if (gj >= d || (now.diag && gj > gi)) continue;
          const ff v = ff_add(ff{out[q].x, out[q].y}, ff{-acc[q].h, -acc[q].l});
          Y[static_cast<int64_t>(gi) * d + gj] = make_float2(v.h, v.l);
        }
      task = next;
    }
    if (blockIdx.x == 0 && npanel > 0) {
      // block k+1: factor it (its tile was CTA 0's task), write L into A and publish L^-1
      __syncthreads();
      const int k1 = k0 + kFb;
      if (factor_diag(sm, A, d, k1)) {
        for (int e = threadIdx.x; e < kFb * kFb; e += kFThreads) {
          const int i = e >> 5, j = e & 31;
          if (k1 + i < d && j <= i) A[static_cast<int64_t>(k1 + i) * d + k1 + j] = make_float2(sm.Dh[i][j], sm.Dl[i][j]);
          Dbuf[kFb * kFb + e] = make_float2(sm.Ih[i][j], sm.Il[i][j]);
        }
      } else if (threadIdx.x == 0) {
        atomicExch(reinterpret_cast<int*>(bar + 3), 1);
      }
    }
    if (!sync_all()) return;
  }
  // L = D^-1 L' (row i times 2^e_i) and R^-1 = X^T with X = X' D (column i of X' times 2^-e_i)
  for (int64_t e = gtid; e < dd; e += gstride) {
    const int i = static_cast<int>(e / d), j = static_cast<int>(e % d);
    if (j <= i) {
      const float2 a = A[e];
      L[e] = times_pow2(static_cast<double>(a.x) + static_cast<double>(a.y), cexp[i]);
    }
    const float2 x = X[e];  // X'[i][j]: (R^-1)_ji at Rinv[i d + j]
    Rinv[e] = j <= i ? times_pow2(static_cast<double>(x.x) + static_cast<double>(x.y), -cexp[j]) : 0.0;
  }
  // M = R^-1 Pi = diag(2^-e) Out[:, :k] (float64) and Y'' = Out[:, k..k+3] (float-float)
  const int width = k_rhs + 4;
  for (int64_t e = gtid; e < static_cast<int64_t>(d) * width; e += gstride) {
    const int i = static_cast<int>(e / width), c = static_cast<int>(e % width);
    const float2 o = Out[e];
    if (c < k_rhs) M[static_cast<int64_t>(i) * k_rhs + c] = times_pow2(static_cast<double>(o.x) + static_cast<double>(o.y), -cexp[i]);
    else Yff[i * 4 + (c - k_rhs)] = o;
  }
  if (k_rhs > 0 && blockIdx.x == 0 && threadIdx.x == 0) st->m_ready = 1;
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
  const int E = ex - 1075 - e;  // |a 2^-e| = m 2^E, m in [2^52, 2^53)
  if (ex == 0 || E < -126 || E + 29 > 127) {  // zero, subnormal or far below the column's maximum: the float64 path (rare)
    const double v = ldexp(a, -e);
    const float h = __double2float_rn(v);
    return {h, __double2float_rn(v - static_cast<double>(h))};
  }
  // m = hi 2^29 + lo with hi = round(m / 2^29) (at most 2^24) and |lo| <= 2^28, in 32-bit integers;
  // the powers of two are built from their bits (both in float32's normal range here)
  const unsigned int rnd = static_cast<unsigned int>(u >> 28) & 1u;
  const unsigned int hi = (static_cast<unsigned int>(u >> 29) & 0x7FFFFFu) + (1u << 23) + rnd;
  const int lo = static_cast<int>(static_cast<unsigned int>(u) & 0x1FFFFFFFu) - static_cast<int>(rnd << 29);
  float fh = static_cast<float>(hi) * __int_as_float((E + 29 + 127) << 23);
  float fl = static_cast<float>(lo) * __int_as_float((E + 127) << 23);
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
  // blocks of 8 columns per lane: the 8 loads are issued before the arithmetic that uses them;
  // the (S, C) pairs are folded after every block (8 terms)
  for (int j0 = lane; j0 < d; j0 += 32 * 8) {
    double xv[8];
    int ev[8];
#pragma unroll
    for (int u = 0; u < 8; ++u) {
      const int j = j0 + 32 * u;
      xv[u] = j < d ? row[j] : 0.0;
      ev[u] = j < d ? cexp[j] : 0;
    }
#pragma unroll
    for (int u = 0; u < 8; ++u) {
      const int j = j0 + 32 * u;
      if (j < d) {
        const ff a = split_scaled(xv[u], ev[u]);
        const float4 y0 = *reinterpret_cast<const float4*>(Yff + 4 * j);      // probes 0, 1
        const float4 y1 = *reinterpret_cast<const float4*>(Yff + 4 * j + 2);  // probes 2, 3
        dot_term(a.h, a.l, y0.x, y0.y, S[0], C[0]);
        dot_term(a.h, a.l, y0.z, y0.w, S[1], C[1]);
        dot_term(a.h, a.l, y1.x, y1.y, S[2], C[2]);
        dot_term(a.h, a.l, y1.z, y1.w, S[3], C[3]);
      }
    }
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

// vpart[b][j][q] = sum over the rows r of chunk b of SX'[r, j] W[r, q] (float-float).  Grid: chunks
// x column blocks of 256 (one column per thread).
__global__ void __launch_bounds__(256) probe_v_ff_kernel(const double* __restrict__ SX, int64_t s, int d,
                                                         const int* __restrict__ cexp, const float2* __restrict__ Wff,
                                                         int64_t rows_per_chunk, float2* __restrict__ vpart,
                                                         const DevState* __restrict__ st) {
  if (*reinterpret_cast<const volatile int32_t*>(&st->gram_ok) == 0) return;
  const int64_t r0 = blockIdx.x * rows_per_chunk;
  const int64_t r1 = r0 + rows_per_chunk < s ? r0 + rows_per_chunk : s;
  const int j = blockIdx.y * blockDim.x + threadIdx.x;
  if (j < d) {
    const int e = cexp[j];
    float S[4] = {0.f, 0.f, 0.f, 0.f}, C[4] = {0.f, 0.f, 0.f, 0.f};
    ff acc[4] = {{0.f, 0.f}, {0.f, 0.f}, {0.f, 0.f}, {0.f, 0.f}};
    // blocks of 8 rows: the next block's 8 loads are issued before this block's arithmetic;
    // folds after every block
    double xn[8];
#pragma unroll
    for (int u = 0; u < 8; ++u) xn[u] = r0 + u < r1 ? SX[(r0 + u) * d + j] : 0.0;
    for (int64_t rb = r0; rb < r1; rb += 8) {
      double xv[8];
#pragma unroll
      for (int u = 0; u < 8; ++u) xv[u] = xn[u];
#pragma unroll
      for (int u = 0; u < 8; ++u) xn[u] = rb + 8 + u < r1 ? SX[(rb + 8 + u) * d + j] : 0.0;
#pragma unroll
      for (int u = 0; u < 8; ++u) {
        const int64_t r = rb + u;
        if (r < r1) {
          const ff a = split_scaled(xv[u], e);
          const float4 w0 = *reinterpret_cast<const float4*>(Wff + 4 * r);
          const float4 w1 = *reinterpret_cast<const float4*>(Wff + 4 * r + 2);
          dot_term(a.h, a.l, w0.x, w0.y, S[0], C[0]);
          dot_term(a.h, a.l, w0.z, w0.w, S[1], C[1]);
          dot_term(a.h, a.l, w1.x, w1.y, S[2], C[2]);
          dot_term(a.h, a.l, w1.z, w1.w, S[3], C[3]);
        }
      }
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

// V''[j][q] = the chunk partials added in a fixed order: a CTA takes 32 consecutive entries
// e = 4j + q (coalesced), warp w adds the chunks b = w, w + 8, ... and the eight warp sums are
// added in warp order.
__global__ void __launch_bounds__(256) probe_vsum_ff_kernel(const float2* __restrict__ vpart, int chunks, int d,
                                                            float2* __restrict__ V, const DevState* __restrict__ st) {
  if (*reinterpret_cast<const volatile int32_t*>(&st->gram_ok) == 0) return;
  __shared__ float2 part[8][32];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const int e = blockIdx.x * 32 + lane;
  ff v{0.f, 0.f};
  if (e < d * 4) {
    int b = w;
    for (; b + 24 < chunks; b += 32) {  // four loads in flight
      float2 p[4];
#pragma unroll
      for (int u = 0; u < 4; ++u) p[u] = vpart[static_cast<int64_t>(b + 8 * u) * d * 4 + e];
#pragma unroll
      for (int u = 0; u < 4; ++u) v = ff_add(v, ff{p[u].x, p[u].y});
    }
    for (; b < chunks; b += 8) {
      const float2 p = vpart[static_cast<int64_t>(b) * d * 4 + e];
      v = ff_add(v, ff{p.x, p.y});
    }
  }
  part[w][lane] = make_float2(v.h, v.l);
  __syncthreads();
  if (w == 0 && e < d * 4) {
    ff t{0.f, 0.f};
#pragma unroll
    for (int ww = 0; ww < 8; ++ww) t = ff_add(t, ff{part[ww][lane].x, part[ww][lane].y});
    V[e] = make_float2(t.h, t.l);
  }
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
  probe_v_ff_kernel<<<dim3(vb, static_cast<unsigned>(ceil_div(d, 256))), 256, 0, st>>>(SX, s, d_i, cexp, Wff, rpc,
                                                                                       vpart, h.state);
  SLSO_CHECK_LAUNCH();
  probe_vsum_ff_kernel<<<static_cast<unsigned>(ceil_div(d * 4, 32)), 256, 0, st>>>(vpart, static_cast<int>(vb), d_i,
                                                                                   Vff, h.state);
  SLSO_CHECK_LAUNCH();
  probe_u_ff_kernel<<<static_cast<unsigned>(d), 128, 0, st>>>(X, d_i, Vff, Z, eres, h.state);
  SLSO_CHECK_LAUNCH();
  return SLSO_OK;
}

size_t chol_ff_smem() { return sizeof(Smem); }

bool chol_ff_applies(int64_t d) { return d >= 1 && d <= kMaxD; }

slso_status run_chol_ff(Handle& h, double* L, const int* cexp, int64_t d, float2* A, float2* X, double* Rinv,
                        const double* Pi, int64_t k, const double* Z, double* M, float2* Yff, unsigned int* bar,
                        float2* Dbuf, float2* Out, cudaStream_t st) {
  if (h.num_sms < 2) return fail(SLSO_ERR_CUDA, "the float-float Cholesky needs at least two SMs");
  const size_t smem = sizeof(Smem);
  SLSO_TRY(raise_smem_limit(chol_ff_kernel, smem));
  int occ = 0;
  SLSO_CHECK_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, chol_ff_kernel, kFThreads, smem));
  if (occ < 1) return fail(SLSO_ERR_CUDA, "float-float Cholesky kernel cannot be resident (smem %zu)", smem);
  SLSO_CHECK_CUDA(cudaMemsetAsync(bar, 0, sizeof(unsigned int) * kBarWords, st));
  int d_i = static_cast<int>(d);
  DevState* stp = h.state;
  int k_i = static_cast<int>(k);
  void* args[] = {&L, &cexp, &d_i, &A, &X, &Rinv, &Pi, &k_i, &Z, &M, &Yff, &bar, &Dbuf, &Out, &stp};
  SLSO_CHECK_CUDA(cudaLaunchCooperativeKernel(reinterpret_cast<void*>(chol_ff_kernel), dim3(h.num_sms), dim3(kFThreads),
                                              args, smem, st));
  note_launch();
  return SLSO_OK;
}

}  // namespace slso
