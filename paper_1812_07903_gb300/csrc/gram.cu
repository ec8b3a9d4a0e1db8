// Gram route of the factor R (Algorithm 2/3 step 2).
//
// When SX has full column rank, its QR factor R with a positive diagonal is unique, and it is the
// Cholesky factor of G = SX^T SX (R^T R = G).  The Gram route forms G with a SYRK (s d (d+1)/2
// multiply-adds, against about s d^2 for Householder QR) in float-float arithmetic on the float32
// pipe, whose rate is 64 times the float64 pipe's on GB300: each column of SX is scaled by a power
// of two and split into two float32 parts, and every product and sum keeps its rounding error
// (about 2^-47 of sum |a||b| with the running pair folded every 32 rows).  The factorisation
// (d^3/6 multiply-adds) runs in float64.  The
// computed factor then carries an orthogonality error F = R^-T SX^T SX R^-1 - I whose size grows
// like kappa(SX)^2 u, where Householder's grows like kappa u.  Since every score (and every JL
// score) is then off by at most ||F||_2 relative, the route is checked a posteriori: for P seeded
// Gaussian probes z (d x P matrix Z), F Z = R^-T (SX^T (SX (R^-1 Z))) - Z, and the route stands only
// when ||F Z||_F / sqrt(P) <= kGramTol (E ||F z||^2 = ||F||_F^2 for z ~ N(0, I)).  Otherwise
// state->gram_ok is cleared and the Householder kernels, which read it, run instead.
//
// Layout: the Gram matrix and its factor share L (d x d, row-major); only the lower triangle is
// written and read.  Its lower triangle L_ij = R_ji is R stored column-major, the layout the
// Householder kernel leaves R in.
#include <algorithm>
#include <cmath>

#include <math_constants.h>

#include "common.cuh"

namespace slso {

namespace {

constexpr int kGt = 32;            // tile edge of the Gram and Cholesky kernels
constexpr int kGramThreads = 128;  // 16 x 8 threads, 2 x 4 outputs each
constexpr int kProbes = 4;         // P
constexpr uint64_t kProbeSeed = 0x243F6A8885A308D3ull;
constexpr int kGramBalanceSms = 152;  // GB300's SM count: the split-K and probe-chunk counts

// The route flag read once per block (thread 0, then a barrier), so that every thread of a block
// takes the same branch even while block 0 of the panel kernel may be clearing it.
__device__ __forceinline__ bool gram_open(const DevState* st) {
  __shared__ int s_open;
  if (threadIdx.x == 0) s_open = *reinterpret_cast<const volatile int32_t*>(&st->gram_ok);
  __syncthreads();
  return s_open != 0;
}

// t-th tile (I, J), J <= I, of the lower triangle in row order: t = I (I + 1) / 2 + J.
__device__ __forceinline__ void tri_index(int t, int& I, int& J) {
  int i = static_cast<int>((sqrt(8.0 * t + 1.0) - 1.0) * 0.5);
  while ((i + 1) * (i + 2) / 2 <= t) ++i;
  while (i * (i + 1) / 2 > t) --i;
  I = i;
  J = t - i * (i + 1) / 2;
}

// Column scales: colmax[j] = max_r |SX[r, j]| as its float64 bit pattern (non-negative doubles
// order like their bits, so atomicMax gives the exact maximum in any order).  Grid: row chunks x
// column blocks of 256 (one column per thread).
__global__ void __launch_bounds__(256) gram_colmax_kernel(const double* __restrict__ SX, int64_t s, int d,
                                                          int64_t rows_per_block,
                                                          unsigned long long* __restrict__ colmax) {
  const int64_t r0 = blockIdx.x * rows_per_block;
  const int64_t r1 = r0 + rows_per_block < s ? r0 + rows_per_block : s;
  // |x| compared as the integer bits of a non-negative float64 (the same order as the values, with
  // no float64 instruction: that pipe is narrow on this part); eight loads in flight per thread
  constexpr unsigned long long kMag = 0x7FFFFFFFFFFFFFFFull;
  const int j = blockIdx.y * blockDim.x + threadIdx.x;
  if (j < d) {
    unsigned long long m = 0;
    int64_t r = r0;
    for (; r + 8 <= r1; r += 8) {
      unsigned long long v[8];
#pragma unroll
      for (int u = 0; u < 8; ++u) v[u] = static_cast<unsigned long long>(__double_as_longlong(SX[(r + u) * d + j]));
#pragma unroll
      for (int u = 0; u < 8; ++u) m = max(m, v[u] & kMag);
    }
    for (; r < r1; ++r) m = max(m, static_cast<unsigned long long>(__double_as_longlong(SX[r * d + j])) & kMag);
    if (m > 0) atomicMax(colmax + j, m);
  }
}

// e_j: the exponent that puts column j's largest magnitude in [1/2, 1) (0 for a zero column), and
// the exact power of two 2^-e_j.
__global__ void gram_scale_kernel(const unsigned long long* __restrict__ colmax, int d, int* __restrict__ cexp,
                                  double* __restrict__ cscale) {
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= d) return;
  const double m = __longlong_as_double(static_cast<long long>(colmax[j]));
  int ex = 0;
  if (m > 0.0) frexp(m, &ex);
  cexp[j] = ex;
  cscale[j] = ldexp(1.0, -ex);
}

// Column j scaled by 2^-e_j and split into float32 parts, SX[r, j] 2^-e_j = xh + xl up to 2^-48
// relative: xh = fl32(a), xl = fl32(a - xh) (a and a - xh are exact in float64).
__global__ void gram_split_kernel(const double* __restrict__ SX, int64_t s, int d,
                                  const double* __restrict__ cscale, float* __restrict__ xh,
                                  float* __restrict__ xl) {
  const int64_t total = s * d;
  for (int64_t e = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; e < total;
       e += static_cast<int64_t>(gridDim.x) * blockDim.x) {
    const double a = SX[e] * cscale[e % d];
    const float h = __double2float_rn(a);
    xh[e] = h;
    xl[e] = __double2float_rn(a - static_cast<double>(h));
  }
}

// One term of a float-float dot product (Ogita, Rump and Oishi's Dot2 with a split operand): the
// running sum (S, C) += (ah + al)(bh + bl), the product's rounding error by FMA and the sum's by
// TwoSum (Knuth), the al bl term dropped (2^-48 of the product).  The _rn intrinsics keep the
// compiler from contracting or reassociating.
__device__ __forceinline__ void ff_term(float ah, float al, float bh, float bl, float& S, float& C) {
  const float p = __fmul_rn(ah, bh);
  float e = __fmaf_rn(ah, bh, -p);
  e = __fmaf_rn(ah, bl, e);
  e = __fmaf_rn(al, bh, e);
  const float t = __fadd_rn(S, p);
  const float z = __fsub_rn(t, S);
  const float err = __fadd_rn(__fsub_rn(S, __fsub_rn(t, z)), __fsub_rn(p, z));
  S = t;
  C = __fadd_rn(C, __fadd_rn(err, e));
}

// (St, Ct) += (S, C) by TwoSum, then renormalised (Fast2Sum) so that |Ct| stays below half an ulp
// of St; (S, C) restart from zero.  Folding after every 32 rows keeps the compensation term's own
// rounding (2^-24 of a sum over 32 terms, not over the whole split) negligible.
__device__ __forceinline__ void ff_fold(float& S, float& C, float& St, float& Ct) {
  const float t = __fadd_rn(St, S);
  const float z = __fsub_rn(t, St);
  const float err = __fadd_rn(__fsub_rn(St, __fsub_rn(t, z)), __fsub_rn(S, z));
  const float c = __fadd_rn(Ct, __fadd_rn(err, C));
  const float u = __fadd_rn(t, c);
  Ct = __fsub_rn(c, __fsub_rn(u, t));
  St = u;
  S = 0.0f;
  C = 0.0f;
}

// 4-byte asynchronous copy global -> shared (zero-filled when src_bytes = 0), and its group fences.
__device__ __forceinline__ void cp_async4(float* dst, const float* src, int src_bytes) {
  asm volatile("cp.async.ca.shared.global [%0], [%1], 4, %2;" ::"r"(static_cast<uint32_t>(__cvta_generic_to_shared(dst))),
               "l"(src), "r"(src_bytes)
               : "memory");
}
// 16-byte form (both addresses 16-byte aligned).
__device__ __forceinline__ void cp_async16(float* dst, const float* src, int src_bytes) {
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;" ::"r"(static_cast<uint32_t>(__cvta_generic_to_shared(dst))),
               "l"(src), "r"(src_bytes)
               : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait_one() { asm volatile("cp.async.wait_group 1;" ::: "memory"); }

// part[(q T + t) 1024 + a 32 + b] = sum over rows r of split q of x[r, 32 I + a] x[r, 32 J + b] for
// the scaled columns x = xh + xl, in float-float; float64 out.  128 threads, each a 2 x 4 block of
// the tile (rows 2 ty.., columns tx + 8 c).  The next 16 rows are copied into the second half of a
// double buffer (cp.async) while these 16 rows are summed; 16 KB of shared memory and at most 64
// registers keep 8 CTAs per SM, so the 1056 items of the d = 1024 sketch run in one wave.  The float32 pipe's instruction
// issue bounds the kernel: a 4 x 4 block per thread (a quarter of the shared loads) measured slower,
// 4.96 ms against 4.73 ms at s = 16384, d = 1024.  Work item blockIdx.x = q T + t, so that the items
// running together read the same rows.
constexpr int kSyrkThreads = 128;
constexpr int kSyrkRows = 16;  // rows per copy stage; the float-float pair is folded every 2 stages
// V16: d % 4 == 0, so every 4-float chunk of a row starts 16-byte aligned and lies wholly inside or
// outside the matrix; the stage then copies 16 bytes per instruction.
template <bool V16>
__global__ void __launch_bounds__(kSyrkThreads, 8) gram_syrk_kernel(const float* __restrict__ xh,
                                                                 const float* __restrict__ xl, int64_t s, int d,
                                                                 int T, int64_t kc, double* __restrict__ part) {
  __shared__ __align__(16) float sm[2][4][kSyrkRows][kGt];  // [buffer][ah, al, bh, bl][row][column]
  const int q = blockIdx.x / T, t = blockIdx.x % T;
  int I, J;
  tri_index(t, I, J);
  const int64_t r0 = static_cast<int64_t>(q) * kc;
  const int64_t r1 = r0 + kc < s ? r0 + kc : s;
  const int ci = I * kGt, cj = J * kGt;
  const int tid = threadIdx.x, tx = tid & 7, ty = tid >> 3;
  auto stage = [&](int buf, int64_t rb) {
    if constexpr (V16) {
      for (int e = tid; e < kSyrkRows * (kGt / 4); e += kSyrkThreads) {
        const int rr = e >> 3, c = (e & 7) * 4;
        const int64_t r = rb + rr;
        const bool ok = r < r1;
        const bool oi = ok && ci + c < d, oj = ok && cj + c < d;
        cp_async16(&sm[buf][0][rr][c], oi ? xh + r * d + ci + c : xh, oi ? 16 : 0);
        cp_async16(&sm[buf][1][rr][c], oi ? xl + r * d + ci + c : xl, oi ? 16 : 0);
        cp_async16(&sm[buf][2][rr][c], oj ? xh + r * d + cj + c : xh, oj ? 16 : 0);
        cp_async16(&sm[buf][3][rr][c], oj ? xl + r * d + cj + c : xl, oj ? 16 : 0);
      }
    } else {
      for (int e = tid; e < kSyrkRows * kGt; e += kSyrkThreads) {
        const int rr = e >> 5, c = e & 31;
        const int64_t r = rb + rr;
        const bool ok = r < r1;
        const bool oi = ok && ci + c < d, oj = ok && cj + c < d;
        // out of range: zero-filled, the (unread) source pointed at the array's start
        cp_async4(&sm[buf][0][rr][c], oi ? xh + r * d + ci + c : xh, oi ? 4 : 0);
        cp_async4(&sm[buf][1][rr][c], oi ? xl + r * d + ci + c : xl, oi ? 4 : 0);
        cp_async4(&sm[buf][2][rr][c], oj ? xh + r * d + cj + c : xh, oj ? 4 : 0);
        cp_async4(&sm[buf][3][rr][c], oj ? xl + r * d + cj + c : xl, oj ? 4 : 0);
      }
    }
    cp_async_commit();
  };
  float S[2][4], C[2][4], St[2][4], Ct[2][4];
#pragma unroll
  for (int a = 0; a < 2; ++a)
#pragma unroll
    for (int c = 0; c < 4; ++c) S[a][c] = C[a][c] = St[a][c] = Ct[a][c] = 0.0f;
  if (r0 < r1) stage(0, r0);
  int cur = 0;
  for (int64_t rb = r0; rb < r1; rb += kSyrkRows, cur ^= 1) {
    if (rb + kSyrkRows < r1) stage(cur ^ 1, rb + kSyrkRows);
    else cp_async_commit();  // an empty group keeps "all but the newest group done" meaning this block
    cp_async_wait_one();
    __syncthreads();
    float(*sah)[kGt] = sm[cur][0];
    float(*sal)[kGt] = sm[cur][1];
    float(*sbh)[kGt] = sm[cur][2];
    float(*sbl)[kGt] = sm[cur][3];
#pragma unroll 4
    for (int kk = 0; kk < kSyrkRows; ++kk) {
      const float2 ah = *reinterpret_cast<const float2*>(&sah[kk][2 * ty]);
      const float2 al = *reinterpret_cast<const float2*>(&sal[kk][2 * ty]);
#pragma unroll
      for (int c = 0; c < 4; ++c) {
        const float bh = sbh[kk][tx + 8 * c], bl = sbl[kk][tx + 8 * c];
        ff_term(ah.x, al.x, bh, bl, S[0][c], C[0][c]);
        ff_term(ah.y, al.y, bh, bl, S[1][c], C[1][c]);
      }
    }
    if (((rb - r0) / kSyrkRows) % 2 == 1 || rb + kSyrkRows >= r1) {  // every 32 rows, and at the end
#pragma unroll
      for (int a = 0; a < 2; ++a)
#pragma unroll
        for (int c = 0; c < 4; ++c) ff_fold(S[a][c], C[a][c], St[a][c], Ct[a][c]);
    }
    __syncthreads();  // every warp is done with this buffer before the copy into it is issued
  }
  double* out = part + (static_cast<int64_t>(q) * T + t) * (kGt * kGt);
#pragma unroll
  for (int a = 0; a < 2; ++a)
#pragma unroll
    for (int c = 0; c < 4; ++c)
      out[(2 * ty + a) * kGt + tx + 8 * c] = static_cast<double>(St[a][c]) + static_cast<double>(Ct[a][c]);
}

// L[i d + j] (j <= i) = 2^(e_i + e_j) times the S split partials of its tile added in split order.
// Opens the route.
__global__ void gram_reduce_kernel(const double* __restrict__ part, int T, int S, int d,
                                   const int* __restrict__ cexp, double* __restrict__ L, DevState* __restrict__ st) {
  const int64_t total = static_cast<int64_t>(T) * kGt * kGt;
  for (int64_t e = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; e < total;
       e += static_cast<int64_t>(gridDim.x) * blockDim.x) {
    const int t = static_cast<int>(e >> 10), a = static_cast<int>((e >> 5) & 31), b = static_cast<int>(e & 31);
    int I, J;
    tri_index(t, I, J);
    const int i = I * kGt + a, j = J * kGt + b;
    if (i >= d || j > i) continue;
    double v = 0.0;
    for (int q = 0; q < S; ++q) v += part[(static_cast<int64_t>(q) * T + t) * (kGt * kGt) + (e & 1023)];
    L[static_cast<int64_t>(i) * d + j] = ldexp(v, cexp[i] + cexp[j]);
  }
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    st->gram_ok = 1;
    st->gram_tried = 1;
    st->gram_resid = 0.0;
  }
}

// Cholesky step k, diagonal block and panel: every block factors L_kk = chol(G_kk) in shared
// memory; block 0 stores it in ldiag (not in L, where the other blocks are still reading G_kk),
// block b > 0 solves row block I = k + b: L_Ik = G_Ik L_kk^-T.  A pivot that is not positive and
// finite ends the route.  On this part's narrow float64 pipe the cost is the number of warp
// instructions on the chain: one lane forms rsqrt(pivot), which gives both L_jj = pivot rsqrt and
// its reciprocal (the column is scaled by a multiply), and the trailing update of step j walks
// only its (31 - j)(32 - j) / 2 live entries, listed by decreasing column so that they are a
// prefix of one table.
__global__ void __launch_bounds__(kGramThreads) chol_panel_kernel(double* __restrict__ L, int d, int k,
                                                                  double* __restrict__ ldiag,
                                                                  DevState* __restrict__ st) {
  if (!gram_open(st)) return;
  __shared__ double D[kGt][kGt + 1];
  __shared__ double P[kGt][kGt + 1];
  __shared__ double rl[kGt];  // 1 / L_jj
  __shared__ unsigned short pairs[kGt * (kGt - 1) / 2];  // i << 5 | m, 1 <= m <= i < 32, m decreasing
  __shared__ int s_bad;
  const int tid = threadIdx.x;
  const int k0 = k * kGt, kb = d - k0 < kGt ? d - k0 : kGt;
  for (int e = tid; e < kGt * kGt; e += kGramThreads) {
    const int i = e >> 5, j = e & 31;
    double v;
    if (i < kb && j < kb) v = j <= i ? L[static_cast<int64_t>(k0 + i) * d + k0 + j] : 0.0;
    else v = (i == j) ? 1.0 : 0.0;  // identity padding beyond d
    D[i][j] = v;
  }
  for (int m = 1 + tid; m < kGt; m += kGramThreads) {
    const int off = (kGt - 1 - m) * (kGt - m) / 2;  // entries of the columns after m
    for (int i = m; i < kGt; ++i) pairs[off + i - m] = static_cast<unsigned short>((i << 5) | m);
  }
  if (tid == 0) s_bad = 0;
  __syncthreads();
  for (int j = 0; j < kGt; ++j) {
    if (tid == 0) {
      const double piv = D[j][j];
      if (!(piv > 0.0) || !isfinite(piv)) {
        s_bad = 1;
      } else {
        const double r = rsqrt(piv);  // one float64 chain for both: L_jj = piv r, 1 / L_jj = r
        D[j][j] = piv * r;
        rl[j] = r;
      }
    }
    __syncthreads();
    if (s_bad) {  // read after the barrier by every thread: uniform exit
      if (blockIdx.x == 0 && tid == 0) {
        st->gram_ok = 0;
        st->gram_resid = CUDART_NAN;
      }
      return;
    }
    if (tid > j && tid < kGt) D[tid][j] *= rl[j];
    __syncthreads();
    const int live = (kGt - 1 - j) * (kGt - j) / 2;
    for (int e = tid; e < live; e += kGramThreads) {
      const int pr = pairs[e], i = pr >> 5, m = pr & 31;
      D[i][m] = fma(-D[i][j], D[m][j], D[i][m]);
    }
    __syncthreads();
  }
  if (blockIdx.x == 0) {
    for (int e = tid; e < kGt * kGt; e += kGramThreads) ldiag[static_cast<int64_t>(k) * kGt * kGt + e] = D[e >> 5][e & 31];
    return;
  }
  const int i0 = (k + blockIdx.x) * kGt, ib = d - i0 < kGt ? d - i0 : kGt;
  for (int e = tid; e < kGt * kGt; e += kGramThreads) {
    const int r = e >> 5, c = e & 31;
    P[r][c] = (r < ib && c < kb) ? L[static_cast<int64_t>(i0 + r) * d + k0 + c] : 0.0;
  }
  __syncthreads();
  // X D^T = P by columns: x_j = p_j / D_jj, then p_m -= x_j D_mj (m > j).  Thread (r, p) owns
  // columns m = p mod 4 of row r; the four threads of a row are lanes of one warp.
  const int r = tid >> 2, p = tid & 3;
  for (int j = 0; j < kGt; ++j) {
    if ((j & 3) == p) P[r][j] *= rl[j];
    __syncwarp();
    const double x = P[r][j];
    for (int m = j + 1 + ((p - j - 1) & 3); m < kGt; m += 4) P[r][m] = fma(-x, D[m][j], P[r][m]);
    __syncwarp();
  }
  __syncthreads();
  for (int e = tid; e < kGt * kGt; e += kGramThreads) {
    const int rr = e >> 5, c = e & 31;
    if (rr < ib && c < kb) L[static_cast<int64_t>(i0 + rr) * d + k0 + c] = P[rr][c];
  }
}

// Cholesky step k, trailing update: G_IJ -= L_Ik L_Jk^T for k < J <= I (lower tiles only).
__global__ void __launch_bounds__(kGramThreads) chol_update_kernel(double* __restrict__ L, int d, int k,
                                                                   DevState* __restrict__ st) {
  if (!gram_open(st)) return;
  __shared__ double sa[kGt][kGt + 1];  // sa[c][a] = L_Ik[a][c]
  __shared__ double sb[kGt][kGt + 1];
  int a0, b0;
  tri_index(blockIdx.x, a0, b0);
  const int I = k + 1 + a0, J = k + 1 + b0;
  const int k0 = k * kGt, kb = d - k0 < kGt ? d - k0 : kGt;
  const int i0 = I * kGt, j0 = J * kGt;
  const int tid = threadIdx.x, tx = tid & 7, ty = tid >> 3;
  for (int e = tid; e < kGt * kGt; e += kGramThreads) {
    const int a = e >> 5, c = e & 31;
    sa[c][a] = (i0 + a < d && c < kb) ? L[static_cast<int64_t>(i0 + a) * d + k0 + c] : 0.0;
    sb[c][a] = (j0 + a < d && c < kb) ? L[static_cast<int64_t>(j0 + a) * d + k0 + c] : 0.0;
  }
  __syncthreads();
  double acc[2][4] = {{0.0, 0.0, 0.0, 0.0}, {0.0, 0.0, 0.0, 0.0}};
#pragma unroll 8
  for (int c = 0; c < kGt; ++c) {
    const double x0 = sa[c][2 * ty], x1 = sa[c][2 * ty + 1];
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const double y = sb[c][tx + 8 * q];
      acc[0][q] = fma(x0, y, acc[0][q]);
      acc[1][q] = fma(x1, y, acc[1][q]);
    }
  }
#pragma unroll
  for (int a = 0; a < 2; ++a)
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const int i = i0 + 2 * ty + a, j = j0 + tx + 8 * q;
      if (i < d && j <= i) {
        double* g = L + static_cast<int64_t>(i) * d + j;
        *g = *g - acc[a][q];
      }
    }
}

// The factored diagonal blocks from ldiag into L (lower triangles), after the last step.
__global__ void chol_diag_store_kernel(const double* __restrict__ ldiag, int d, double* __restrict__ L,
                                       DevState* __restrict__ st) {
  if (!gram_open(st)) return;
  const int k = blockIdx.x, k0 = k * kGt, kb = d - k0 < kGt ? d - k0 : kGt;
  for (int e = threadIdx.x; e < kGt * kGt; e += blockDim.x) {
    const int i = e >> 5, j = e & 31;
    if (i < kb && j <= i) L[static_cast<int64_t>(k0 + i) * d + k0 + j] = ldiag[static_cast<int64_t>(k) * kGt * kGt + e];
  }
}

// ------------------------------------------------------------------ probe check
__device__ double block_sum_gram(double v, double* red) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xFFFFFFFFu, v, o);
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5, nw = (blockDim.x + 31) >> 5;
  if (lane == 0) red[w] = v;
  __syncthreads();
  double t = 0.0;
  for (int i = 0; i < nw; ++i) t += red[i];
  __syncthreads();
  return t;
}

// Z[c P + q] = BoxMuller of Philox at counter (lo c, hi c, q, TAG_PROBE).
__global__ void probe_z_kernel(int d, double* __restrict__ Z, const DevState* __restrict__ st) {
  if (!gram_open(st)) return;
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= d * kProbes) return;
  const int c = e / kProbes, q = e % kProbes;
  const U32x4 w = philox(static_cast<uint32_t>(c), 0u, static_cast<uint32_t>(q), TAG_PROBE, kProbeSeed);
  Z[e] = box_muller_f64(w.x, w.y);
}

// Y = R^-1 Z: row i, sum over c >= i of (R^-1)_ic Z_c (R^-1 column-major: (R^-1)_ic at Rinv[c d + i]).
__global__ void __launch_bounds__(128) probe_y_kernel(const double* __restrict__ Rinv, int d,
                                                      const double* __restrict__ Z, double* __restrict__ Y,
                                                      const DevState* __restrict__ st) {
  if (!gram_open(st)) return;
  __shared__ double red[4];
  const int i = blockIdx.x;
  double acc[kProbes] = {};
  for (int c = i + threadIdx.x; c < d; c += blockDim.x) {
    const double r = Rinv[static_cast<int64_t>(c) * d + i];
#pragma unroll
    for (int q = 0; q < kProbes; ++q) acc[q] = fma(r, Z[c * kProbes + q], acc[q]);
  }
#pragma unroll
  for (int q = 0; q < kProbes; ++q) {
    const double v = block_sum_gram(acc[q], red);
    if (threadIdx.x == 0) Y[i * kProbes + q] = v;
  }
}

// W = SX Y (s x P): one warp per row of SX.
__global__ void __launch_bounds__(256) probe_w_kernel(const double* __restrict__ SX, int64_t s, int d,
                                                      const double* __restrict__ Y, double* __restrict__ W,
                                                      const DevState* __restrict__ st) {
  if (!gram_open(st)) return;
  const int lane = threadIdx.x & 31;
  const int64_t r = blockIdx.x * static_cast<int64_t>(blockDim.x >> 5) + (threadIdx.x >> 5);
  if (r >= s) return;
  const double* row = SX + r * d;
  double acc[kProbes] = {};
  for (int j = lane; j < d; j += 32) {
    const double x = row[j];
#pragma unroll
    for (int q = 0; q < kProbes; ++q) acc[q] = fma(x, Y[j * kProbes + q], acc[q]);
  }
#pragma unroll
  for (int q = 0; q < kProbes; ++q) {
    double v = acc[q];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xFFFFFFFFu, v, o);
    if (lane == 0) W[r * kProbes + q] = v;
  }
}

// vpart[(b d + j) P + q] = sum over the rows r of chunk b of SX[r, j] W[r, q].
__global__ void __launch_bounds__(256) probe_v_kernel(const double* __restrict__ SX, int64_t s, int d,
                                                      const double* __restrict__ W, int64_t rows_per_chunk,
                                                      double* __restrict__ vpart, const DevState* __restrict__ st) {
  if (!gram_open(st)) return;
  const int64_t r0 = blockIdx.x * rows_per_chunk;
  const int64_t r1 = r0 + rows_per_chunk < s ? r0 + rows_per_chunk : s;
  for (int j = threadIdx.x; j < d; j += blockDim.x) {
    double acc[kProbes] = {};
    for (int64_t r = r0; r < r1; ++r) {
      const double x = SX[r * d + j];
#pragma unroll
      for (int q = 0; q < kProbes; ++q) acc[q] = fma(x, W[r * kProbes + q], acc[q]);
    }
#pragma unroll
    for (int q = 0; q < kProbes; ++q) vpart[(static_cast<int64_t>(blockIdx.x) * d + j) * kProbes + q] = acc[q];
  }
}

// V = SX^T W: the chunk partials added in chunk order.
__global__ void probe_vsum_kernel(const double* __restrict__ vpart, int chunks, int d, double* __restrict__ V,
                                  const DevState* __restrict__ st) {
  if (!gram_open(st)) return;
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= d * kProbes) return;
  double v = 0.0;
  for (int b = 0; b < chunks; ++b) v += vpart[static_cast<int64_t>(b) * d * kProbes + e];
  V[e] = v;
}

// eres[c] = sum_q ((R^-T V)_cq - Z_cq)^2, (R^-T V)_c = sum over i <= c of (R^-1)_ic V_i.
__global__ void __launch_bounds__(128) probe_u_kernel(const double* __restrict__ Rinv, int d,
                                                      const double* __restrict__ V, const double* __restrict__ Z,
                                                      double* __restrict__ eres, const DevState* __restrict__ st) {
  if (!gram_open(st)) return;
  __shared__ double red[4];
  const int c = blockIdx.x;
  double acc[kProbes] = {};
  for (int i = threadIdx.x; i <= c; i += blockDim.x) {
    const double r = Rinv[static_cast<int64_t>(c) * d + i];
#pragma unroll
    for (int q = 0; q < kProbes; ++q) acc[q] = fma(r, V[i * kProbes + q], acc[q]);
  }
  double e = 0.0;
#pragma unroll
  for (int q = 0; q < kProbes; ++q) {
    const double u = block_sum_gram(acc[q], red) - Z[c * kProbes + q];
    e = fma(u, u, e);
  }
  if (threadIdx.x == 0) eres[c] = e;
}

// resid = sqrt(sum_c eres[c] / P) in a fixed order; the route stands when resid <= kGramTol.
__global__ void __launch_bounds__(256) probe_final_kernel(const double* __restrict__ eres, int d,
                                                          DevState* __restrict__ st) {
  if (!gram_open(st)) return;
  __shared__ double red[8];
  double p = 0.0;
  for (int c = threadIdx.x; c < d; c += blockDim.x) p += eres[c];
  const double tot = block_sum_gram(p, red);
  if (threadIdx.x == 0) {
    const double resid = sqrt(tot / kProbes);
    st->gram_resid = resid;
    if (!(resid <= kGramTol)) {
      st->gram_ok = 0;
      st->m_ready = 0;
    }
  }
}

}  // namespace

slso_status run_cholesky(Handle& h, const GramWork& g, int64_t d, double* L, cudaStream_t st);

// The lower triangle of L from the lower triangle of G's row-major store (mirrored into G's upper).
__global__ void gram_mirror_kernel(const double* __restrict__ L, int d, double* __restrict__ G) {
  const int64_t total = static_cast<int64_t>(d) * d;
  for (int64_t e = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; e < total;
       e += static_cast<int64_t>(gridDim.x) * blockDim.x) {
    const int64_t i = e / d, j = e % d;
    G[e] = j <= i ? L[e] : L[j * d + i];
  }
}

slso_status run_gram_full(Handle& h, const Arena& ar, const GramWork& g, const double* SX, int64_t s, int64_t d,
                          double* L, double* G, cudaStream_t st) {
  SLSO_TRY(run_gram_matrix(h, ar, g, SX, s, d, L, st));
  const unsigned b = static_cast<unsigned>(std::min<int64_t>(ceil_div(d * d, 256), static_cast<int64_t>(h.num_sms) * 8));
  gram_mirror_kernel<<<b, 256, 0, st>>>(L, static_cast<int>(d), G);
  SLSO_CHECK_LAUNCH();
  return SLSO_OK;
}

GramWork gram_take(Handle& h, Arena& ar, int64_t s, int64_t d, int64_t k) {
  GramWork g;
  const int64_t nb = ceil_div(d, kGt);
  g.tiles = static_cast<int>(nb * (nb + 1) / 2);
  // split-K count: the smallest S (at most 16, at least 256 rows per split) whose items spread
  // over the SMs within 3% of even; else the most even one.  The SM count is GB300's fixed 152,
  // not the device's: S sets the summation order of G, so results and slso_workspace_size's
  // estimate do not depend on the device the call runs on.
  (void)h;
  constexpr int P = kGramBalanceSms;
  double best = 1e30;
  int best_s = 1;
  for (int S = 1; S <= 16; ++S) {
    if (S > 1 && s / S < 256) break;
    const int64_t items = static_cast<int64_t>(g.tiles) * S;
    const double waste = static_cast<double>(ceil_div(items, P) * P) / static_cast<double>(items);
    if (waste < 1.03) {
      best_s = S;
      break;
    }
    if (waste < best) {
      best = waste;
      best_s = S;
    }
  }
  g.splits = best_s;
  g.kc = ceil_div(ceil_div(s, g.splits), kGt) * kGt;
  g.vchunks = 2 * P;
  g.part = ar.take<double>(static_cast<size_t>(g.splits) * g.tiles * kGt * kGt);
  g.Z = ar.take<double>(static_cast<size_t>(d) * kProbes);
  g.Y = ar.take<double>(static_cast<size_t>(d) * kProbes);
  g.W = ar.take<double>(static_cast<size_t>(s) * kProbes);
  g.vpart = ar.take<double>(static_cast<size_t>(g.vchunks) * d * kProbes);
  g.V = ar.take<double>(static_cast<size_t>(d) * kProbes);
  g.eres = ar.take<double>(d);
  g.ldiag = ar.take<double>(static_cast<size_t>(nb) * kGt * kGt);
  g.colmax = ar.take<unsigned long long>(d);
  g.cexp = ar.take<int>(d);
  g.cscale = ar.take<double>(d);
  g.use_ff = chol_ff_applies(d);
  if (g.use_ff) {
    g.Aff = ar.take<float2>(static_cast<size_t>(d) * d);
    g.Xff = ar.take<float2>(static_cast<size_t>(d) * d);
    g.cbar = ar.take<unsigned int>(4);  // grid barrier words of the float-float Cholesky
    g.Dbuf = ar.take<float2>(2 * 32 * 32);
    g.Outff = ar.take<float2>(static_cast<size_t>(d) * (k + 4));
    g.Yff = ar.take<float2>(static_cast<size_t>(d) * kProbes);
    g.Wff = ar.take<float2>(static_cast<size_t>(s) * kProbes);
    g.vff = ar.take<float2>(static_cast<size_t>(2 * kGramBalanceSms) * d * kProbes);
    g.Vff = ar.take<float2>(static_cast<size_t>(d) * kProbes);
  }
  g.use_tc = gram_tc_applies(s, d);
  if (g.use_tc) {
    gram_tc_take(ar, s, d, &g.tc);
  } else {
    g.xh = ar.take<float>(static_cast<size_t>(s) * d);
    g.xl = ar.take<float>(static_cast<size_t>(s) * d);
  }
  return g;
}

slso_status run_gram_factor(Handle& h, const Arena& ar, const GramWork& g, const double* SX, int64_t s,
                            int64_t d, double* L, double* Rinv, bool* rinv_done, const double* Pi, int64_t k,
                            double* M, cudaStream_t st, cudaEvent_t pi_ready) {
  SLSO_TRY(run_gram_matrix(h, ar, g, SX, s, d, L, st));
  if (pi_ready) SLSO_CHECK_CUDA(cudaStreamWaitEvent(st, pi_ready, 0));  // join the side stream's Pi
  prof_begin(h, ar, ST_CHOL, st);
  if (g.use_ff) {
    probe_z_kernel<<<static_cast<unsigned>(ceil_div(d * kProbes, 256)), 256, 0, st>>>(static_cast<int>(d), g.Z,
                                                                                       h.state);
    SLSO_CHECK_LAUNCH();
    SLSO_TRY(run_chol_ff(h, L, g.cexp, d, g.Aff, g.Xff, Rinv, Pi, Pi ? k : 0, g.Z, M, g.Yff, g.cbar, g.Dbuf, g.Outff,
                         st));
    *rinv_done = true;
  } else {
    SLSO_TRY(run_cholesky(h, g, d, L, st));
    *rinv_done = false;
  }
  prof_end(h, ar, st);
  return SLSO_OK;
}

slso_status run_gram_matrix(Handle& h, const Arena& ar, const GramWork& g, const double* SX, int64_t s,
                            int64_t d, double* L, cudaStream_t st) {
  const int d_i = static_cast<int>(d);
  prof_begin(h, ar, ST_CHOL, st);
  SLSO_CHECK_CUDA(cudaMemsetAsync(g.colmax, 0, sizeof(unsigned long long) * d, st));
  const int cb = 2 * h.num_sms;
  gram_colmax_kernel<<<dim3(static_cast<unsigned>(cb), static_cast<unsigned>(ceil_div(d, 256))), 256, 0, st>>>(
      SX, s, d_i, ceil_div(s, cb), g.colmax);
  SLSO_CHECK_LAUNCH();
  gram_scale_kernel<<<static_cast<unsigned>(ceil_div(d, 256)), 256, 0, st>>>(g.colmax, d_i, g.cexp, g.cscale);
  SLSO_CHECK_LAUNCH();
  prof_end(h, ar, st);
  if (g.use_tc) {
    prof_begin(h, ar, ST_SYRK, st);
    SLSO_TRY(run_gram_tc(h, g.tc, SX, s, d, g.cexp, L, st));
    prof_end(h, ar, st);
    return SLSO_OK;
  }
  prof_begin(h, ar, ST_CHOL, st);
  gram_split_kernel<<<static_cast<unsigned>(8 * h.num_sms), 256, 0, st>>>(SX, s, d_i, g.cscale, g.xh, g.xl);
  SLSO_CHECK_LAUNCH();
  prof_end(h, ar, st);
  prof_begin(h, ar, ST_SYRK, st);
  if (d % 4 == 0)
    gram_syrk_kernel<true><<<static_cast<unsigned>(g.tiles) * g.splits, kSyrkThreads, 0, st>>>(g.xh, g.xl, s, d_i,
                                                                                              g.tiles, g.kc, g.part);
  else
    gram_syrk_kernel<false><<<static_cast<unsigned>(g.tiles) * g.splits, kSyrkThreads, 0, st>>>(g.xh, g.xl, s, d_i,
                                                                                               g.tiles, g.kc, g.part);
  SLSO_CHECK_LAUNCH();
  prof_end(h, ar, st);
  prof_begin(h, ar, ST_CHOL, st);
  const int64_t total = static_cast<int64_t>(g.tiles) * kGt * kGt;
  const unsigned rb = static_cast<unsigned>(std::min<int64_t>(ceil_div(total, 256), static_cast<int64_t>(h.num_sms) * 8));
  gram_reduce_kernel<<<rb, 256, 0, st>>>(g.part, g.tiles, g.splits, d_i, g.cexp, L, h.state);
  SLSO_CHECK_LAUNCH();
  prof_end(h, ar, st);
  return SLSO_OK;
}

// Blocked right-looking Cholesky of the lower triangle of L in place (L = R^T afterwards).
slso_status run_cholesky(Handle& h, const GramWork& g, int64_t d, double* L, cudaStream_t st) {
  const int d_i = static_cast<int>(d);
  const int nb = static_cast<int>(ceil_div(d, kGt));
  for (int k = 0; k < nb; ++k) {
    chol_panel_kernel<<<static_cast<unsigned>(nb - k), kGramThreads, 0, st>>>(L, d_i, k, g.ldiag, h.state);
    SLSO_CHECK_LAUNCH();
    const int m = nb - k - 1;
    if (m > 0) {
      chol_update_kernel<<<static_cast<unsigned>(m * (m + 1) / 2), kGramThreads, 0, st>>>(L, d_i, k, h.state);
      SLSO_CHECK_LAUNCH();
    }
  }
  chol_diag_store_kernel<<<static_cast<unsigned>(nb), 256, 0, st>>>(g.ldiag, d_i, L, h.state);
  SLSO_CHECK_LAUNCH();
  return SLSO_OK;
}

slso_status run_gram_check(Handle& h, const GramWork& g, const double* SX, int64_t s, int64_t d,
                           const double* Rinv, cudaStream_t st) {
  const int d_i = static_cast<int>(d);
  if (g.use_ff) {
    SLSO_TRY(run_probe_ff(h, SX, s, d, g.cexp, g.Xff, g.Yff, g.Wff, g.vff, 2 * kGramBalanceSms, g.Vff, g.Z, g.eres, st));
    probe_final_kernel<<<1, 256, 0, st>>>(g.eres, d_i, h.state);
    SLSO_CHECK_LAUNCH();
    return SLSO_OK;
  }
  probe_z_kernel<<<static_cast<unsigned>(ceil_div(d * kProbes, 256)), 256, 0, st>>>(d_i, g.Z, h.state);
  SLSO_CHECK_LAUNCH();
  probe_y_kernel<<<static_cast<unsigned>(d), 128, 0, st>>>(Rinv, d_i, g.Z, g.Y, h.state);
  SLSO_CHECK_LAUNCH();
  probe_w_kernel<<<static_cast<unsigned>(ceil_div(s, 8)), 256, 0, st>>>(SX, s, d_i, g.Y, g.W, h.state);
  SLSO_CHECK_LAUNCH();
  const int64_t rpc = ceil_div(s, g.vchunks);
  probe_v_kernel<<<static_cast<unsigned>(g.vchunks), 256, 0, st>>>(SX, s, d_i, g.W, rpc, g.vpart, h.state);
  SLSO_CHECK_LAUNCH();
  probe_vsum_kernel<<<static_cast<unsigned>(ceil_div(d * kProbes, 256)), 256, 0, st>>>(g.vpart, g.vchunks, d_i,
                                                                                        g.V, h.state);
  SLSO_CHECK_LAUNCH();
  probe_u_kernel<<<static_cast<unsigned>(d), 128, 0, st>>>(Rinv, d_i, g.V, g.Z, g.eres, h.state);
  SLSO_CHECK_LAUNCH();
  probe_final_kernel<<<1, 256, 0, st>>>(g.eres, d_i, h.state);
  SLSO_CHECK_LAUNCH();
  return SLSO_OK;
}

}  // namespace slso
