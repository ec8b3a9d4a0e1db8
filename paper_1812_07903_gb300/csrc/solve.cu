// FP64 small solve on the sketch (Algorithm 2/3 steps 2-4):
//
//   R      unpivoted Householder QR of SX (s x d), R_jj >= 0          qr_kernel
//   route  ||R||_F ||R^-1||_F < 1e-3/tau certifies rank d, so R^+_tau = R^-1 exactly
//   M      = R^-1 Pi (certified)  or  V_r Sigma_r^-1 U_R,r^T Pi (one-sided Jacobi SVD of R)
//
// All steps run on the GPU in float64.  The route is decided on the device (no host
// synchronisation); kernels of the route not taken return immediately.
//
// QR layout: SX is transposed to column-major A (column l at A + l*s).  A persistent
// cooperative grid owns columns round-robin (column l belongs to CTA l % G); reflector j is
// stored in place (beta on the diagonal, its vector below it, coefficients aside) and announced
// by a per-column ready flag, the only inter-CTA synchronisation (a bounded wait).
//   qr_left_kernel (s <= 16384): left-looking; the owner holds its column in registers, applies
//     every earlier reflector as it is announced (the vector staged in shared memory by one bulk
//     copy), forms its own reflector and stores the column once.  HBM traffic is one read and one
//     write of SX; the float64 FMA pipe and the chain of reflectors bound it.  Forming reflector
//     c sits on that chain (column c+1 waits for it), so it is kept to one pass: the norm is
//     accumulated while reflector c-1 is applied, and the vector is published unscaled,
//     u = den * v with den = alpha - beta, beside g = tau/den and 1/den, so that a consumer
//     applies H = I - tau v v^T as x -= g ((u^T x) / den) u.  Scaling by 1/den in the owner
//     would put one float64 division (or multiply) per row on the chain; on GB300's float64
//     pipe that alone cost more than applying a reflector.
//   qr_kernel (larger s): right-looking; after reflector j is announced each CTA applies it to
//     its own trailing columns, the owner of column j+1 first so the next reflector follows.
#include <algorithm>
#include <cmath>

#include <math_constants.h>

#include "common.cuh"

namespace slso {

namespace {

constexpr int kQrThreads = 512;
constexpr long long kWaitPolls = 1LL << 24;  // ~1-2 s before a wait gives up

__device__ double block_sum(double v, double* red) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xFFFFFFFFu, v, o);
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5, nw = (blockDim.x + 31) >> 5;
  if (lane == 0) red[w] = v;
  __syncthreads();
  if (w == 0) {
    double t = lane < nw ? red[lane] : 0.0;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) t += __shfl_down_sync(0xFFFFFFFFu, t, o);
    if (lane == 0) red[32] = t;
  }
  __syncthreads();
  const double r = red[32];
  __syncthreads();
  return r;
}

__global__ void transpose_kernel(const double* __restrict__ in, int64_t rows, int64_t cols,
                                 double* __restrict__ out, int64_t ldo, const int32_t* skip) {
  // in: rows x cols row-major; out: cols x rows with row stride ldo (= in column-major).
  // Returns at once when skip is set (the Gram route's factor stands).
  if (skip && *skip) return;
  __shared__ double tile[32][33];
  const int64_t r0 = static_cast<int64_t>(blockIdx.y) * 32, c0 = static_cast<int64_t>(blockIdx.x) * 32;
  for (int rr = threadIdx.y; rr < 32; rr += blockDim.y) {
    const int64_t r = r0 + rr, c = c0 + threadIdx.x;
    if (r < rows && c < cols) tile[rr][threadIdx.x] = in[r * cols + c];
  }
  __syncthreads();
  for (int cc = threadIdx.y; cc < 32; cc += blockDim.y) {
    const int64_t c = c0 + cc, r = r0 + threadIdx.x;
    if (r < rows && c < cols) out[c * ldo + r] = tile[threadIdx.x][cc];
  }
}

// Householder reflector of column j (run by every thread of the owning CTA).
__device__ void make_reflector(double* __restrict__ A, int s, int lda, int j, double* __restrict__ taus,
                               int* __restrict__ ready, double* red) {
  double* col = A + static_cast<int64_t>(j) * lda;
  const double alpha = col[j];
  double part = 0.0;
  for (int i = j + 1 + threadIdx.x; i < s; i += blockDim.x) part += col[i] * col[i];
  const double xn2 = block_sum(part, red);
  double tau = 0.0;
  if (xn2 != 0.0) {
    const double norm = sqrt(alpha * alpha + xn2);
    const double beta = alpha >= 0.0 ? -norm : norm;
    tau = (beta - alpha) / beta;
    const double den = alpha - beta;
    for (int i = j + 1 + threadIdx.x; i < s; i += blockDim.x) col[i] = col[i] / den;
    if (threadIdx.x == 0) col[j] = beta;
  }
  if (threadIdx.x == 0) taus[j] = tau;
  __threadfence();
  __syncthreads();
  if (threadIdx.x == 0) atomicExch(&ready[j], 1);
}

template <bool V_SMEM>
__global__ void __launch_bounds__(kQrThreads, 1) qr_kernel(double* __restrict__ A, int s, int lda, int d,
                                                           int* __restrict__ ready,
                                                           double* __restrict__ taus,
                                                           DevState* __restrict__ state) {
  if (state->gram_ok) return;  // the Gram route's factor stands
  extern __shared__ double vs[];
  __shared__ double red[33];
  __shared__ int s_abort;
  const int G = gridDim.x, me = blockIdx.x;
  if (threadIdx.x == 0) s_abort = 0;
  __syncthreads();
  if (me == 0) make_reflector(A, s, lda, 0, taus, ready, red);
  for (int j = 0; j < d; ++j) {
    // smallest column > j owned by this CTA
    int lf = j + 1 + ((me - (j + 1)) % G + G) % G;
    if (lf >= d) break;  // nothing of ours is left to update
    if (threadIdx.x == 0) {
      if (!wait_flag_geq(ready + j, 1, kWaitPolls)) {
        atomicExch(&state->timeout, 1);
        s_abort = 1;
      }
      __threadfence();
    }
    __syncthreads();
    if (s_abort) return;
    const double tau = __ldcg(taus + j);
    const double* vg = A + static_cast<int64_t>(j) * lda;
    if (tau == 0.0) {  // H_j = I
      if (lf == j + 1) make_reflector(A, s, lda, j + 1, taus, ready, red);
      continue;
    }
    if (V_SMEM) {
      for (int i = j + 1 + threadIdx.x; i < s; i += blockDim.x) vs[i] = __ldcg(vg + i);
      __syncthreads();
    }
    for (int l = lf; l < d; l += G) {
      double* col = A + static_cast<int64_t>(l) * lda;
      double part = 0.0;
      for (int i = j + 1 + threadIdx.x; i < s; i += blockDim.x)
        part += (V_SMEM ? vs[i] : __ldcg(vg + i)) * col[i];
      const double c = col[j] + block_sum(part, red);
      const double tc = tau * c;
      for (int i = j + 1 + threadIdx.x; i < s; i += blockDim.x)
        col[i] -= tc * (V_SMEM ? vs[i] : __ldcg(vg + i));
      if (threadIdx.x == 0) col[j] -= tc;
      __syncthreads();
      if (l == j + 1) make_reflector(A, s, lda, j + 1, taus, ready, red);
    }
  }
}

// Left-looking variant for s <= RPT * 256: CTA c % G owns column c; it loads the column into
// registers once (RPT rows per thread, in pairs of adjacent rows so loads and stores are 16
// bytes), applies reflectors 0..c-1 as they are announced, forms reflector c, stores the column
// once and announces ready[c].  Every column is read and written exactly once; the float64 work
// is that of the right-looking loop.  Reflector c needs reflector c-1 applied to column c, so
// reflectors are announced in increasing order and one bounded wait on ready[j] covers
// reflector j.
//
// Storage: R's column c (rows 0..c) goes to Rc (column-major, leading dimension d); column c of
// A becomes reflector c's unscaled vector over all rows: zeros above row c, den = alpha - beta at
// row c, the subcolumn below (and zero padding rows).  A consumer therefore stages the whole
// column and uses it as is: the dot and update passes have no per-row conditions.
//
// Staging: the vector is copied by cp.async.bulk in two fixed halves (rows [0, HA) and [HA, lda))
// completing on full[0], full[1].  After its update pass over a half each warp arrives on that
// half's empty barrier; thread 0 waits for all 8 warps there before copying the next vector into
// it, so the copy of half A overlaps the update of half B and no CTA-wide barrier is needed.
//
// Reductions: on GB300 every float64 warp instruction costs the SM the same ~19 clocks however
// many lanes are active, and a dependent chain of them is latency-bound while the other warps
// wait.  Each reduction therefore writes the 256 per-thread partials to shared memory and lets
// warp 0 alone sum them (8 values per lane, then a 5-level butterfly) and form the scalar.
constexpr int kQrlThreads = 256;
constexpr int64_t kQrlMaxS = 16384;  // s up to this uses qr_left_kernel (64 rows per thread)
constexpr int kQrlWarps = kQrlThreads / 32;
constexpr unsigned long long kMbarTimeoutNs = 2000000000ull;

__device__ __forceinline__ uint32_t smem_addr(const void* p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

// Bounded wait on an mbarrier phase (2 s of %globaltimer); gives up early when *abort is set.
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t* bar, uint32_t parity, const volatile int* abort) {
  uint64_t t0;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t0));
  while (true) {
    uint32_t ok;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}"
        : "=r"(ok) : "r"(smem_addr(bar)), "r"(parity) : "memory");
    if (ok) return true;
    if (abort && *abort) return false;
    uint64_t t1;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t1));
    if (t1 - t0 > kMbarTimeoutNs) return false;
  }
}

__device__ __forceinline__ void mbar_arrive(uint64_t* bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_addr(bar)) : "memory");
}

// Copy rows [lo, hi) of a column into buf (same offsets), completion on bar; an empty range
// only arrives.  lo and hi are even, so the size is a multiple of 16 bytes and both addresses
// are 16-byte aligned.
__device__ __forceinline__ void bulk_stage(double* buf, const double* col, int lo, int hi, uint64_t* bar) {
  if (hi <= lo) {
    mbar_arrive(bar);
    return;
  }
  const uint32_t bytes = static_cast<uint32_t>(hi - lo) * 8u;
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(bar)), "r"(bytes)
               : "memory");
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
          smem_addr(buf + lo)),
      "l"(col + lo), "r"(bytes), "r"(smem_addr(bar))
      : "memory");
}

// Sum of the NT values in red (warp 0 only; every lane returns the same bits): lane l adds
// red[l + 32 m] for m = 0..NT/32-1 in a fixed pairwise tree, then a 5-level butterfly.
template <int NT>
__device__ __forceinline__ double warp0_sum(const double* red) {
  constexpr int NW = NT / 32;
  static_assert(NW == 4 || NW == 8, "4 or 8 warps");
  const int lane = threadIdx.x & 31;
  double v[NW];
#pragma unroll
  for (int m = 0; m < NW; ++m) v[m] = red[lane + 32 * m];
  double t;
  if constexpr (NW == 8) t = ((v[0] + v[1]) + (v[2] + v[3])) + ((v[4] + v[5]) + (v[6] + v[7]));
  else t = (v[0] + v[1]) + (v[2] + v[3]);
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) t += __shfl_xor_sync(0xFFFFFFFFu, t, o);
  return t;
}

// Dot of the staged vector with pairs [Q0, Q1) of the column: two chains (even, odd rows).
template <int NT, int Q0, int Q1>
__device__ __forceinline__ void dot_pairs(const double* a, const double* vsm, int t2, double& p0, double& p1) {
#pragma unroll
  for (int q = Q0; q < Q1; ++q) {
    const double2 w = *reinterpret_cast<const double2*>(vsm + 2 * NT * q + t2);
    p0 = fma(w.x, a[2 * q], p0);
    p1 = fma(w.y, a[2 * q + 1], p1);
  }
}

// a -= tc * u over pairs [Q0, Q1); with NORM also the squared norm of rows > c (x0, x1) and the
// element at row c (to *alpha) of the updated column.
template <int NT, int Q0, int Q1, bool NORM>
__device__ __forceinline__ void axpy_pairs(double* a, const double* vsm, int t2, double tc, int c, int s,
                                           double& x0, double& x1, double* alpha) {
#pragma unroll
  for (int q = Q0; q < Q1; ++q) {
    const int i = 2 * NT * q + t2;
    const double2 w = *reinterpret_cast<const double2*>(vsm + i);
    a[2 * q] = fma(-tc, w.x, a[2 * q]);
    a[2 * q + 1] = fma(-tc, w.y, a[2 * q + 1]);
    if (NORM) {
      if (i > c && i < s) x0 = fma(a[2 * q], a[2 * q], x0);
      if (i + 1 > c && i + 1 < s) x1 = fma(a[2 * q + 1], a[2 * q + 1], x1);
      if (i == c) *alpha = a[2 * q];
      if (i + 1 == c) *alpha = a[2 * q + 1];
    }
  }
}

// Per-column coefficients of the unscaled reflectors: coef[4c] = g = tau/den (0: H_c = I),
// coef[4c+1] = g/den, so that applying reflector j is x -= ((u_j^T x) g/den) u_j.
// Dynamic shared memory: 2 * NT * (RPT/2) doubles.  NT = 256 threads (one CTA per SM), or 128 with
// two CTAs per SM so that one CTA's reductions overlap the other's FMAs (s <= 8192).
template <int RPT, int NT>
__global__ void __launch_bounds__(NT, 256 / NT) qr_left_kernel(double* __restrict__ A, int s, int lda, int d,
                                                                 double* __restrict__ Rc,
                                                                 int* __restrict__ ready,
                                                                 double* __restrict__ coef,
                                                                 DevState* __restrict__ state) {
  static_assert(RPT % 2 == 0, "rows are held in pairs");
  if (state->gram_ok) return;  // the Gram route's factor stands
  constexpr int P = RPT / 2;                    // row pairs per thread
  constexpr int QA = P / 2;                     // pairs in staging half A
  constexpr int HA = 2 * NT * QA;      // rows in staging half A
  constexpr int VROWS = 2 * NT * P;    // rows of the staging buffer (>= lda)
  extern __shared__ __align__(128) double vsm[];
  __shared__ double red[NT];
  __shared__ __align__(8) uint64_t full[2];
  __shared__ __align__(8) uint64_t empty[2];
  __shared__ double s_alpha;
  __shared__ double s_coef[2];  // g, g/den of the staged reflector (written before arming full[0])
  __shared__ double s_scalar;   // warp 0's result of a reduction
  __shared__ double s_form[2];  // den and R_cc of the reflector being formed
  __shared__ int s_abort;       // hint only: lets waits give up early once a wait or stage failed
  const int G = gridDim.x, tid = threadIdx.x, t2 = 2 * threadIdx.x, lane = threadIdx.x & 31;
  for (int i = lda + tid; i < VROWS; i += NT) vsm[i] = 0.0;  // never written by a copy
  if (tid == 0) {
    s_abort = 0;
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_addr(&full[0])));
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_addr(&full[1])));
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(&empty[0])), "r"((NT / 32)));
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(&empty[1])), "r"((NT / 32)));
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  __syncthreads();
  volatile int* abort_flag = &s_abort;
  bool bad = false;   // this thread saw a failed wait; decided on by __syncthreads_or
  uint32_t nvec = 0;  // vectors consumed so far by this CTA (phase of full/empty barriers)
  // thread 0 only
  int known = -1;        // ready[0..known] observed
  uint32_t staged = 0;   // vectors staged so far (both halves issued)
  uint32_t issued[2] = {0u, 0u};  // copies issued per half
  // thread 0: stage reflector j's vector as vector number `staged` (both halves, each after
  // every warp released the previous vector's half)
  auto stage_half = [&](int j, int h) {
    if (*abort_flag) return;
    if (staged > 0 && !mbar_wait_bounded(&empty[h], (staged - 1) & 1u, abort_flag)) {
      bad = true;
      *abort_flag = 1;
      return;
    }
    if (h == 0) {
      if (j > known) {
        if (!wait_flag_geq(ready + j, 1, kWaitPolls)) {
          bad = true;
          *abort_flag = 1;
          return;
        }
        __threadfence();
        asm volatile("fence.proxy.async.global;" ::: "memory");  // generic writes -> bulk-copy reads
        known = j;
      }
      s_coef[0] = __ldcg(coef + 4 * j);
      s_coef[1] = __ldcg(coef + 4 * j + 1);
    }
    const double* src = A + static_cast<int64_t>(j) * lda;
    if (h == 0) bulk_stage(vsm, src, 0, HA, &full[0]);
    else bulk_stage(vsm, src, HA, lda, &full[1]);
    ++issued[h];
    if (h == 1) ++staged;
  };
  // thread 0 on abort: let every issued copy land before the CTA exits (at most one per half
  // is ahead of the consumers)
  auto drain = [&]() {
    for (int h = 0; h < 2; ++h)
      if (issued[h] > nvec) mbar_wait_bounded(&full[h], nvec & 1u, nullptr);
  };
  for (int c = blockIdx.x; c < d; c += G) {
    double* col = A + static_cast<int64_t>(c) * lda;
    double a[RPT];
#pragma unroll
    for (int q = 0; q < P; ++q) {
      const int i = 2 * NT * q + t2;
      double2 v = make_double2(0.0, 0.0);
      if (i < lda) v = __ldcg(reinterpret_cast<const double2*>(col + i));
      a[2 * q] = i < s ? v.x : 0.0;
      a[2 * q + 1] = i + 1 < s ? v.y : 0.0;
    }
    double x0 = 0.0, x1 = 0.0;  // squared norm of rows > c, accumulated with the last update
    bool fused = false;
    if (c > 0 && tid == 0) {
      stage_half(0, 0);
      stage_half(0, 1);
    }
    for (int j = 0; j < c; ++j) {
      const uint32_t par = nvec & 1u;
      if (!mbar_wait_bounded(&full[0], par, abort_flag)) {
        bad = true;
        *abort_flag = 1;
      }
      // the same bits in every thread: written once by thread 0 before it armed full[0]
      const double g = s_coef[0], ginv = s_coef[1];
      double p0 = 0.0, p1 = 0.0;
      if (g != 0.0) dot_pairs<NT, 0, QA>(a, vsm, t2, p0, p1);
      if (!mbar_wait_bounded(&full[1], par, abort_flag)) {
        bad = true;
        *abort_flag = 1;
      }
      if (g != 0.0) {
        dot_pairs<NT, QA, P>(a, vsm, t2, p0, p1);
        red[tid] = p0 + p1;
      }
      // any failed wait or stage so far ends the kernel (uniformly)
      if (__syncthreads_or(bad)) {
        if (tid == 0) {
          atomicExch(&state->timeout, 1);
          drain();
        }
        return;
      }
      const bool last = (j + 1 == c) && g != 0.0;
      if (g != 0.0) {
        if (tid < 32) {
          const double sum = warp0_sum<NT>(red);
          if (lane == 0) s_scalar = sum * ginv;
        }
        __syncthreads();
        const double tc = s_scalar;
        if (last) axpy_pairs<NT, 0, QA, true>(a, vsm, t2, tc, c, s, x0, x1, &s_alpha);
        else axpy_pairs<NT, 0, QA, false>(a, vsm, t2, tc, c, s, x0, x1, &s_alpha);
        __syncwarp();
        if (lane == 0) mbar_arrive(&empty[0]);
        if (tid == 0 && j + 1 < c) stage_half(j + 1, 0);
        if (last) axpy_pairs<NT, QA, P, true>(a, vsm, t2, tc, c, s, x0, x1, &s_alpha);
        else axpy_pairs<NT, QA, P, false>(a, vsm, t2, tc, c, s, x0, x1, &s_alpha);
        __syncwarp();
        if (lane == 0) mbar_arrive(&empty[1]);
      } else {
        __syncwarp();
        if (lane == 0) {
          mbar_arrive(&empty[0]);
          mbar_arrive(&empty[1]);
        }
        if (tid == 0 && j + 1 < c) stage_half(j + 1, 0);
      }
      if (tid == 0 && j + 1 < c) stage_half(j + 1, 1);
      ++nvec;
      fused = last;
    }
    if (!fused) {
#pragma unroll
      for (int q = 0; q < P; ++q) {
        const int i = 2 * NT * q + t2;
        if (i > c && i < s) x0 = fma(a[2 * q], a[2 * q], x0);
        if (i + 1 > c && i + 1 < s) x1 = fma(a[2 * q + 1], a[2 * q + 1], x1);
        if (i == c) s_alpha = a[2 * q];
        if (i + 1 == c) s_alpha = a[2 * q + 1];
      }
    }
    // reflector c: beta = -sign(alpha) ||(alpha, x)||, tau = (beta - alpha) / beta; no
    // reflection when the subcolumn below the diagonal is exactly zero.  The vector's rows
    // (zeros above row c, the subcolumn below it) do not depend on the scalars, so they are
    // stored first; one thread forms the scalars (tau / den = -1 / beta, 1 / den, den) while
    // the stores drain, and R's column is written after the announcement (it is read only
    // after the kernel).
    red[tid] = x0 + x1;
#pragma unroll
    for (int q = 0; q < P; ++q) {
      const int i = 2 * NT * q + t2;
      if (i < lda) {
        double2 v;
        v.x = (i < c) ? 0.0 : a[2 * q];
        v.y = (i + 1 < c) ? 0.0 : a[2 * q + 1];
        *reinterpret_cast<double2*>(col + i) = v;  // row c is rewritten with den below
      }
    }
    __syncthreads();
    if (tid < 32) {
      const double xn2 = warp0_sum<NT>(red);
      if (lane == 0) {
        const double alpha = s_alpha;
        double g = 0.0, inv = 0.0, den = 0.0, rcc = alpha;
        if (xn2 != 0.0) {
          const double norm = sqrt(alpha * alpha + xn2);
          const double beta = alpha >= 0.0 ? -norm : norm;
          den = alpha - beta;
          inv = 1.0 / den;
          g = -1.0 / beta;
          rcc = beta;
        }
        s_form[0] = den;
        s_form[1] = rcc;
        coef[4 * c] = g;
        coef[4 * c + 1] = g * inv;
      }
    }
    __syncthreads();
    if (t2 == (c & (2 * NT - 1)) - (c & 1)) col[c] = s_form[0];  // the thread holding row c
    __threadfence();
    __syncthreads();
    if (tid == 0) atomicExch(&ready[c], 1);
    double* rcol = Rc + static_cast<int64_t>(c) * d;
    const double rcc = s_form[1];
#pragma unroll
    for (int q = 0; q < P; ++q) {
      const int i = 2 * NT * q + t2;
      if (i <= c) rcol[i] = (i == c) ? rcc : a[2 * q];
      if (i + 1 <= c) rcol[i + 1] = (i + 1 == c) ? rcc : a[2 * q + 1];
    }
  }
}

// R (d x d row-major) from the QR storage, rows negated where the diagonal is negative.
__global__ void r_extract_kernel(const double* __restrict__ A, int64_t lda, int64_t d,
                                 double* __restrict__ R, double* __restrict__ sgn) {
  for (int64_t e = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; e < d * d;
       e += static_cast<int64_t>(gridDim.x) * blockDim.x) {
    const int64_t i = e / d, l = e % d;
    const double sg = A[i * lda + i] < 0.0 ? -1.0 : 1.0;
    R[e] = (l >= i) ? sg * A[l * lda + i] : 0.0;
    if (l == 0) sgn[i] = sg;
  }
}

// The upper triangle of R from the right-looking kernel's storage A into Rc (column-major, leading
// dimension d), where the Gram route leaves its factor; only when *guard == 0 (Householder ran).
__global__ void r_to_rc_kernel(const double* __restrict__ A, int64_t lda, int64_t d, double* __restrict__ Rc,
                               const int32_t* guard) {
  if (*guard) return;
  for (int64_t e = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; e < d * d;
       e += static_cast<int64_t>(gridDim.x) * blockDim.x) {
    const int64_t l = e / d, i = e % d;
    if (i <= l) Rc[l * d + i] = A[l * lda + i];
  }
}

// Sum of squares in two fixed-order stages: block b of kSumBlocks sums a contiguous chunk into
// part[b]; the consumer (certify_kernel) adds the kSumBlocks partials in order.
constexpr int kSumBlocks = 64;

__global__ void sumsq_partial_kernel(const double* __restrict__ x, int64_t n, double* __restrict__ part) {
  __shared__ double red[33];
  const int64_t chunk = (n + gridDim.x - 1) / gridDim.x;
  const int64_t lo = blockIdx.x * chunk, hi = lo + chunk < n ? lo + chunk : n;
  double p = 0.0;
  for (int64_t i = lo + threadIdx.x; i < hi; i += blockDim.x) p = fma(x[i], x[i], p);
  const double t = block_sum(p, red);
  if (threadIdx.x == 0) part[blockIdx.x] = t;
}

// Column c of R^-1 (column-major, d x d).  The storage holds R = diag(sgn) Rs with Rs_ik =
// A[k*lda + i] (sgn NULL: all +1), so R^-1 = Rs^-1 diag(sgn) and column c is sgn_c times the
// solution of Rs x = e_c: the back substitution carries no signs, and every inner step is one
// float64 FMA.  It runs in 32-row blocks from the bottom.  One warp solves each 32 x 32 diagonal
// block with shuffles; then all threads subtract that block's contribution from the rows above (a
// GEMV over column-major Rs).  invd[k] = 1 / Rs_kk (inv_diag_kernel), so that the chain of the
// diagonal solve holds a multiply where a float64 division would cost ten times as many
// instructions.  Runs only when guard == nullptr or *guard == want.
__global__ void __launch_bounds__(256) trinv_kernel(const double* __restrict__ A, int64_t lda, int64_t d,
                                                    const double* __restrict__ sgn, const double* __restrict__ invd,
                                                    double* __restrict__ Rinv, const int32_t* guard, int want) {
  if (guard && *guard != want) return;
  extern __shared__ double b[];
  const int c = blockIdx.x;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  for (int i = threadIdx.x; i <= c; i += blockDim.x) b[i] = (i == c) ? 1.0 : 0.0;
  __syncthreads();
  for (int hi = c; hi >= 0; hi -= 32) {
    const int lo = hi >= 31 ? hi - 31 : 0;
    if (warp == 0) {
      const int row = lo + lane;
      double y = (row <= hi) ? b[row] : 0.0;
      for (int k = hi; k >= lo; --k) {
        const int o = k - lo;
        const double xk = __shfl_sync(0xFFFFFFFFu, y, o) * invd[k];
        if (lane == o) y = xk;
        else if (lane < o) y = fma(-A[static_cast<int64_t>(k) * lda + row], xk, y);
      }
      if (row <= hi) b[row] = y;
    }
    __syncthreads();
    for (int i = threadIdx.x; i < lo; i += blockDim.x) {
      double acc = b[i];
      for (int k = lo; k <= hi; ++k) acc = fma(-A[static_cast<int64_t>(k) * lda + i], b[k], acc);
      b[i] = acc;
    }
    __syncthreads();
  }
  const double sc = sgn ? sgn[c] : 1.0;
  for (int64_t i = threadIdx.x; i < d; i += blockDim.x) Rinv[static_cast<int64_t>(c) * d + i] = (i <= c) ? sc * b[i] : 0.0;
}

// invd[k] = 1 / A[k*lda + k] (the unsigned diagonal); only when guard == nullptr or *guard == want.
__global__ void inv_diag_kernel(const double* __restrict__ A, int64_t lda, int64_t d, double* __restrict__ invd,
                                const int32_t* guard, int want) {
  if (guard && *guard != want) return;
  const int64_t k = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x;
  if (k < d) invd[k] = 1.0 / A[k * lda + k];
}

__global__ void certify_kernel(DevState* __restrict__ st, const double* __restrict__ fro2,
                               int64_t d, double tau, int force_svd) {
  double f0 = 0.0, f1 = 0.0;
  for (int b = 0; b < kSumBlocks; ++b) {
    f0 += fro2[b];
    f1 += fro2[kSumBlocks + b];
  }
  const double fr = sqrt(f0), fi = sqrt(f1);
  st->fro_r = fr;
  st->fro_rinv = fi;
  st->tau = tau;
  const bool ok = !force_svd && isfinite(fi) && fi > 0.0 && fr * fi < 1e-3 / tau;
  st->need_svd = ok ? 0 : 1;
  st->gemm_gate = (ok && !st->m_ready) ? 1 : 0;
  if (ok) {
    st->rank = static_cast<int32_t>(d);
    st->sigma_max = CUDART_NAN;
    st->sigma_min_kept = CUDART_NAN;
  }
}

__global__ void pi_kernel(int64_t d, int64_t k, uint64_t seed, double* __restrict__ Pi) {
  const double sk = sqrt(static_cast<double>(k));
  for (int64_t e = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; e < d * k;
       e += static_cast<int64_t>(gridDim.x) * blockDim.x) {
    const int64_t j = e / k, c = e % k;
    const U32x4 w = philox(static_cast<uint32_t>(c), static_cast<uint32_t>(static_cast<uint64_t>(c) >> 32),
                           static_cast<uint32_t>(j), TAG_JL, seed);
    Pi[e] = box_muller_f64(w.x, w.y) / sk;
  }
}

// C (m x n, row-major) = A (m x K) B (K x n); element (r, c) of A at A[r*ars + c*acs].
// Runs only when guard == nullptr or *guard == want.
__global__ void gemm_f64_kernel(int64_t m, int64_t n, int64_t K, const double* __restrict__ A,
                                int64_t ars, int64_t acs, const double* __restrict__ B, int64_t brs,
                                int64_t bcs, double* __restrict__ C, const int32_t* guard, int want) {
  if (guard && *guard != want) return;
  __shared__ double As[32][33], Bs[32][33];
  const int tx = threadIdx.x % 32, ty = threadIdx.x / 32;  // 32 x 8
  const int64_t r0 = static_cast<int64_t>(blockIdx.y) * 32, c0 = static_cast<int64_t>(blockIdx.x) * 32;
  double acc[4] = {0.0, 0.0, 0.0, 0.0};
  for (int64_t k0 = 0; k0 < K; k0 += 32) {
    for (int t = threadIdx.x; t < 32 * 32; t += 256) {
      const int a = t / 32, b = t % 32;
      const int64_t r = r0 + a, kk = k0 + b;
      As[a][b] = (r < m && kk < K) ? A[r * ars + kk * acs] : 0.0;
      const int64_t kb = k0 + a, c = c0 + b;
      Bs[a][b] = (kb < K && c < n) ? B[kb * brs + c * bcs] : 0.0;
    }
    __syncthreads();
#pragma unroll 8
    for (int kk = 0; kk < 32; ++kk) {
      const double bv = Bs[kk][tx];
#pragma unroll
      for (int q = 0; q < 4; ++q) acc[q] = fma(As[ty * 4 + q][kk], bv, acc[q]);
    }
    __syncthreads();
  }
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    const int64_t r = r0 + ty * 4 + q, c = c0 + tx;
    if (r < m && c < n) C[r * n + c] = acc[q];
  }
}

// ------------------------------------------------------------------ one-sided Jacobi SVD of R
__device__ bool grid_barrier(unsigned int* count, volatile unsigned int* gen, unsigned int nblocks,
                             int* abort_flag) {
  __syncthreads();
  __shared__ int s_ok;
  if (threadIdx.x == 0) {
    s_ok = 1;
    const unsigned int g = *gen;
    __threadfence();
    if (atomicAdd(count, 1u) == nblocks - 1) {
      *count = 0;
      __threadfence();
      atomicAdd(const_cast<unsigned int*>(gen), 1u);
    } else {
      long long it = 0;
      while (*gen == g) {
        if (++it > kWaitPolls || *abort_flag) {
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

// W: dp x dp column-major (column p at W + p*dp), V likewise; dp even, column d.. are zero.
// Blocks of kJacobiThreads (two warps, one column pair per warp per round): the d/2 pairs of a
// round spread over every SM (at most a few per SM), since a pair's float64 work is what bounds
// a round.
constexpr int kJacobiThreads = 64;
// d from which the float64 sweeps start from a float32-preconditioned basis, and the float32
// sweep limit (float32 sweeps cost a fraction of float64 ones on this part's narrow FP64 pipe).
constexpr int64_t kJacobiPrecondMin = 64;
constexpr int kJacobiF32Sweeps = 30;

// Rotation test threshold: |w_p . w_q| > tol sqrt(|w_p|^2 |w_q|^2) with tol = sqrt(dp) u, u the unit
// roundoff of T (float64 2^-53, the convergence test of the result; float32 2^-24 for the
// preconditioning sweeps, which the sweep limit bounds).  Measured at d = 784..1024, the float32
// sweeps run to 2^-24 leave fewer float64 sweeps (137 ms against 153 ms at 2^-21, d = 1024).
template <class T> __device__ __forceinline__ T jacobi_tol(int dp);
template <> __device__ __forceinline__ double jacobi_tol<double>(int dp) { return sqrt(static_cast<double>(dp)) * 0x1p-53; }
template <> __device__ __forceinline__ float jacobi_tol<float>(int dp) { return sqrtf(static_cast<float>(dp)) * 0x1p-24f; }

template <class T>
__global__ void __launch_bounds__(kJacobiThreads) jacobi_kernel(T* __restrict__ W, T* __restrict__ V, T* nrm,
                                                     int d, int dp, int max_sweeps,
                                                     DevState* __restrict__ st,
                                                     unsigned int* bar, int* rot_count,
                                                     int require_svd_flag) {
  if (require_svd_flag && st->need_svd == 0) return;
  const int lane = threadIdx.x & 31;
  const int wpb = blockDim.x >> 5;
  const int gw = blockIdx.x * wpb + (threadIdx.x >> 5);
  const int nwarps = gridDim.x * wpb;
  const T tol = jacobi_tol<T>(dp);
  int* abort_flag = reinterpret_cast<int*>(bar + 2);
  for (int p = gw; p < d; p += nwarps) {  // squared column norms, kept exact below
    const T* wp = W + static_cast<int64_t>(p) * dp;
    T a = 0;
    for (int i = lane; i < d; i += 32) a = fma(wp[i], wp[i], a);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) a += __shfl_xor_sync(0xFFFFFFFFu, a, o);
    if (lane == 0) nrm[p] = a;
  }
  if (!grid_barrier(bar, bar + 1, gridDim.x, abort_flag)) {
    if (threadIdx.x == 0) atomicExch(&st->timeout, 2);
    return;
  }
  for (int sweep = 0; sweep < max_sweeps; ++sweep) {
    int local_rot = 0;
    for (int r = 0; r < dp - 1; ++r) {
      for (int kp = gw; kp < dp / 2; kp += nwarps) {
        const int p = (kp == 0) ? 0 : ((r + kp - 1) % (dp - 1)) + 1;
        const int t2 = dp - 1 - kp;
        const int q = ((r + t2 - 1) % (dp - 1)) + 1;
        if (p >= d || q >= d) continue;
        T* wp = W + static_cast<int64_t>(p) * dp;
        T* wq = W + static_cast<int64_t>(q) * dp;
        T g = 0;
        for (int i = lane; i < d; i += 32) g = fma(wp[i], wq[i], g);
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) g += __shfl_xor_sync(0xFFFFFFFFu, g, o);
        const T a = nrm[p], b = nrm[q];
        if (g != T(0) && fabs(g) > tol * sqrt(a * b)) {
          const T zeta = (b - a) / (T(2) * g);
          const T t = copysign(T(1), zeta) / (fabs(zeta) + sqrt(T(1) + zeta * zeta));
          const T c = T(1) / sqrt(T(1) + t * t);
          const T sn = c * t;
          T na = 0, nb = 0;  // norms of the rotated columns, from the stored values
          for (int i = lane; i < d; i += 32) {
            const T x = wp[i], y = wq[i];
            const T xn = c * x - sn * y, yn = sn * x + c * y;
            wp[i] = xn;
            wq[i] = yn;
            na = fma(xn, xn, na);
            nb = fma(yn, yn, nb);
          }
#pragma unroll
          for (int o = 16; o > 0; o >>= 1) {
            na += __shfl_xor_sync(0xFFFFFFFFu, na, o);
            nb += __shfl_xor_sync(0xFFFFFFFFu, nb, o);
          }
          if (lane == 0) {
            nrm[p] = na;
            nrm[q] = nb;
          }
          T* vp = V + static_cast<int64_t>(p) * dp;
          T* vq = V + static_cast<int64_t>(q) * dp;
          for (int i = lane; i < d; i += 32) {
            const T x = vp[i], y = vq[i];
            vp[i] = c * x - sn * y;
            vq[i] = sn * x + c * y;
          }
          ++local_rot;
        }
        __syncwarp();
      }
      if (!grid_barrier(bar, bar + 1, gridDim.x, abort_flag)) {
        if (threadIdx.x == 0) atomicExch(&st->timeout, 2);
        return;
      }
    }
    if (lane == 0 && local_rot) atomicAdd(rot_count + sweep, local_rot);
    if (!grid_barrier(bar, bar + 1, gridDim.x, abort_flag)) {
      if (threadIdx.x == 0) atomicExch(&st->timeout, 2);
      return;
    }
    const int total = *reinterpret_cast<volatile int*>(rot_count + sweep);
    if (blockIdx.x == 0 && threadIdx.x == 0) st->sweeps = sweep + 1;
    if (total == 0) break;
  }
}

// The same sweeps for d <= 32 * CPL with each lane's share of a column pair held in registers
// (CPL elements per column): one load and one store per column per round, with every load of a
// column in flight at once, instead of two dependent passes over L2.  Same pairing, same
// rotation formulas, same convergence test.
template <class T, int CPL>
__global__ void __launch_bounds__(kJacobiThreads) jacobi_reg_kernel(T* __restrict__ W, T* __restrict__ V, T* nrm,
                                                                    int d, int dp, int max_sweeps,
                                                                    DevState* __restrict__ st, unsigned int* bar,
                                                                    int* rot_count, int require_svd_flag) {
  if (require_svd_flag && st->need_svd == 0) return;
  const int lane = threadIdx.x & 31;
  const int wpb = blockDim.x >> 5;
  const int gw = blockIdx.x * wpb + (threadIdx.x >> 5);
  const int nwarps = gridDim.x * wpb;
  const T tol = jacobi_tol<T>(dp);
  int* abort_flag = reinterpret_cast<int*>(bar + 2);
  for (int sweep = 0; sweep < max_sweeps; ++sweep) {
    // squared column norms, recomputed exactly at every sweep's start (the sweep updates them)
    for (int p = gw; p < d; p += nwarps) {
      const T* wp = W + static_cast<int64_t>(p) * dp;
      T a = 0;
#pragma unroll
      for (int e = 0; e < CPL; ++e) {
        const int i = lane + 32 * e;
        const T x = (i < d) ? wp[i] : T(0);
        a = fma(x, x, a);
      }
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) a += __shfl_xor_sync(0xFFFFFFFFu, a, o);
      if (lane == 0) nrm[p] = a;
    }
    if (!grid_barrier(bar, bar + 1, gridDim.x, abort_flag)) {
      if (threadIdx.x == 0) atomicExch(&st->timeout, 2);
      return;
    }
    int local_rot = 0;
    for (int r = 0; r < dp - 1; ++r) {
      for (int kp = gw; kp < dp / 2; kp += nwarps) {
        const int p = (kp == 0) ? 0 : ((r + kp - 1) % (dp - 1)) + 1;
        const int t2 = dp - 1 - kp;
        const int q = ((r + t2 - 1) % (dp - 1)) + 1;
        if (p >= d || q >= d) continue;
        T* wp = W + static_cast<int64_t>(p) * dp;
        T* wq = W + static_cast<int64_t>(q) * dp;
        T x[CPL], y[CPL];
        T* vp = V + static_cast<int64_t>(p) * dp;
        T* vq = V + static_cast<int64_t>(q) * dp;
        // V's columns are fetched with W's when they fit in registers beside them (float32, or
        // float64 with CPL <= 16), so a rotation does not wait for a second round trip to L2
        constexpr bool kPrefetchV = sizeof(T) == 4 || CPL <= 16;
        T u[kPrefetchV ? CPL : 1], v[kPrefetchV ? CPL : 1];
#pragma unroll
        for (int e = 0; e < CPL; ++e) {
          const int i = lane + 32 * e;
          x[e] = (i < d) ? wp[i] : T(0);
          y[e] = (i < d) ? wq[i] : T(0);
          if constexpr (kPrefetchV) {
            u[e] = (i < d) ? vp[i] : T(0);
            v[e] = (i < d) ? vq[i] : T(0);
          }
        }
        T g = 0;
#pragma unroll
        for (int e = 0; e < CPL; ++e) g = fma(x[e], y[e], g);
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) g += __shfl_xor_sync(0xFFFFFFFFu, g, o);
        const T a = nrm[p], b = nrm[q];
        if (g != T(0) && fabs(g) > tol * sqrt(a * b)) {
          const T zeta = (b - a) / (T(2) * g);
          const T t = copysign(T(1), zeta) / (fabs(zeta) + sqrt(T(1) + zeta * zeta));
          const T c = T(1) / sqrt(T(1) + t * t);
          const T sn = c * t;
          // new squared norms: a - t g and b + t g exactly in real arithmetic; taken so when the
          // change is at most half of either norm (no cancellation: a few roundings), else
          // recomputed from the rotated values
          const T tg = t * g;
          if (fabs(tg) <= T(0.5) * fmin(a, b)) {
#pragma unroll
            for (int e = 0; e < CPL; ++e) {
              const int i = lane + 32 * e;
              if (i < d) {
                wp[i] = c * x[e] - sn * y[e];
                wq[i] = sn * x[e] + c * y[e];
              }
            }
            if (lane == 0) {
              nrm[p] = a - tg;
              nrm[q] = b + tg;
            }
          } else {
            T na = 0, nb = 0;  // norms of the rotated columns, from the stored values
#pragma unroll
            for (int e = 0; e < CPL; ++e) {
              const int i = lane + 32 * e;
              const T xn = c * x[e] - sn * y[e], yn = sn * x[e] + c * y[e];
              if (i < d) {
                wp[i] = xn;
                wq[i] = yn;
              }
              na = fma(xn, xn, na);  // padding lanes hold zeros: xn = yn = 0 there
              nb = fma(yn, yn, nb);
            }
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) {
              na += __shfl_xor_sync(0xFFFFFFFFu, na, o);
              nb += __shfl_xor_sync(0xFFFFFFFFu, nb, o);
            }
            if (lane == 0) {
              nrm[p] = na;
              nrm[q] = nb;
            }
          }
          if constexpr (kPrefetchV) {
#pragma unroll
            for (int e = 0; e < CPL; ++e) {
              const int i = lane + 32 * e;
              if (i < d) {
                vp[i] = c * u[e] - sn * v[e];
                vq[i] = sn * u[e] + c * v[e];
              }
            }
          } else {
#pragma unroll
            for (int e = 0; e < CPL; ++e) {
              const int i = lane + 32 * e;
              x[e] = (i < d) ? vp[i] : T(0);
              y[e] = (i < d) ? vq[i] : T(0);
            }
#pragma unroll
            for (int e = 0; e < CPL; ++e) {
              const int i = lane + 32 * e;
              if (i < d) {
                vp[i] = c * x[e] - sn * y[e];
                vq[i] = sn * x[e] + c * y[e];
              }
            }
          }
          ++local_rot;
        }
        __syncwarp();
      }
      if (!grid_barrier(bar, bar + 1, gridDim.x, abort_flag)) {
        if (threadIdx.x == 0) atomicExch(&st->timeout, 2);
        return;
      }
    }
    if (lane == 0 && local_rot) atomicAdd(rot_count + sweep, local_rot);
    if (!grid_barrier(bar, bar + 1, gridDim.x, abort_flag)) {
      if (threadIdx.x == 0) atomicExch(&st->timeout, 2);
      return;
    }
    const int total = *reinterpret_cast<volatile int*>(rot_count + sweep);
    if (blockIdx.x == 0 && threadIdx.x == 0) st->sweeps = sweep + 1;
    if (total == 0) break;
  }
}

// Block one-sided Jacobi for the float32 preconditioning sweeps (d <= 1024): the columns are split
// into nb blocks of kJacobiKB, block pairs follow the same round-robin tournament as columns do,
// and a CTA of 8 warps loads its block pair's W and V columns (2 * kJacobiKB of each) into shared
// memory, rotates every cross pair there (kJacobiKB sub-rounds of kJacobiKB disjoint pairs, one
// pair per warp, __syncthreads between them; in a sweep's first round also the pairs inside each
// block), and writes the columns back.  One grid barrier per block round: nb - 1 per sweep instead
// of dp - 1.  The rotation formulas, norm bookkeeping and convergence test are those of
// jacobi_reg_kernel.
constexpr int kJacobiKB = 8;
constexpr int kJacobiBlockThreads = 256;
constexpr int kCopyCols = 4, kCopyRows = 4;  // 16 loads of each of W and V in flight per thread

// One column pair of a block round, by one warp, on the shared-memory copies: each lane holds its
// CPL elements of both columns in registers (all loads in flight at once, four partial sums),
// as jacobi_reg_kernel does with global memory.
template <int CPL>
__device__ __forceinline__ void jacobi_smem_pair(float* __restrict__ Ws, float* __restrict__ Vs, float* nrm_s,
                                                 int a, int b, int d, float tol, int lane, int* rot) {
  float* wa = Ws + a * d;
  float* wb = Ws + b * d;
  float x[CPL], y[CPL];
#pragma unroll
  for (int e = 0; e < CPL; ++e) {
    const int i = lane + 32 * e;
    x[e] = (i < d) ? wa[i] : 0.0f;
    y[e] = (i < d) ? wb[i] : 0.0f;
  }
  float gp[4] = {0.0f, 0.0f, 0.0f, 0.0f};
#pragma unroll
  for (int e = 0; e < CPL; ++e) gp[e & 3] = fmaf(x[e], y[e], gp[e & 3]);
  float g = (gp[0] + gp[1]) + (gp[2] + gp[3]);
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) g += __shfl_xor_sync(0xFFFFFFFFu, g, o);
  const float x2 = nrm_s[a], y2 = nrm_s[b];
  if (!(g != 0.0f && fabsf(g) > tol * sqrtf(x2 * y2))) return;
  const float zeta = (y2 - x2) / (2.0f * g);
  const float t = copysignf(1.0f, zeta) / (fabsf(zeta) + sqrtf(1.0f + zeta * zeta));
  const float c = 1.0f / sqrtf(1.0f + t * t);
  const float sn = c * t;
  float na[2] = {0.0f, 0.0f}, nb[2] = {0.0f, 0.0f};
#pragma unroll
  for (int e = 0; e < CPL; ++e) {
    const int i = lane + 32 * e;
    const float xn = c * x[e] - sn * y[e], yn = sn * x[e] + c * y[e];
    if (i < d) {
      wa[i] = xn;
      wb[i] = yn;
    }
    na[e & 1] = fmaf(xn, xn, na[e & 1]);  // padding elements are zero
    nb[e & 1] = fmaf(yn, yn, nb[e & 1]);
  }
  float va_[CPL], vb_[CPL];
  float* va = Vs + a * d;
  float* vb = Vs + b * d;
#pragma unroll
  for (int e = 0; e < CPL; ++e) {
    const int i = lane + 32 * e;
    va_[e] = (i < d) ? va[i] : 0.0f;
    vb_[e] = (i < d) ? vb[i] : 0.0f;
  }
#pragma unroll
  for (int e = 0; e < CPL; ++e) {
    const int i = lane + 32 * e;
    if (i < d) {
      va[i] = c * va_[e] - sn * vb_[e];
      vb[i] = sn * va_[e] + c * vb_[e];
    }
  }
  float sa = na[0] + na[1], sb = nb[0] + nb[1];
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    sa += __shfl_xor_sync(0xFFFFFFFFu, sa, o);
    sb += __shfl_xor_sync(0xFFFFFFFFu, sb, o);
  }
  __syncwarp();
  if (lane == 0) {
    nrm_s[a] = sa;
    nrm_s[b] = sb;
    ++*rot;
  }
}

template <int CPL>
__global__ void __launch_bounds__(kJacobiBlockThreads) jacobi_block_f32_kernel(
    float* __restrict__ W, float* __restrict__ V, float* nrm, int d, int dp, int nb, int max_sweeps,
    DevState* __restrict__ st, unsigned int* bar, int* rot_count, int require_svd_flag) {
  if (require_svd_flag && st->need_svd == 0) return;
  extern __shared__ __align__(16) float jsm[];
  float* Ws = jsm;                                  // [2 kJacobiKB][d]
  float* Vs = jsm + 2 * kJacobiKB * d;              // [2 kJacobiKB][d]
  __shared__ float nrm_s[2 * kJacobiKB];
  __shared__ int gcol[2 * kJacobiKB];               // global column of each local column, -1: padding
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const float tol = jacobi_tol<float>(dp);
  int* abort_flag = reinterpret_cast<int*>(bar + 2);
  // squared column norms, kept exact below
  for (int p = blockIdx.x * (kJacobiBlockThreads / 32) + warp; p < d; p += gridDim.x * (kJacobiBlockThreads / 32)) {
    float a = 0.0f;
    for (int i = lane; i < d; i += 32) a = fmaf(W[static_cast<int64_t>(p) * dp + i], W[static_cast<int64_t>(p) * dp + i], a);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) a += __shfl_xor_sync(0xFFFFFFFFu, a, o);
    if (lane == 0) nrm[p] = a;
  }
  if (!grid_barrier(bar, bar + 1, gridDim.x, abort_flag)) {
    if (threadIdx.x == 0) atomicExch(&st->timeout, 2);
    return;
  }
  for (int sweep = 0; sweep < max_sweeps; ++sweep) {
    int local_rot = 0;
    for (int r = 0; r < nb - 1; ++r) {
      for (int kp = blockIdx.x; kp < nb / 2; kp += gridDim.x) {
        const int P = (kp == 0) ? 0 : ((r + kp - 1) % (nb - 1)) + 1;
        const int Q = ((r + (nb - 1 - kp) - 1) % (nb - 1)) + 1;
        if (threadIdx.x < 2 * kJacobiKB) {
          const int lc = threadIdx.x;
          const int gc = (lc < kJacobiKB ? P : Q) * kJacobiKB + (lc % kJacobiKB);
          gcol[lc] = gc < d ? gc : -1;
          nrm_s[lc] = gc < d ? nrm[gc] : 0.0f;
        }
        __syncthreads();
        // copy in: batches of kCopyBatch independent loads per thread, then their stores
        for (int lc0 = 0; lc0 < 2 * kJacobiKB; lc0 += kCopyCols) {
          for (int i0 = threadIdx.x; i0 < d; i0 += kJacobiBlockThreads * kCopyRows) {
            float wv[kCopyCols][kCopyRows], vv[kCopyCols][kCopyRows];
#pragma unroll
            for (int cc = 0; cc < kCopyCols; ++cc) {
              const int gc = gcol[lc0 + cc];
#pragma unroll
              for (int rr = 0; rr < kCopyRows; ++rr) {
                const int i = i0 + rr * kJacobiBlockThreads;
                const bool ok = gc >= 0 && i < d;
                wv[cc][rr] = ok ? W[static_cast<int64_t>(gc) * dp + i] : 0.0f;
                vv[cc][rr] = ok ? V[static_cast<int64_t>(gc) * dp + i] : 0.0f;
              }
            }
#pragma unroll
            for (int cc = 0; cc < kCopyCols; ++cc)
#pragma unroll
              for (int rr = 0; rr < kCopyRows; ++rr) {
                const int i = i0 + rr * kJacobiBlockThreads;
                if (i < d) {
                  Ws[(lc0 + cc) * d + i] = wv[cc][rr];
                  Vs[(lc0 + cc) * d + i] = vv[cc][rr];
                }
              }
          }
        }
        __syncthreads();
        if (r == 0) {
          // pairs inside each block: kJacobiKB - 1 sub-rounds of kJacobiKB / 2 pairs per block
          for (int t = 0; t < kJacobiKB - 1; ++t) {
            const int blk = warp / (kJacobiKB / 2), k = warp % (kJacobiKB / 2);
            const int u = (k == 0) ? 0 : ((t + k - 1) % (kJacobiKB - 1)) + 1;
            const int v = ((t + (kJacobiKB - 1 - k) - 1) % (kJacobiKB - 1)) + 1;
            const int a = blk * kJacobiKB + u, b = blk * kJacobiKB + v;
            if (gcol[a] >= 0 && gcol[b] >= 0) jacobi_smem_pair<CPL>(Ws, Vs, nrm_s, a, b, d, tol, lane, &local_rot);
            __syncthreads();
          }
        }
        for (int t = 0; t < kJacobiKB; ++t) {  // cross pairs (P_i, Q_(i+t) mod KB), one per warp
          const int a = warp, b = kJacobiKB + (warp + t) % kJacobiKB;
          if (gcol[a] >= 0 && gcol[b] >= 0) jacobi_smem_pair<CPL>(Ws, Vs, nrm_s, a, b, d, tol, lane, &local_rot);
          __syncthreads();
        }
        for (int lc = 0; lc < 2 * kJacobiKB; ++lc) {
          const int gc = gcol[lc];
          if (gc < 0) continue;
          for (int i = threadIdx.x; i < d; i += kJacobiBlockThreads) {
            W[static_cast<int64_t>(gc) * dp + i] = Ws[lc * d + i];
            V[static_cast<int64_t>(gc) * dp + i] = Vs[lc * d + i];
          }
        }
        if (threadIdx.x < 2 * kJacobiKB && gcol[threadIdx.x] >= 0) nrm[gcol[threadIdx.x]] = nrm_s[threadIdx.x];
        __syncthreads();
      }
      if (!grid_barrier(bar, bar + 1, gridDim.x, abort_flag)) {
        if (threadIdx.x == 0) atomicExch(&st->timeout, 2);
        return;
      }
    }
    if (lane == 0 && local_rot) atomicAdd(rot_count + sweep, local_rot);
    if (!grid_barrier(bar, bar + 1, gridDim.x, abort_flag)) {
      if (threadIdx.x == 0) atomicExch(&st->timeout, 2);
      return;
    }
    const int total = *reinterpret_cast<volatile int*>(rot_count + sweep);
    if (blockIdx.x == 0 && threadIdx.x == 0) st->sweeps = sweep + 1;
    if (total == 0) break;
  }
}

__global__ void jacobi_init_kernel(const double* __restrict__ R, int64_t d, int64_t dp,
                                   double* __restrict__ W, double* __restrict__ V) {
  for (int64_t e = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; e < dp * dp;
       e += static_cast<int64_t>(gridDim.x) * blockDim.x) {
    const int64_t col = e / dp, row = e % dp;
    W[e] = (row < d && col < d) ? R[row * d + col] : 0.0;
    V[e] = (row == col) ? 1.0 : 0.0;
  }
}

// float32 preconditioning of the Jacobi SVD: W32 = float32(R) (column-major dp x dp), V32 = I.
__global__ void jacobi_init_f32_kernel(const double* __restrict__ R, int64_t d, int64_t dp,
                                       float* __restrict__ W, float* __restrict__ V, const int32_t* guard) {
  if (guard && *guard == 0) return;
  for (int64_t e = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; e < dp * dp;
       e += static_cast<int64_t>(gridDim.x) * blockDim.x) {
    const int64_t col = e / dp, row = e % dp;
    W[e] = (row < d && col < d) ? static_cast<float>(R[row * d + col]) : 0.0f;
    V[e] = (row == col) ? 1.0f : 0.0f;
  }
}

__global__ void f32_to_f64_kernel(const float* __restrict__ a, int64_t n, double* __restrict__ b,
                                  const int32_t* guard) {
  if (guard && *guard == 0) return;
  for (int64_t e = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; e < n;
       e += static_cast<int64_t>(gridDim.x) * blockDim.x)
    b[e] = static_cast<double>(a[e]);
}

// E = G - I in place (G = V0^T V0, d x d row-major).
__global__ void sub_identity_kernel(double* __restrict__ G, int64_t d, const int32_t* guard) {
  if (guard && *guard == 0) return;
  for (int64_t e = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; e < d * d;
       e += static_cast<int64_t>(gridDim.x) * blockDim.x)
    if (e / d == e % d) G[e] -= 1.0;
}

// P = (I + E)^(-1/2) to third order: I - E/2 + 3/8 E^2 - 5/16 E^3, written over E2 (with
// ||E|| ~ 1e-5 the next term is below 1e-19).
__global__ void inv_sqrt_series_kernel(const double* __restrict__ E, double* __restrict__ E2P,
                                       const double* __restrict__ E3, int64_t d, const int32_t* guard) {
  if (guard && *guard == 0) return;
  for (int64_t e = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; e < d * d;
       e += static_cast<int64_t>(gridDim.x) * blockDim.x)
    E2P[e] = ((e / d == e % d) ? 1.0 : 0.0) - 0.5 * E[e] + 0.375 * E2P[e] - 0.3125 * E3[e];
}

// W = W0, V = Q (both d x d row-major) into the column-major dp x dp Jacobi storage.
__global__ void jacobi_init_from_kernel(const double* __restrict__ W0, const double* __restrict__ Q, int64_t d,
                                        int64_t dp, double* __restrict__ W, double* __restrict__ V,
                                        const int32_t* guard) {
  if (guard && *guard == 0) return;
  for (int64_t e = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; e < dp * dp;
       e += static_cast<int64_t>(gridDim.x) * blockDim.x) {
    const int64_t col = e / dp, row = e % dp;
    const bool in = row < d && col < d;
    W[e] = in ? W0[row * d + col] : 0.0;
    V[e] = in ? Q[row * d + col] : ((row == col) ? 1.0 : 0.0);
  }
}

__global__ void colnorm_kernel(const double* __restrict__ W, int64_t d, int64_t dp, double* __restrict__ sig,
                               const int32_t* guard) {
  if (guard && *guard == 0) return;
  const int lane = threadIdx.x & 31;
  const int64_t col = (blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x) >> 5;
  if (col >= d) return;
  double a = 0.0;
  for (int64_t i = lane; i < d; i += 32) a = fma(W[col * dp + i], W[col * dp + i], a);
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) a += __shfl_xor_sync(0xFFFFFFFFu, a, o);
  if (lane == 0) sig[col] = sqrt(a);
}

// Sort sigma descending (ties by column index), rank, and the scaled factors:
//   sigma_out (d), Vout (d x d row-major, column a = v_(a)), Vs = V_r diag(1/sigma_r) (d x d,
//   zero columns beyond r), Ur (d x d, column a = w_(a) / sigma_(a) for a < r, else 0).
__global__ void svd_finalize_kernel(const double* __restrict__ W, const double* __restrict__ Vw,
                                    const double* __restrict__ sig, int64_t d, int64_t dp, double tau,
                                    double* __restrict__ sigma_out, double* __restrict__ Vout,
                                    double* __restrict__ Vs, double* __restrict__ Ur, int* __restrict__ perm,
                                    DevState* __restrict__ st, const int32_t* guard) {
  if (guard && *guard == 0) return;
  // one CTA
  // NaN (from non-finite input) ranks below every number, so the order stays total and perm
  // is a permutation.
  for (int64_t j = threadIdx.x; j < d; j += blockDim.x) {
    int64_t pos = 0;
    const double sj = isnan(sig[j]) ? -1.0 : sig[j];
    for (int64_t i = 0; i < d; ++i) {
      const double si = isnan(sig[i]) ? -1.0 : sig[i];
      pos += (si > sj) || (si == sj && i < j);
    }
    perm[pos] = static_cast<int>(j);
  }
  __syncthreads();
  __shared__ double s_max;
  __shared__ int s_rank;
  if (threadIdx.x == 0) {
    s_max = sig[perm[0]];
    int r = 0;
    if (s_max > 0.0)
      for (int64_t a = 0; a < d; ++a) r += sig[perm[a]] > tau * s_max;
    s_rank = r;
    st->rank = r;
    st->sigma_max = s_max;
    st->sigma_min_kept = r > 0 ? sig[perm[r - 1]] : 0.0;
    st->tau = tau;
  }
  __syncthreads();
  const int r = s_rank;
  for (int64_t e = threadIdx.x; e < d * d; e += blockDim.x) {
    const int64_t i = e / d, a = e % d;
    const int j = perm[a];
    const double sj = sig[j];
    const double v = Vw[static_cast<int64_t>(j) * dp + i];
    if (Vout) Vout[e] = v;
    if (Vs) Vs[e] = (a < r) ? v / sj : 0.0;
    if (Ur) Ur[e] = (a < r) ? W[static_cast<int64_t>(j) * dp + i] / sj : 0.0;
  }
  if (sigma_out)
    for (int64_t a = threadIdx.x; a < d; a += blockDim.x) sigma_out[a] = sig[perm[a]];
}

__global__ void copy_guarded_kernel(const double* __restrict__ a, int64_t n, double* __restrict__ b,
                                    const int32_t* guard, int want) {
  if (guard && *guard != want) return;
  for (int64_t i = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; i < n;
       i += static_cast<int64_t>(gridDim.x) * blockDim.x)
    b[i] = a[i];
}

// Rinv column-major -> row-major copy (M for k = 0 on the certified route)
__global__ void rinv_rowmajor_kernel(const double* __restrict__ Rinv, int64_t d, double* __restrict__ M,
                                     const int32_t* guard) {
  if (guard && *guard != 0) return;
  for (int64_t e = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; e < d * d;
       e += static_cast<int64_t>(gridDim.x) * blockDim.x) {
    const int64_t i = e / d, c = e % d;
    M[e] = Rinv[c * d + i];
  }
}

int grid1d(int64_t n, const Handle& h) {
  return static_cast<int>(std::max<int64_t>(1, std::min<int64_t>(ceil_div(n, 256), 8LL * h.num_sms)));
}

template <class T>
void* jacobi_fn(int64_t d) {
  if (d <= 256) return reinterpret_cast<void*>(jacobi_reg_kernel<T, 8>);
  if (d <= 512) return reinterpret_cast<void*>(jacobi_reg_kernel<T, 16>);
  if (d <= 1024) return reinterpret_cast<void*>(jacobi_reg_kernel<T, 32>);
  return reinterpret_cast<void*>(jacobi_kernel<T>);
}

slso_status launch_gemm(int64_t m, int64_t n, int64_t K, const double* A, int64_t ars, int64_t acs,
                        const double* B, int64_t brs, int64_t bcs, double* C, const int32_t* guard,
                        int want, cudaStream_t st) {
  dim3 grid(static_cast<unsigned>(ceil_div(n, 32)), static_cast<unsigned>(ceil_div(m, 32)));
  gemm_f64_kernel<<<grid, 256, 0, st>>>(m, n, K, A, ars, acs, B, brs, bcs, C, guard, want);
  SLSO_CHECK_LAUNCH();
  return SLSO_OK;
}

}  // namespace

slso_status run_solve(Handle& h, Arena& ar, const double* SX, int64_t s, int64_t d, double tau,
                      int64_t k, uint64_t seed_pi, int mode, SolveOut* out, cudaStream_t st, bool gram) {
  gram = gram && mode == 0;
  const int64_t dp = d + (d & 1);
  const int64_t kk = (k > 0) ? k : d;
  const int64_t lda = s + (s & 1);  // even: 16-byte aligned columns for the bulk copies
  double* A = ar.take<double>(static_cast<size_t>(lda) * d);
  int* ready = ar.take<int>(d);
  double* taus = ar.take<double>(4 * d);  // qr_kernel: tau per column; qr_left_kernel: 4 coefficients
  double* Rc = ar.take<double>(static_cast<size_t>(d) * d);  // qr_left_kernel: R column-major
  double* R = ar.take<double>(static_cast<size_t>(d) * d);
  double* sgn = ar.take<double>(d);
  double* invd = ar.take<double>(d);  // 1 / R_kk for trinv_kernel
  double* fro2 = ar.take<double>(2 * kSumBlocks);
  double* Rinv = (mode == 0) ? ar.take<double>(static_cast<size_t>(d) * d) : nullptr;
  double* Pi = (k > 0) ? ar.take<double>(static_cast<size_t>(d) * k) : nullptr;
  double* W = ar.take<double>(static_cast<size_t>(dp) * dp);
  double* Vw = ar.take<double>(static_cast<size_t>(dp) * dp);
  double* sig = ar.take<double>(d);
  int* perm = ar.take<int>(d);
  unsigned int* bar = ar.take<unsigned int>(4);
  double* nrm = ar.take<double>(dp);  // Jacobi squared column norms (float32 phase uses the first half)
  int* rot = ar.take<int>(64);
  double* Vs = (mode == 0) ? ar.take<double>(static_cast<size_t>(d) * d) : nullptr;
  double* Ur = (mode == 0 && k > 0) ? ar.take<double>(static_cast<size_t>(d) * d) : nullptr;
  double* Z = (mode == 0 && k > 0) ? ar.take<double>(static_cast<size_t>(d) * k) : nullptr;
  double* M = (mode == 0) ? ar.take<double>(static_cast<size_t>(d) * kk) : nullptr;
  double* sigma_out = (mode == 1) ? ar.take<double>(d) : nullptr;
  double* Vout = (mode == 1) ? ar.take<double>(static_cast<size_t>(d) * d) : nullptr;
  const bool precond = d >= kJacobiPrecondMin;
  float* W32 = precond ? ar.take<float>(static_cast<size_t>(dp) * dp) : nullptr;
  float* V32 = precond ? ar.take<float>(static_cast<size_t>(dp) * dp) : nullptr;
  double* Gm = precond ? ar.take<double>(static_cast<size_t>(d) * d) : nullptr;
  double* E2 = precond ? ar.take<double>(static_cast<size_t>(d) * d) : nullptr;
  double* Qm = precond ? ar.take<double>(static_cast<size_t>(d) * d) : nullptr;
  double* W0m = precond ? ar.take<double>(static_cast<size_t>(d) * d) : nullptr;
  const GramWork gw = gram ? gram_take(h, ar, s, d, k) : GramWork{};
  if (ar.measure()) return SLSO_OK;

  // ---- Gram route (leverage only): R = chol(SX^T SX) into Rc, R^-1, probe check.  gram_ok
  // stays 1 when it stands; the Householder kernels below then return at once.
  int32_t* gram_ok = &h.state->gram_ok;
  // trinv_kernel keeps one column of R^-1 in shared memory: d doubles, above 48 KB for d > 6144
  SLSO_TRY(raise_smem_limit(trinv_kernel, sizeof(double) * d));
  if (gram) {
    cudaEvent_t pi_ready = nullptr;
    if (k > 0) {  // M = R^-1 Pi comes out of the float-float factorisation
      // Pi on the side stream, overlapping the Gram product; joined before the factorisation
      cudaStream_t ps = st;
      if (h.side) {
        SLSO_CHECK_CUDA(cudaEventRecord(h.ev_fork, st));
        SLSO_CHECK_CUDA(cudaStreamWaitEvent(h.side, h.ev_fork, 0));
        ps = h.side;
      }
      pi_kernel<<<grid1d(d * k, h), 256, 0, ps>>>(d, k, seed_pi, Pi);
      SLSO_CHECK_LAUNCH();
      if (h.side) {
        SLSO_CHECK_CUDA(cudaEventRecord(h.ev_ready[0], ps));
        pi_ready = h.ev_ready[0];
      }
    }
    bool rinv_done = false;
    SLSO_TRY(run_gram_factor(h, ar, gw, SX, s, d, Rc, Rinv, &rinv_done, Pi, k, M, st, pi_ready));
    prof_begin(h, ar, ST_CHOL, st);
    if (!rinv_done) {
      inv_diag_kernel<<<static_cast<unsigned>(ceil_div(d, 256)), 256, 0, st>>>(Rc, d, d, invd, gram_ok, 1);
      SLSO_CHECK_LAUNCH();
      trinv_kernel<<<static_cast<unsigned>(d), 256, sizeof(double) * d, st>>>(Rc, d, d, nullptr, invd, Rinv, gram_ok, 1);
      SLSO_CHECK_LAUNCH();
    }
    SLSO_TRY(run_gram_check(h, gw, SX, s, d, Rinv, st));
    prof_end(h, ar, st);
  }

  // ---- QR
  prof_begin(h, ar, ST_SOLVE, st);
  {
    dim3 g(static_cast<unsigned>(ceil_div(d, 32)), static_cast<unsigned>(ceil_div(s, 32)));
    transpose_kernel<<<g, dim3(32, 8), 0, st>>>(SX, s, d, A, lda, gram ? gram_ok : nullptr);
    SLSO_CHECK_LAUNCH();
  }
  SLSO_CHECK_CUDA(cudaMemsetAsync(ready, 0, sizeof(int) * d, st));
  {
    // left-looking register-resident kernel when a column fits in registers, else right-looking
    void* fn = nullptr;
    int threads = kQrlThreads;
    int rpt = 0;  // rows per thread of the left-looking kernel (0: right-looking)
    // the smallest instantiated row count per thread that covers s (padding rows cost FMAs).  For
    // 2048 < s <= 8192 and at least 4 columns per SM, CTAs of 128 threads (twice the rows per
    // thread) run two per SM, so that one CTA's reductions and barriers overlap the other's FMAs
    // (measured: 6144 x 3072 141 -> 117 ms, 4096 x 1024 14.6 -> 12.4 ms); with fewer columns the
    // reflector chain dominates and sharing an SM slows it (8192 x 128 1.5 -> 1.9 ms), so one
    // 256-thread CTA per SM is used.
    if (s > 2048 && s <= 8192 && d >= 4 * static_cast<int64_t>(h.num_sms)) {
      static const int kRpts128[] = {24, 32, 40, 48, 56, 64};
      for (int r : kRpts128)
        if (s <= static_cast<int64_t>(128) * r) {
          rpt = r;
          break;
        }
      threads = 128;
      switch (rpt) {
        case 24: fn = reinterpret_cast<void*>(qr_left_kernel<24, 128>); break;
        case 32: fn = reinterpret_cast<void*>(qr_left_kernel<32, 128>); break;
        case 40: fn = reinterpret_cast<void*>(qr_left_kernel<40, 128>); break;
        case 48: fn = reinterpret_cast<void*>(qr_left_kernel<48, 128>); break;
        case 56: fn = reinterpret_cast<void*>(qr_left_kernel<56, 128>); break;
        default: fn = reinterpret_cast<void*>(qr_left_kernel<64, 128>); break;
      }
    } else {
      static const int kRpts[] = {2, 4, 8, 16, 24, 32, 40, 48, 56, 64};
      for (int r : kRpts)
        if (s <= static_cast<int64_t>(kQrlThreads) * r) {
          rpt = r;
          break;
        }
      switch (rpt) {
        case 2: fn = reinterpret_cast<void*>(qr_left_kernel<2, 256>); break;
        case 4: fn = reinterpret_cast<void*>(qr_left_kernel<4, 256>); break;
        case 8: fn = reinterpret_cast<void*>(qr_left_kernel<8, 256>); break;
        case 16: fn = reinterpret_cast<void*>(qr_left_kernel<16, 256>); break;
        case 24: fn = reinterpret_cast<void*>(qr_left_kernel<24, 256>); break;
        case 32: fn = reinterpret_cast<void*>(qr_left_kernel<32, 256>); break;
        case 40: fn = reinterpret_cast<void*>(qr_left_kernel<40, 256>); break;
        case 48: fn = reinterpret_cast<void*>(qr_left_kernel<48, 256>); break;
        case 56: fn = reinterpret_cast<void*>(qr_left_kernel<56, 256>); break;
        case 64: fn = reinterpret_cast<void*>(qr_left_kernel<64, 256>); break;
        default: break;
      }
    }
    size_t smem = sizeof(double) * threads * rpt;  // staging buffer of the left-looking kernel
    if (rpt == 0) {
      const bool vsm = s <= 24576;
      smem = vsm ? sizeof(double) * s : 0;
      fn = vsm ? reinterpret_cast<void*>(qr_kernel<true>) : reinterpret_cast<void*>(qr_kernel<false>);
      threads = kQrThreads;
    }
    SLSO_TRY(raise_smem_limit(fn, smem));
    int occ = 0;
    SLSO_CHECK_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, fn, threads, smem));
    if (occ < 1) return fail(SLSO_ERR_CUDA, "QR kernel cannot be resident (smem %zu)", smem);
    int G = static_cast<int>(std::min<int64_t>(static_cast<int64_t>(h.num_sms) * (rpt ? std::min(occ, 256 / threads) : 1),
                                               d));
    int s_i = static_cast<int>(s), lda_i = static_cast<int>(lda), d_i = static_cast<int>(d);
    void* args_left[] = {&A, &s_i, &lda_i, &d_i, &Rc, &ready, &taus, &h.state};
    void* args_right[] = {&A, &s_i, &lda_i, &d_i, &ready, &taus, &h.state};
    prof_end(h, ar, st);
    prof_begin(h, ar, ST_QR, st);
    SLSO_CHECK_CUDA(cudaLaunchCooperativeKernel(fn, dim3(G), dim3(threads), rpt ? args_left : args_right, smem, st));
    note_launch();
    prof_end(h, ar, st);
    prof_begin(h, ar, ST_SOLVE, st);
  }
  // the upper triangle of R: Rc (leading dimension d) from the left-looking kernel or the Gram
  // route, else in A
  const bool left = s <= kQrlMaxS;
  if (gram && !left) {
    r_to_rc_kernel<<<grid1d(d * d, h), 256, 0, st>>>(A, lda, d, Rc, gram_ok);
    SLSO_CHECK_LAUNCH();
  }
  const double* Rsrc = (left || gram) ? Rc : A;
  const int64_t ldr = (left || gram) ? d : lda;
  r_extract_kernel<<<grid1d(d * d, h), 256, 0, st>>>(Rsrc, ldr, d, R, sgn);
  SLSO_CHECK_LAUNCH();
  sumsq_partial_kernel<<<kSumBlocks, 256, 0, st>>>(R, d * d, fro2);
  SLSO_CHECK_LAUNCH();

  // ---- certified route: R^-1
  if (mode == 0) {
    // on the Gram route R^-1 is already in Rinv (computed for the probe check)
    inv_diag_kernel<<<static_cast<unsigned>(ceil_div(d, 256)), 256, 0, st>>>(Rsrc, ldr, d, invd,
                                                                             gram ? gram_ok : nullptr, 0);
    SLSO_CHECK_LAUNCH();
    trinv_kernel<<<static_cast<unsigned>(d), 256, sizeof(double) * d, st>>>(Rsrc, ldr, d, sgn, invd, Rinv,
                                                                            gram ? gram_ok : nullptr, 0);
    SLSO_CHECK_LAUNCH();
    sumsq_partial_kernel<<<kSumBlocks, 256, 0, st>>>(Rinv, d * d, fro2 + kSumBlocks);
    SLSO_CHECK_LAUNCH();
  }
  certify_kernel<<<1, 1, 0, st>>>(h.state, fro2, d, tau, mode == 1 ? 1 : 0);
  SLSO_CHECK_LAUNCH();
  const int32_t* need = &h.state->need_svd;
  if (k > 0 && !gram) {
    pi_kernel<<<grid1d(d * k, h), 256, 0, st>>>(d, k, seed_pi, Pi);
    SLSO_CHECK_LAUNCH();
  }
  if (mode == 0) {
    if (k > 0) {
      // M = R^-1 Pi, R^-1 column-major: element (i, m) at Rinv[m*d + i]; skipped when the
      // float-float Gram route has written M already (gemm_gate, set by certify_kernel)
      SLSO_TRY(launch_gemm(d, k, d, Rinv, 1, d, Pi, k, 1, M, &h.state->gemm_gate, 1, st));
    } else {
      rinv_rowmajor_kernel<<<grid1d(d * d, h), 256, 0, st>>>(Rinv, d, M, need);
      SLSO_CHECK_LAUNCH();
    }
  }

  // ---- SVD route (always for mode 1)
  const int32_t* guard = (mode == 0) ? need : nullptr;
  auto launch_jacobi = [&](void* jfn, void* Wp, void* Vp, int max_sweeps) -> slso_status {
    void* np_ = nrm;
    SLSO_CHECK_CUDA(cudaMemsetAsync(bar, 0, sizeof(unsigned int) * 4, st));
    SLSO_CHECK_CUDA(cudaMemsetAsync(rot, 0, sizeof(int) * 64, st));
    int occ = 0;
    SLSO_CHECK_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, jfn, kJacobiThreads, 0));
    const int warps_needed = static_cast<int>(dp / 2);
    int G = static_cast<int>(std::min<int64_t>(static_cast<int64_t>(h.num_sms) * occ,
                                               ceil_div(warps_needed, kJacobiThreads / 32)));
    G = std::max(G, 1);
    int d_i = static_cast<int>(d), dp_i = static_cast<int>(dp), sweeps = max_sweeps, req = (mode == 0) ? 1 : 0;
    DevState* stp = h.state;
    void* args[] = {&Wp, &Vp, &np_, &d_i, &dp_i, &sweeps, &stp, &bar, &rot, &req};
    SLSO_CHECK_CUDA(cudaLaunchCooperativeKernel(jfn, dim3(G), dim3(kJacobiThreads), args, 0, st));
    note_launch();
    return SLSO_OK;
  };
  if (precond) {
    // float32 sweeps from R give V32 (orthogonal to ~1e-6); V0 = float64(V32) made orthogonal in
    // float64, Q = V0 (V0^T V0)^(-1/2) by the third-order series; the float64 sweeps then start
    // from W0 = R Q, V = Q, whose columns are already orthogonal to float32 accuracy.
    jacobi_init_f32_kernel<<<grid1d(dp * dp, h), 256, 0, st>>>(R, d, dp, W32, V32, guard);
    SLSO_CHECK_LAUNCH();
    if (d <= 1024) {
      // block sweeps: one grid barrier per block round
      SLSO_CHECK_CUDA(cudaMemsetAsync(bar, 0, sizeof(unsigned int) * 4, st));
      SLSO_CHECK_CUDA(cudaMemsetAsync(rot, 0, sizeof(int) * 64, st));
      int nb = static_cast<int>(ceil_div(d, kJacobiKB));
      nb += nb & 1;
      const size_t smem = sizeof(float) * 2 * 2 * kJacobiKB * static_cast<size_t>(d);
      void* fn = d <= 256 ? reinterpret_cast<void*>(jacobi_block_f32_kernel<8>)
                 : d <= 512 ? reinterpret_cast<void*>(jacobi_block_f32_kernel<16>)
                            : reinterpret_cast<void*>(jacobi_block_f32_kernel<32>);
      SLSO_TRY(raise_smem_limit(fn, smem));
      int occ = 0;
      SLSO_CHECK_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, fn, kJacobiBlockThreads, smem));
      if (occ < 1) return fail(SLSO_ERR_CUDA, "block Jacobi kernel cannot be resident (smem %zu)", smem);
      int G = static_cast<int>(std::min<int64_t>(static_cast<int64_t>(h.num_sms) * occ, nb / 2));
      G = std::max(G, 1);
      float* nrm32 = reinterpret_cast<float*>(nrm);
      int d_i = static_cast<int>(d), dp_i = static_cast<int>(dp), sweeps = kJacobiF32Sweeps,
          req = (mode == 0) ? 1 : 0;
      DevState* stp = h.state;
      void* args[] = {&W32, &V32, &nrm32, &d_i, &dp_i, &nb, &sweeps, &stp, &bar, &rot, &req};
      SLSO_CHECK_CUDA(cudaLaunchCooperativeKernel(fn, dim3(G), dim3(kJacobiBlockThreads), args, smem, st));
      note_launch();
    } else {
      SLSO_TRY(launch_jacobi(jacobi_fn<float>(d), W32, V32, kJacobiF32Sweeps));
    }
    double* V0 = W;  // dp x dp column-major; W is rewritten below
    f32_to_f64_kernel<<<grid1d(dp * dp, h), 256, 0, st>>>(V32, dp * dp, V0, guard);
    SLSO_CHECK_LAUNCH();
    const int want = 1;
    SLSO_TRY(launch_gemm(d, d, d, V0, dp, 1, V0, 1, dp, Gm, guard, want, st));  // G = V0^T V0
    sub_identity_kernel<<<grid1d(d * d, h), 256, 0, st>>>(Gm, d, guard);
    SLSO_CHECK_LAUNCH();
    SLSO_TRY(launch_gemm(d, d, d, Gm, d, 1, Gm, d, 1, E2, guard, want, st));  // E^2
    SLSO_TRY(launch_gemm(d, d, d, E2, d, 1, Gm, d, 1, Qm, guard, want, st));  // E^3 (in Q's buffer)
    inv_sqrt_series_kernel<<<grid1d(d * d, h), 256, 0, st>>>(Gm, E2, Qm, d, guard);
    SLSO_CHECK_LAUNCH();
    SLSO_TRY(launch_gemm(d, d, d, V0, 1, dp, E2, d, 1, Qm, guard, want, st));  // Q = V0 P
    SLSO_TRY(launch_gemm(d, d, d, R, d, 1, Qm, d, 1, W0m, guard, want, st));   // W0 = R Q
    jacobi_init_from_kernel<<<grid1d(dp * dp, h), 256, 0, st>>>(W0m, Qm, d, dp, W, Vw, guard);
    SLSO_CHECK_LAUNCH();
  } else {
    jacobi_init_kernel<<<grid1d(dp * dp, h), 256, 0, st>>>(R, d, dp, W, Vw);
    SLSO_CHECK_LAUNCH();
  }
  SLSO_TRY(launch_jacobi(jacobi_fn<double>(d), W, Vw, 60));
  colnorm_kernel<<<static_cast<unsigned>(ceil_div(d * 32, 256)), 256, 0, st>>>(W, d, dp, sig, guard);
  SLSO_CHECK_LAUNCH();
  svd_finalize_kernel<<<1, 1024, 0, st>>>(W, Vw, sig, d, dp, tau, sigma_out, Vout, Vs, Ur, perm, h.state, guard);
  SLSO_CHECK_LAUNCH();
  if (mode == 0) {
    if (k > 0) {
      // Z = Ur^T Pi (d x k), M = Vs Z
      SLSO_TRY(launch_gemm(d, k, d, Ur, 1, d, Pi, k, 1, Z, need, 1, st));
      SLSO_TRY(launch_gemm(d, k, d, Vs, d, 1, Z, k, 1, M, need, 1, st));
    } else {
      copy_guarded_kernel<<<grid1d(d * d, h), 256, 0, st>>>(Vs, d * d, M, need, 1);
      SLSO_CHECK_LAUNCH();
    }
  }
  prof_end(h, ar, st);
  out->M = M;
  out->kk = kk;
  out->R = R;
  out->sigma = sigma_out;
  out->V = Vout;
  return SLSO_OK;
}

}  // namespace slso
