// Sketch SX = S X (Algorithm 2/3 step 1) for the three sketch families of Sec. 2.1.
//
// CountSketch (Sec. 3.1.2, "a pair of hash functions"): rows are hashed to buckets, sorted by
// bucket with the stable radix sort (so each bucket lists its rows in ascending order), and one
// CTA per (bucket, column tile) streams its rows from HBM -- every row of X is read exactly once,
// whole and coalesced -- summing sign(i) x_i with compensated float32 (float64 for F64 X).
//
// SRHT: X is conceptually zero-padded to n_pad = 2^m rows.  With n_pad = n1 * n2 and row
// i = i1 n2 + i2, (H D X)[j1 n2 + j2] = sum_i1 (-1)^popc(i1 & j1) (H_n2 (D X)_chunk i1)[j2].
// One CTA per (chunk i1, 4-column slab) transforms its chunk in shared memory and writes, for
// every sampled row, its signed contribution; a second kernel sums the n1 contributions in
// ascending i1 (float64) and scales by 1/sqrt(s).
//
// Gaussian: tiles of SX = (1/sqrt s) G X over row chunks of X with G generated on the fly
// from Philox (never stored); chunk partials are merged in float64 in chunk order.
#include <algorithm>
#include <cmath>

#include "common.cuh"

namespace slso {

namespace {

// ---------------------------------------------------------------- CountSketch
// Hashes of CountSketch (z = 1, tag 1) and OSNAP (z blocks, tag 7): entry e = b n + i (block b,
// row i) gets bucket b (s/z) + ((w0 (s/z)) >> 32) and sign 1 - 2 (w1 & 1) from Philox at counter
// (lo i, hi i, b, tag).  Within a bucket (one block) the stable sort keeps rows ascending.
__global__ void cs_hash_kernel(int64_t n, int64_t row0, uint32_t s, int z, uint32_t tag, uint64_t seed,
                               uint32_t* __restrict__ keys, uint32_t* __restrict__ vals) {
  const uint32_t m = s / static_cast<uint32_t>(z);
  const int64_t total = n * z;
  for (int64_t e = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; e < total;
       e += static_cast<int64_t>(gridDim.x) * blockDim.x) {
    const uint32_t b = static_cast<uint32_t>(e / n);
    const int64_t i = e - static_cast<int64_t>(b) * n;
    const uint64_t ig = static_cast<uint64_t>(row0 + i);  // row of the whole X: the hash's counter
    const U32x4 w = philox(static_cast<uint32_t>(ig), static_cast<uint32_t>(ig >> 32), b, tag, seed);
    keys[e] = b * m + static_cast<uint32_t>((static_cast<uint64_t>(w.x) * m) >> 32);
    vals[e] = static_cast<uint32_t>(i) | ((w.y & 1u) << 31);  // sign bit: 1 means -1
  }
}

// start[b] = first position of bucket b in the sorted key list; start[s] = n.
__global__ void bucket_start_kernel(const uint32_t* __restrict__ keys, int64_t n, uint32_t s,
                                    uint32_t* __restrict__ start) {
  for (int64_t i = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; i <= n;
       i += static_cast<int64_t>(gridDim.x) * blockDim.x) {
    const int64_t prev = (i == 0) ? -1 : static_cast<int64_t>(keys[i - 1]);
    const int64_t cur = (i == n) ? static_cast<int64_t>(s) : static_cast<int64_t>(keys[i]);
    for (int64_t b = prev + 1; b <= cur; ++b) start[b] = static_cast<uint32_t>(i);
  }
}

template <class T, int VEC>
struct VecLoad;
template <>
struct VecLoad<float, 4> {
  __device__ static void load(const float* p, float* o) {
    const float4 v = __ldg(reinterpret_cast<const float4*>(p));
    o[0] = v.x; o[1] = v.y; o[2] = v.z; o[3] = v.w;
  }
};
template <>
struct VecLoad<__nv_bfloat16, 4> {
  __device__ static void load(const __nv_bfloat16* p, float* o) {
    const uint2 v = __ldg(reinterpret_cast<const uint2*>(p));
    const __nv_bfloat162 a = *reinterpret_cast<const __nv_bfloat162*>(&v.x);
    const __nv_bfloat162 b = *reinterpret_cast<const __nv_bfloat162*>(&v.y);
    o[0] = __low2float(a); o[1] = __high2float(a); o[2] = __low2float(b); o[3] = __high2float(b);
  }
};
template <class T>
struct VecLoad<T, 1> {
  __device__ static void load(const T* p, float* o) { o[0] = to_float(p[0]); }
};

// One CTA per (group of bpc consecutive buckets, column tile of blockDim*VEC columns).  float32/bf16
// X.  CMAX: also the largest |x| of every column over the rows the CTA reads (an atomicMax of the
// float bits per column and CTA), so that the FP8 scores' column scales need no pass of their own.
template <class T, int VEC, int UNROLL, bool CMAX>
__global__ void __launch_bounds__(256) cs_gather_kernel(const T* __restrict__ X, int64_t d, int64_t ldx,
                                                        const uint32_t* __restrict__ rows,
                                                        const uint32_t* __restrict__ start,
                                                        double* __restrict__ SX, double scale, int acc,
                                                        DevState* __restrict__ state, uint32_t nbuckets, int bpc,
                                                        unsigned int* __restrict__ colmax) {
  const int64_t c0 = (static_cast<int64_t>(blockIdx.y) * blockDim.x + threadIdx.x) * VEC;
  const bool active = c0 < d;
  bool bad = false;
  float cm[VEC];
#pragma unroll
  for (int v = 0; v < VEC; ++v) cm[v] = 0.0f;
  const uint32_t bfirst = blockIdx.x * static_cast<uint32_t>(bpc);
  const uint32_t blast = bfirst + bpc < nbuckets ? bfirst + bpc : nbuckets;
  for (uint32_t b = bfirst; b < blast; ++b) {
  float hi[VEC], lo[VEC];
#pragma unroll
  for (int v = 0; v < VEC; ++v) hi[v] = lo[v] = 0.0f;
  const uint32_t p0 = start[b], p1 = start[b + 1];
  uint32_t p = p0;
  for (; p + UNROLL <= p1; p += UNROLL) {
    float x[UNROLL][VEC];
    uint32_t rv[UNROLL];
#pragma unroll
    for (int u = 0; u < UNROLL; ++u) rv[u] = rows[p + u];
#pragma unroll
    for (int u = 0; u < UNROLL; ++u)
      if (active) VecLoad<T, VEC>::load(X + static_cast<int64_t>(rv[u] & 0x7FFFFFFFu) * ldx + c0, x[u]);
#pragma unroll
    for (int u = 0; u < UNROLL; ++u) {
      const bool neg = rv[u] >> 31;
#pragma unroll
      for (int v = 0; v < VEC; ++v) {
        const float xv = active ? x[u][v] : 0.0f;
        bad |= !isfinite(xv);
        if (CMAX) cm[v] = fmaxf(cm[v], fabsf(xv));
        two_sum_acc(hi[v], lo[v], neg ? -xv : xv);
      }
    }
  }
  for (; p < p1; ++p) {
    const uint32_t rv = rows[p];
    float x[VEC];
    if (active) VecLoad<T, VEC>::load(X + static_cast<int64_t>(rv & 0x7FFFFFFFu) * ldx + c0, x);
    const bool neg = rv >> 31;
#pragma unroll
    for (int v = 0; v < VEC; ++v) {
      const float xv = active ? x[v] : 0.0f;
      bad |= !isfinite(xv);
      if (CMAX) cm[v] = fmaxf(cm[v], fabsf(xv));
      two_sum_acc(hi[v], lo[v], neg ? -xv : xv);
    }
  }
  if (active) {
#pragma unroll
    for (int v = 0; v < VEC; ++v)
      if (c0 + v < d) {
        double* o = SX + static_cast<int64_t>(b) * d + c0 + v;
        const double t = (static_cast<double>(hi[v]) + static_cast<double>(lo[v])) * scale;
        *o = acc ? *o + t : t;
      }
  }
  }
  if (CMAX && active) {
#pragma unroll
    for (int v = 0; v < VEC; ++v)
      if (c0 + v < d && cm[v] > 0.0f) atomicMax(colmax + c0 + v, __float_as_uint(cm[v]));
  }
  if (__syncthreads_or(bad) && threadIdx.x == 0) atomicOr(&state->nonfinite, 1);
}

// float64 X: plain float64 sums in ascending row order.
__global__ void __launch_bounds__(256) cs_gather_f64_kernel(const double* __restrict__ X, int64_t d,
                                                            int64_t ldx, const uint32_t* __restrict__ rows,
                                                            const uint32_t* __restrict__ start,
                                                            double* __restrict__ SX, double scale, int accum,
                                                            DevState* __restrict__ state) {
  const uint32_t b = blockIdx.x;
  const int64_t c = static_cast<int64_t>(blockIdx.y) * blockDim.x + threadIdx.x;
  double acc = 0.0;
  bool bad = false;
  if (c < d) {
    for (uint32_t p = start[b]; p < start[b + 1]; ++p) {
      const uint32_t rv = rows[p];
      const double x = X[static_cast<int64_t>(rv & 0x7FFFFFFFu) * ldx + c];
      bad |= !isfinite(x);
      acc += (rv >> 31) ? -x : x;
    }
    double* o = SX + static_cast<int64_t>(b) * d + c;
    *o = accum ? *o + acc * scale : acc * scale;
  }
  if (__syncthreads_or(bad) && threadIdx.x == 0) atomicOr(&state->nonfinite, 1);
}

// ---------------------------------------------------------------- SRHT
__global__ void srht_sample_keys_kernel(int64_t n_pad, uint64_t seed, uint32_t* __restrict__ keys,
                                        uint32_t* __restrict__ vals) {
  for (int64_t j = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; j < n_pad;
       j += static_cast<int64_t>(gridDim.x) * blockDim.x) {
    const U32x4 w = philox(static_cast<uint32_t>(j), static_cast<uint32_t>(static_cast<uint64_t>(j) >> 32),
                           0u, TAG_SRHT_SAMPLE, seed);
    keys[j] = w.x;
    vals[j] = static_cast<uint32_t>(j);
  }
}

__global__ void copy_u32_kernel(const uint32_t* __restrict__ a, int64_t n, uint32_t* __restrict__ b,
                                uint32_t* __restrict__ c) {
  for (int64_t i = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; i < n;
       i += static_cast<int64_t>(gridDim.x) * blockDim.x) {
    b[i] = a[i];
    c[i] = 0u;
  }
}

constexpr int kSrhtSlab = 4;       // columns per CTA
constexpr int kSrhtThreads = 512;

// CTA (i1, slab): chunk i1 of n2 rows, columns [c0, c0 + 4).  Acc = float (F32/BF16 X) or double.
template <class T, class Acc>
__global__ void __launch_bounds__(kSrhtThreads) srht_chunk_kernel(
    const T* __restrict__ X, int64_t n, int64_t d, int64_t ldx, int64_t row0, int log2_n2, uint64_t seed,
    const uint32_t* __restrict__ sample, int64_t s, Acc* __restrict__ P, DevState* __restrict__ state) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  Acc* T_s = reinterpret_cast<Acc*>(smem_raw);  // [n2][kSrhtSlab]
  const int64_t n2 = int64_t(1) << log2_n2;
  const int64_t i1 = blockIdx.x;
  const int64_t c0 = static_cast<int64_t>(blockIdx.y) * kSrhtSlab;
  bool bad = false;
  for (int64_t r = threadIdx.x; r < n2; r += kSrhtThreads) {
    const int64_t i = i1 * n2 + r;  // row of this block; row0 + i of the whole X
    Acc v[kSrhtSlab];
    if (i < n) {
      const uint64_t ig = static_cast<uint64_t>(row0 + i);
      const U32x4 w = philox(static_cast<uint32_t>(ig), static_cast<uint32_t>(ig >> 32), 0u, TAG_SRHT_SIGN, seed);
      const bool neg = w.x & 1u;
#pragma unroll
      for (int c = 0; c < kSrhtSlab; ++c) {
        Acc x = (c0 + c < d) ? static_cast<Acc>(to_float_or_double(X[i * ldx + c0 + c])) : Acc(0);
        bad |= !isfinite(static_cast<double>(x));
        v[c] = neg ? -x : x;
      }
    } else {
#pragma unroll
      for (int c = 0; c < kSrhtSlab; ++c) v[c] = Acc(0);
    }
#pragma unroll
    for (int c = 0; c < kSrhtSlab; ++c) T_s[r * kSrhtSlab + c] = v[c];
  }
  __syncthreads();
  // in-place fast Walsh-Hadamard transform over the n2 rows (unnormalised, natural order)
  for (int64_t h = 1; h < n2; h <<= 1) {
    for (int64_t t = threadIdx.x; t < (n2 >> 1) * kSrhtSlab; t += kSrhtThreads) {
      const int64_t pr = t / kSrhtSlab, c = t % kSrhtSlab;
      const int64_t a = (pr / h) * (2 * h) + (pr % h);
      const Acc u = T_s[a * kSrhtSlab + c], w = T_s[(a + h) * kSrhtSlab + c];
      T_s[a * kSrhtSlab + c] = u + w;
      T_s[(a + h) * kSrhtSlab + c] = u - w;
    }
    __syncthreads();
  }
  // signed contribution of this chunk to every sampled row: P[(i1*d + c)*s + q]
  for (int64_t q = threadIdx.x; q < s; q += kSrhtThreads) {
    const uint32_t j = sample[q];
    const uint32_t j1 = j >> log2_n2, j2 = j & static_cast<uint32_t>(n2 - 1);
    const bool neg = __popc(static_cast<uint32_t>((row0 >> log2_n2) + i1) & j1) & 1;  // row0: multiple of n2
#pragma unroll
    for (int c = 0; c < kSrhtSlab; ++c) {
      if (c0 + c < d) {
        const Acc v = T_s[static_cast<int64_t>(j2) * kSrhtSlab + c];
        P[(i1 * d + c0 + c) * s + q] = neg ? -v : v;
      }
    }
  }
  if (__syncthreads_or(bad) && threadIdx.x == 0) atomicOr(&state->nonfinite, 1);
}

// SX[q][c] = (sum_i1 P[(i1*d + c)*s + q]) / sqrt(s), float64, ascending i1; 32x32 tile transpose.
template <class Acc>
__global__ void srht_combine_kernel(const Acc* __restrict__ P, int64_t n1, int64_t d, int64_t s, int accum,
                                    double* __restrict__ SX) {
  __shared__ double tile[32][33];
  const int64_t q0 = static_cast<int64_t>(blockIdx.x) * 32, c0 = static_cast<int64_t>(blockIdx.y) * 32;
  const double inv = sqrt(static_cast<double>(s));
  for (int cc = threadIdx.y; cc < 32; cc += blockDim.y) {
    const int64_t c = c0 + cc, q = q0 + threadIdx.x;
    double acc = 0.0;
    if (c < d && q < s)
      for (int64_t i1 = 0; i1 < n1; ++i1) acc += static_cast<double>(P[(i1 * d + c) * s + q]);
    tile[cc][threadIdx.x] = acc / inv;
  }
  __syncthreads();
  for (int qq = threadIdx.y; qq < 32; qq += blockDim.y) {
    const int64_t q = q0 + qq, c = c0 + threadIdx.x;
    if (q < s && c < d) SX[q * d + c] = accum ? SX[q * d + c] + tile[threadIdx.x][qq] : tile[threadIdx.x][qq];
  }
}

// Float32 SRHT chunk transform with coalesced loads and the butterflies in registers (float32 and
// bfloat16 X).  CTA (i1, slab): chunk i1 of N2 = 2^LOG2 rows (64 <= N2 <= 4096), columns
// [8 slab, 8 slab + 8): 512 threads = 64 row groups g x 8 columns; a warp-wide load reads four
// rows' 32-byte column segments.  Row r = g R + t of the chunk (R = N2 / 64):
//   phase 1: thread (g, col) holds rows g R .. g R + R - 1 and runs the log2 R butterfly levels
//            over t in registers;
//   exchange through shared memory (the only cross-warp step), then thread (g, col) with g < R
//            holds rows a R + g for all 64 values of a and runs the remaining 6 levels over a;
//   every sampled row j = j1 N2 + j2 then takes (-1)^popc(i1 & j1) T[j2] (this chunk's share of
//            (H D X)_j) into P[i1][q][c] (row pitch dp: 32-byte segments again).
// Shared rows are stored at r ^ ((r / R) & 3) (R >= 4) so that the four row groups of a warp
// fall on different banks in both phases.  The D signs come from Philox once per row: lane col
// draws the rows t = col (mod 8) of its group and the 8 lanes combine their bit masks by shuffles.
constexpr int kSr2Threads = 512;
constexpr int kSr2Cols = 8;

template <class T, int LOG2>
__global__ void __launch_bounds__(kSr2Threads, 1) srht_chunk_reg_kernel(
    const T* __restrict__ X, int64_t n, int64_t d, int64_t ldx, int64_t row0, uint64_t seed,
    const uint32_t* __restrict__ sample, int64_t s, int64_t dp, float* __restrict__ P, DevState* __restrict__ state) {
  constexpr int N2 = 1 << LOG2, R = N2 / 64;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  float* S = reinterpret_cast<float*>(smem_raw);  // [N2][8], rows permuted by prow
  auto prow = [](int r) { return R >= 4 ? (r ^ ((r / R) & 3)) : r; };
  const int col = threadIdx.x & 7, g = threadIdx.x >> 3;
  const int64_t i1 = blockIdx.x;
  const int64_t c = static_cast<int64_t>(blockIdx.y) * kSr2Cols + col;
  const int64_t rbase = i1 * N2 + static_cast<int64_t>(g) * R;  // first row of the group (block rows)
  float v[64];
  // the group's R rows of this column (issued before the sign draws, so the loads are in flight)
#pragma unroll
  for (int t = 0; t < R; ++t) {
    const int64_t i = rbase + t;
    v[t] = (i < n && c < d) ? to_float_or_double(X[i * ldx + c]) : 0.f;
  }
  // D signs of the group's R rows: bit t set means row rbase + t is negated
  uint32_t m_lo = 0, m_hi = 0;
  for (int t = col; t < R; t += kSr2Cols) {
    const int64_t i = rbase + t;
    if (i < n) {
      const uint64_t ig = static_cast<uint64_t>(row0 + i);
      const U32x4 w = philox(static_cast<uint32_t>(ig), static_cast<uint32_t>(ig >> 32), 0u, TAG_SRHT_SIGN, seed);
      if (w.x & 1u) {
        if (t < 32) m_lo |= 1u << t;
        else m_hi |= 1u << (t - 32);
      }
    }
  }
#pragma unroll
  for (int o = 1; o < kSr2Cols; o <<= 1) {
    m_lo |= __shfl_xor_sync(0xFFFFFFFFu, m_lo, o);
    m_hi |= __shfl_xor_sync(0xFFFFFFFFu, m_hi, o);
  }
  bool bad = false;
#pragma unroll
  for (int t = 0; t < R; ++t) {
    bad |= !isfinite(v[t]);
    const bool neg = ((t < 32 ? m_lo >> t : m_hi >> (t - 32)) & 1u) != 0;
    v[t] = neg ? -v[t] : v[t];
  }
#pragma unroll
  for (int h = 1; h < R; h <<= 1)
#pragma unroll
    for (int t = 0; t < R; ++t)
      if ((t & h) == 0) {
        const float a = v[t], b = v[t + h];
        v[t] = a + b;
        v[t + h] = a - b;
      }
#pragma unroll
  for (int t = 0; t < R; ++t) S[prow(g * R + t) * kSr2Cols + col] = v[t];
  __syncthreads();
  if (g < R) {
#pragma unroll
    for (int a = 0; a < 64; ++a) v[a] = S[prow(a * R + g) * kSr2Cols + col];
#pragma unroll
    for (int h = 1; h < 64; h <<= 1)
#pragma unroll
      for (int a = 0; a < 64; ++a)
        if ((a & h) == 0) {
          const float x = v[a], y = v[a + h];
          v[a] = x + y;
          v[a + h] = x - y;
        }
#pragma unroll
    for (int a = 0; a < 64; ++a) S[prow(a * R + g) * kSr2Cols + col] = v[a];
  }
  __syncthreads();
  const uint32_t ib = static_cast<uint32_t>((row0 >> LOG2) + i1);  // row0: a multiple of N2
  // sampled rows, eight at a time per thread so that their index loads overlap
  for (int64_t q0 = g; q0 < s; q0 += 64 * 8) {
    uint32_t jj[8];
#pragma unroll
    for (int u = 0; u < 8; ++u) {
      const int64_t q = q0 + 64 * u;
      jj[u] = q < s ? sample[q] : 0u;
    }
#pragma unroll
    for (int u = 0; u < 8; ++u) {
      const int64_t q = q0 + 64 * u;
      const uint32_t j1 = jj[u] >> LOG2, j2 = jj[u] & static_cast<uint32_t>(N2 - 1);
      const float val = S[prow(static_cast<int>(j2)) * kSr2Cols + col];
      if (q < s && c < d) P[(i1 * s + q) * dp + c] = (__popc(ib & j1) & 1) ? -val : val;
    }
  }
  if (__syncthreads_or(bad) && threadIdx.x == 0) atomicOr(&state->nonfinite, 1);
}

// SX[q][c] (+)= (sum over i1 ascending of P[i1][q][c]) / sqrt(s) in float64; coalesced along c.
__global__ void srht_combine_reg_kernel(const float* __restrict__ P, int64_t n1, int64_t d, int64_t dp, int64_t s,
                                        int accum, double* __restrict__ SX) {
  const double rs = sqrt(static_cast<double>(s));
  for (int64_t e = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; e < s * d;
       e += static_cast<int64_t>(gridDim.x) * blockDim.x) {
    const int64_t q = e / d, c = e - q * d;
    const float* p = P + q * dp + c;
    const int64_t stride = s * dp;
    double acc = 0.0;
    int64_t i1 = 0;
    for (; i1 + 8 <= n1; i1 += 8) {  // eight loads in flight, added in ascending i1
      float t[8];
#pragma unroll
      for (int u = 0; u < 8; ++u) t[u] = p[(i1 + u) * stride];
#pragma unroll
      for (int u = 0; u < 8; ++u) acc += static_cast<double>(t[u]);
    }
    for (; i1 < n1; ++i1) acc += static_cast<double>(p[i1 * stride]);
    const double v = acc / rs;
    SX[e] = accum ? SX[e] + v : v;
  }
}

// ---------------------------------------------------------------- Gaussian (SIMT)
constexpr int kGbm = 64, kGbn = 64, kGbk = 16;

// grid (ceil(s/64), ceil(d/64), nz); chunk z covers X rows [z*kc, (z+1)*kc).
// Each 16-row step accumulates 16 products in Acc, then adds the step sum into a compensated
// (hi, lo) pair (float32 data) or a float64 sum (float64 data).
template <class T, class Acc>
__global__ void __launch_bounds__(256) gauss_tile_kernel(const T* __restrict__ X, int64_t n, int64_t d,
                                                         int64_t ldx, int64_t row0, int64_t s, uint64_t seed,
                                                         int64_t kc, Acc* __restrict__ P,
                                                         DevState* __restrict__ state) {
  __shared__ Acc Gs[kGbk][kGbm + 1];
  __shared__ Acc Xs[kGbk][kGbn];
  const int tx = threadIdx.x % 16, ty = threadIdx.x / 16;  // 16 x 16 threads, 4x4 outputs each
  const int64_t j0 = static_cast<int64_t>(blockIdx.x) * kGbm, c0 = static_cast<int64_t>(blockIdx.y) * kGbn;
  const int64_t r0 = static_cast<int64_t>(blockIdx.z) * kc;
  const int64_t r1 = (r0 + kc < n) ? r0 + kc : n;
  Acc hi[4][4], lo[4][4];
#pragma unroll
  for (int a = 0; a < 4; ++a)
#pragma unroll
    for (int b = 0; b < 4; ++b) hi[a][b] = lo[a][b] = Acc(0);
  bool bad = false;
  for (int64_t k0 = r0; k0 < r1; k0 += kGbk) {
    for (int t = threadIdx.x; t < kGbk * kGbm; t += 256) {
      const int kk = t / kGbm, jj = t % kGbm;
      const int64_t i = k0 + kk, j = j0 + jj;
      Gs[kk][jj] = (i < r1 && j < s) ? static_cast<Acc>(gaussian_entry(seed, static_cast<uint32_t>(j), row0 + i))
                                     : Acc(0);
    }
    for (int t = threadIdx.x; t < kGbk * kGbn; t += 256) {
      const int kk = t / kGbn, cc = t % kGbn;
      const int64_t i = k0 + kk, c = c0 + cc;
      Acc x = Acc(0);
      if (i < r1 && c < d) {
        x = static_cast<Acc>(to_float_or_double(X[i * ldx + c]));
        bad |= !isfinite(static_cast<double>(x));
      }
      Xs[kk][cc] = x;
    }
    __syncthreads();
    Acc part[4][4];
#pragma unroll
    for (int a = 0; a < 4; ++a)
#pragma unroll
      for (int b = 0; b < 4; ++b) part[a][b] = Acc(0);
#pragma unroll
    for (int kk = 0; kk < kGbk; ++kk) {
      Acc g[4], x[4];
#pragma unroll
      for (int a = 0; a < 4; ++a) g[a] = Gs[kk][ty * 4 + a];
#pragma unroll
      for (int b = 0; b < 4; ++b) x[b] = Xs[kk][tx * 4 + b];
#pragma unroll
      for (int a = 0; a < 4; ++a)
#pragma unroll
        for (int b = 0; b < 4; ++b) part[a][b] = fma(g[a], x[b], part[a][b]);
    }
#pragma unroll
    for (int a = 0; a < 4; ++a)
#pragma unroll
      for (int b = 0; b < 4; ++b) comp_add(hi[a][b], lo[a][b], part[a][b]);
    __syncthreads();
  }
  const int64_t nz_stride = s * d;
#pragma unroll
  for (int a = 0; a < 4; ++a)
#pragma unroll
    for (int b = 0; b < 4; ++b) {
      const int64_t j = j0 + ty * 4 + a, c = c0 + tx * 4 + b;
      if (j < s && c < d) P[blockIdx.z * nz_stride + j * d + c] = hi[a][b] + lo[a][b];
    }
  if (__syncthreads_or(bad) && threadIdx.x == 0) atomicOr(&state->nonfinite, 1);
}

template <class Acc>
__global__ void gauss_combine_kernel(const Acc* __restrict__ P, int64_t nz, int64_t sd, int64_t s, int accum,
                                     double* __restrict__ SX) {
  const double inv = sqrt(static_cast<double>(s));
  for (int64_t e = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; e < sd;
       e += static_cast<int64_t>(gridDim.x) * blockDim.x) {
    double acc = 0.0;
    for (int64_t z = 0; z < nz; ++z) acc += static_cast<double>(P[z * sd + e]);
    SX[e] = accum ? SX[e] + acc / inv : acc / inv;
  }
}

int grid_for(int64_t n, const Handle& h) {
  return static_cast<int>(std::max<int64_t>(1, std::min<int64_t>(ceil_div(n, 256), 16LL * h.num_sms)));
}

// CountSketch (z = 1) and OSNAP (z blocks, entries +-1/sqrt(z)): hash, stable sort of the n z
// entries by bucket, then the deterministic gather of each bucket's rows in ascending order.
// The rows are rows row0 .. row0 + n - 1 of the whole X (their hash counters); acc adds the
// block's sketch to SX.
template <class T>
slso_status countsketch(Handle& h, Arena& ar, const T* X, int64_t n, int64_t d, int64_t ldx,
                        int64_t s, uint64_t seed, int z, uint32_t tag, int64_t row0, int acc, double* SX,
                        cudaStream_t st, unsigned int* colmax) {
  const int64_t N = n * z;
  uint32_t* keys = ar.take<uint32_t>(N);
  uint32_t* vals = ar.take<uint32_t>(N);
  uint32_t* start = ar.take<uint32_t>(s + 1);
  int bits = 0;
  while ((int64_t(1) << bits) < s) ++bits;
  uint32_t* ks = keys;
  uint32_t* vs = vals;
  if (!ar.measure()) {
    cs_hash_kernel<<<grid_for(N, h), 256, 0, st>>>(n, row0, static_cast<uint32_t>(s), z, tag, seed, keys, vals);
    SLSO_CHECK_LAUNCH();
  }
  if (bits > 0) SLSO_TRY(radix_sort_u32(ar, keys, vals, N, bits, st, &ks, &vs));
  if (ar.measure()) return SLSO_OK;
  bucket_start_kernel<<<grid_for(N + 1, h), 256, 0, st>>>(ks, N, static_cast<uint32_t>(s), start);
  SLSO_CHECK_LAUNCH();
  const double scale = (z == 1) ? 1.0 : 1.0 / std::sqrt(static_cast<double>(z));
  if constexpr (std::is_same<T, double>::value) {
    dim3 grid(static_cast<unsigned>(s), static_cast<unsigned>(ceil_div(d, 256)));
    cs_gather_f64_kernel<<<grid, 256, 0, st>>>(X, d, ldx, vs, start, SX, scale, acc, h.state);
  } else {
    const bool vec = (d % 4 == 0) && (ldx % 4 == 0) &&
                     (reinterpret_cast<uintptr_t>(X) % (4 * sizeof(T)) == 0);
    // with the column maxima, a CTA walks 16 consecutive buckets (one atomic per column per CTA)
    const int bpc = colmax ? 16 : 1;
    const unsigned gb = static_cast<unsigned>(ceil_div(s, bpc));
    const uint32_t nbk = static_cast<uint32_t>(s);
    if (vec) {
      const int64_t thr_needed = ceil_div(d, 4);
      const int threads = static_cast<int>(std::min<int64_t>(256, ceil_div(thr_needed, 32) * 32));
      dim3 grid(gb, static_cast<unsigned>(ceil_div(thr_needed, threads)));
      if (colmax)
        cs_gather_kernel<T, 4, 4, true><<<grid, threads, 0, st>>>(X, d, ldx, vs, start, SX, scale, acc, h.state, nbk,
                                                                  bpc, colmax);
      else
        cs_gather_kernel<T, 4, 4, false><<<grid, threads, 0, st>>>(X, d, ldx, vs, start, SX, scale, acc, h.state,
                                                                   nbk, bpc, nullptr);
    } else {
      const int threads = static_cast<int>(std::min<int64_t>(256, ceil_div(d, 32) * 32));
      dim3 grid(gb, static_cast<unsigned>(ceil_div(d, threads)));
      if (colmax)
        cs_gather_kernel<T, 1, 8, true><<<grid, threads, 0, st>>>(X, d, ldx, vs, start, SX, scale, acc, h.state, nbk,
                                                                  bpc, colmax);
      else
        cs_gather_kernel<T, 1, 8, false><<<grid, threads, 0, st>>>(X, d, ldx, vs, start, SX, scale, acc, h.state,
                                                                   nbk, bpc, nullptr);
    }
  }
  SLSO_CHECK_LAUNCH();
  return SLSO_OK;
}

int log2_ceil(int64_t n) {
  int m = 0;
  while ((int64_t(1) << m) < n) ++m;
  return m;
}

// Chunk height: float64 X, 2^12 rows of 4 columns in shared memory (128 KB); float32 / bfloat16
// X, 2^12 rows of 8 columns (128 KB) in the register-butterfly kernel, which needs 64 rows at least
// (smaller padded heights take the shared-memory kernel).
template <class T>
int srht_log2_n2(int64_t n_total) {
  return std::min(log2_ceil(n_total), 12);
}
template <class T>
constexpr bool srht_reg_form() {
  return !std::is_same<T, double>::value;
}

// Rows n .. n_pad - 1 of the padded X are zero, so only the ceil(n / n2) chunks holding rows of
// this block are transformed; the whole X has n_total rows and the block starts at row row0 (a
// multiple of n2).
template <class T>
slso_status srht(Handle& h, Arena& ar, const T* X, int64_t n, int64_t d, int64_t ldx, int64_t s,
                 uint64_t seed, const uint32_t* sample, int64_t row0, int64_t n_total, int acc, double* SX,
                 cudaStream_t st) {
  using Acc = typename std::conditional<std::is_same<T, double>::value, double, float>::type;
  const int log2_n2 = srht_log2_n2<T>(n_total);
  const int64_t n1 = ceil_div(n, int64_t(1) << log2_n2);
  if (sample == nullptr) SLSO_TRY(srht_sample_rows(h, ar, n_total, s, seed, &sample, st));
  if (srht_reg_form<T>() && log2_n2 >= 6) {
    const int64_t dp = ceil_div(d, kSr2Cols) * kSr2Cols;
    float* Pr = ar.take<float>(static_cast<size_t>(n1) * s * dp);
    if (ar.measure()) return SLSO_OK;
    const size_t smem = (size_t(1) << log2_n2) * kSr2Cols * sizeof(float);
    const dim3 g1(static_cast<unsigned>(n1), static_cast<unsigned>(ceil_div(d, kSr2Cols)));
    auto launch = [&](auto kern) -> slso_status {
      SLSO_TRY(raise_smem_limit(kern, smem));
      kern<<<g1, kSr2Threads, smem, st>>>(X, n, d, ldx, row0, seed, sample, s, dp, Pr, h.state);
      SLSO_CHECK_LAUNCH();
      return SLSO_OK;
    };
    switch (log2_n2) {
      case 6: SLSO_TRY(launch(srht_chunk_reg_kernel<T, 6>)); break;
      case 7: SLSO_TRY(launch(srht_chunk_reg_kernel<T, 7>)); break;
      case 8: SLSO_TRY(launch(srht_chunk_reg_kernel<T, 8>)); break;
      case 9: SLSO_TRY(launch(srht_chunk_reg_kernel<T, 9>)); break;
      case 10: SLSO_TRY(launch(srht_chunk_reg_kernel<T, 10>)); break;
      case 11: SLSO_TRY(launch(srht_chunk_reg_kernel<T, 11>)); break;
      default: SLSO_TRY(launch(srht_chunk_reg_kernel<T, 12>)); break;
    }
    const int64_t total = s * d;
    const unsigned gc = static_cast<unsigned>(std::min<int64_t>(ceil_div(total, 256), 16LL * h.num_sms));
    srht_combine_reg_kernel<<<gc, 256, 0, st>>>(Pr, n1, d, dp, s, acc, SX);
    SLSO_CHECK_LAUNCH();
    return SLSO_OK;
  }
  Acc* P = ar.take<Acc>(static_cast<size_t>(n1) * d * s);
  if (ar.measure()) return SLSO_OK;
  const size_t smem = (size_t(1) << log2_n2) * kSrhtSlab * sizeof(Acc);
  SLSO_TRY(raise_smem_limit(srht_chunk_kernel<T, Acc>, smem));
  dim3 g1(static_cast<unsigned>(n1), static_cast<unsigned>(ceil_div(d, kSrhtSlab)));
  srht_chunk_kernel<T, Acc><<<g1, kSrhtThreads, smem, st>>>(X, n, d, ldx, row0, log2_n2, seed, sample, s, P,
                                                            h.state);
  SLSO_CHECK_LAUNCH();
  dim3 g2(static_cast<unsigned>(ceil_div(s, 32)), static_cast<unsigned>(ceil_div(d, 32)));
  srht_combine_kernel<Acc><<<g2, dim3(32, 8), 0, st>>>(P, n1, d, s, acc, SX);
  SLSO_CHECK_LAUNCH();
  return SLSO_OK;
}

template <class T>
slso_status gaussian(Handle& h, Arena& ar, const T* X, int64_t n, int64_t d, int64_t ldx, int64_t s,
                     uint64_t seed, int64_t row0, int acc, double* SX, cudaStream_t st) {
  using Acc = typename std::conditional<std::is_same<T, double>::value, double, float>::type;
  // chunks of >= 2048 rows, at most 32 of them
  const int64_t kc = std::max<int64_t>(2048, ceil_div(ceil_div(n, 32), kGbk) * kGbk);
  const int64_t nz = ceil_div(n, kc);
  Acc* P = ar.take<Acc>(static_cast<size_t>(nz) * s * d);
  if (ar.measure()) return SLSO_OK;
  dim3 g1(static_cast<unsigned>(ceil_div(s, kGbm)), static_cast<unsigned>(ceil_div(d, kGbn)),
          static_cast<unsigned>(nz));
  gauss_tile_kernel<T, Acc><<<g1, 256, 0, st>>>(X, n, d, ldx, row0, s, seed, kc, P, h.state);
  SLSO_CHECK_LAUNCH();
  gauss_combine_kernel<Acc><<<grid_for(s * d, h), 256, 0, st>>>(P, nz, s * d, s, acc, SX);
  SLSO_CHECK_LAUNCH();
  return SLSO_OK;
}

template <class T>
slso_status sketch_typed(Handle& h, Arena& ar, const T* X, int64_t n, int64_t d, int64_t ldx, int32_t kind,
                         int64_t s, uint64_t seed, int nnz, const SketchBlock& b, double* SX, cudaStream_t st) {
  const int acc = b.accumulate ? 1 : 0;
  switch (kind) {
    case SLSO_COUNTSKETCH:
      return countsketch(h, ar, X, n, d, ldx, s, seed, 1, TAG_COUNTSKETCH, b.row0, acc, SX, st, b.colmax);
    case SLSO_OSNAP:
      return countsketch(h, ar, X, n, d, ldx, s, seed, nnz > 0 ? nnz : kOsnapDefaultNnz, TAG_OSNAP, b.row0, acc,
                         SX, st, b.colmax);
    case SLSO_SRHT:
      return srht(h, ar, X, n, d, ldx, s, seed, b.srht_rows, b.row0, b.n_total > 0 ? b.n_total : n, acc, SX, st);
    default:
      return gaussian(h, ar, X, n, d, ldx, s, seed, b.row0, acc, SX, st);
  }
}

}  // namespace

// The s sampled rows of H for an X of n_total rows: the s smallest (Philox key, index) among the
// n_pad = 2^ceil(log2 n_total) rows, then sorted ascending.
slso_status srht_sample_rows(Handle& h, Arena& ar, int64_t n_total, int64_t s, uint64_t seed,
                             const uint32_t** rows, cudaStream_t st) {
  const int m = log2_ceil(n_total);
  const int64_t n_pad = int64_t(1) << m;
  uint32_t* keys = ar.take<uint32_t>(n_pad);
  uint32_t* vals = ar.take<uint32_t>(n_pad);
  uint32_t* skeys = ar.take<uint32_t>(s);
  uint32_t* svals = ar.take<uint32_t>(s);
  uint32_t* ks = nullptr;
  uint32_t* vs = nullptr;
  if (!ar.measure()) {
    srht_sample_keys_kernel<<<grid_for(n_pad, h), 256, 0, st>>>(n_pad, seed, keys, vals);
    SLSO_CHECK_LAUNCH();
  }
  SLSO_TRY(radix_sort_u32(ar, keys, vals, n_pad, 32, st, &ks, &vs));
  // the first s row indices, re-sorted ascending: keys = row index
  if (!ar.measure()) {
    copy_u32_kernel<<<grid_for(s, h), 256, 0, st>>>(vs, s, skeys, svals);
    SLSO_CHECK_LAUNCH();
  }
  uint32_t* sk = skeys;
  uint32_t* sv = nullptr;
  if (m > 0) SLSO_TRY(radix_sort_u32(ar, skeys, svals, s, m, st, &sk, &sv));
  *rows = sk;
  return SLSO_OK;
}

slso_status run_sketch(Handle& h, Arena& ar, const void* X, int64_t n, int64_t d, int64_t ldx,
                       int32_t xdt, int32_t kind, int64_t s, uint64_t seed, int nnz, double* SX,
                       cudaStream_t st, const SketchBlock* blk) {
  const SketchBlock whole{};
  const SketchBlock& b = blk ? *blk : whole;
  if (kind != SLSO_COUNTSKETCH && kind != SLSO_OSNAP && kind != SLSO_SRHT && kind != SLSO_GAUSSIAN)
    return fail(SLSO_ERR_INVALID_ARG, "unknown sketch kind %d", kind);
  if (kind == SLSO_GAUSSIAN) {
    bool used = false;
    SLSO_TRY(run_gauss_tc(h, ar, X, n, d, ldx, xdt, s, seed, b.row0, b.accumulate, SX, st, &used));
    if (used) return SLSO_OK;
  }
  switch (xdt) {
    case SLSO_F32:
      return sketch_typed(h, ar, static_cast<const float*>(X), n, d, ldx, kind, s, seed, nnz, b, SX, st);
    case SLSO_BF16:
      return sketch_typed(h, ar, static_cast<const __nv_bfloat16*>(X), n, d, ldx, kind, s, seed, nnz, b, SX, st);
    default:
      return sketch_typed(h, ar, static_cast<const double*>(X), n, d, ldx, kind, s, seed, nnz, b, SX, st);
  }
}

}  // namespace slso
