// Tensor-core row scores l_i = ||(X M)_i||^2 (Algorithm 3 steps 4-5) on sm_103a.
//
// Persistent, warp-specialised kernel, one CTA per SM, 128-row tiles of X, the whole JL width N
// (k rounded up to 32, <= 256) accumulated in TMEM (two accumulators, so the epilogue of one
// tile overlaps the MMAs of the next):
//   warps 0-3  epilogue: tcgen05.ld 32x32b gives each thread one accumulator row; the thread
//              sums its squares and writes l_i.  Y = X M never leaves the SM.
//   warp 4     TMA producer: X tiles (rows of 128 bytes, 128B swizzle) and the matching K-slices
//              of B = M^T (prepared once per call in global memory).
//   warp 5     TMEM owner and MMA issuer (one thread): tcgen05.mma, commits to mbarriers.
//   warps 6-13 converters (float32 X only): float32 tile -> operand tile(s) in the same layout.
// Modes:
//   TF32X3    float32 X, float32-accurate: X = Xhi + Xlo with Xhi = tf32(X), Xlo = tf32(X - Xhi)
//             (nearest-even), M = Mhi + Mlo likewise; D += Xhi Mhi + Xhi Mlo + Xlo Mhi (kind::tf32).
//   BF16_CVT  float32 X rounded to bfloat16 in shared memory, M in bfloat16 (kind::f16).
//   BF16      bfloat16 X loaded directly (kind::f16).
//   BF16X3    bfloat16 X loaded directly, float32-accurate: M = M1 + M2 + M3 with each piece a
//             bfloat16 (24 significant bits in all), D += X M1 + X M2 + X M3 (products exact).
//   FP8_F32 / FP8_BF16  float32 or bfloat16 X scaled per column by c_j = 448 / max_i |x_ij| and
//             rounded to e4m3 in shared memory; B = e4m3(e M^T diag(1/c)) with one scale e for
//             M; the epilogue multiplies each row's sum of squares by 1/e^2 (kind::f8f6f4).
// All accumulation is float32 in TMEM.  Every mbarrier wait is bounded; a timeout sets an error
// word that the host reports as SLSO_ERR_TIMEOUT.
#include <cuda.h>
#include <cudaTypedefs.h>
#include <cuda_fp8.h>

#include <algorithm>

#include "common.cuh"
#include "tc.cuh"
#include "tmap.cuh"

namespace slso {

namespace {

using namespace tc;

enum Mode : int { MODE_TF32X3 = 0, MODE_BF16_CVT = 1, MODE_BF16 = 2, MODE_FP8_F32 = 3, MODE_FP8_BF16 = 4,
                  MODE_BF16X3 = 5 };

// X tiles go straight from TMA into the operand stage (no converter pass).
__host__ __device__ constexpr bool direct_x(int mode) { return mode == MODE_BF16 || mode == MODE_BF16X3; }
// B = M^T tiles per operand stage.
__host__ __device__ constexpr int b_tiles(int mode) {
  return mode == MODE_TF32X3 ? 2 : (mode == MODE_BF16X3 ? 3 : 1);
}

constexpr int kConvThreads = 256;
constexpr int kThreads = 192 + kConvThreads;
constexpr int kBM = 128;
constexpr int kMaxStages = 8;
constexpr int kWarpProducer = 4, kWarpMma = 5, kWarpConvert0 = 6;
constexpr uint32_t kXTileBytes = kBM * 128;  // one 128-row x 128-byte tile

struct Layout {
  int mode;
  int N;         // accumulator columns (k padded to 32; zero columns add nothing)
  int KB;        // K-blocks
  int kbe;       // K elements per block: 32 (float32 operands) or 64 (bfloat16 operands)
  int RS, OS;    // raw / operand stages
  int raw_boxes; // X boxes (128 rows x 128 bytes) per K-block
  int box_cols;  // X columns per box: 32 (float32 X) or 64 (bfloat16 X)
  uint32_t x_op_bytes;  // X operand bytes in an operand stage
  uint32_t raw_bytes, b_bytes, op_bytes;
  uint32_t raw_off, op_off, bar_off, smem_bytes;
  uint32_t tmem_cols;
};

// Round a float32 (bit pattern) to TF32 (10 explicit mantissa bits), nearest-even, so that the
// tensor core consumes exact TF32 values and no truncation bias enters the products.
__host__ __device__ __forceinline__ uint32_t rne_tf32(uint32_t b) {
  return (b + 0x0FFFu + ((b >> 13) & 1u)) & 0xFFFFE000u;
}

// x = hi + lo with hi = tf32(x) and lo = tf32(x - hi): x to within 2^-22 relative.
__device__ __forceinline__ void split_tf32(uint32_t x, uint32_t& hi, uint32_t& lo) {
  hi = rne_tf32(x);
  lo = rne_tf32(__float_as_uint(__uint_as_float(x) - __uint_as_float(hi)));
}

__global__ void __launch_bounds__(kThreads, 1)
    score_tc_kernel(const __grid_constant__ CUtensorMap tmX, const __grid_constant__ CUtensorMap tmB0,
                    const __grid_constant__ CUtensorMap tmB1, const __grid_constant__ CUtensorMap tmB2,
                    const Layout L, int64_t n, int ntiles, int ncb,
                    const float* __restrict__ cscale, const float* __restrict__ post_scale,
                    float* __restrict__ scores, float* __restrict__ U, int64_t ldu, int64_t ucols,
                    DevState* __restrict__ state) {
  extern __shared__ unsigned char smem_dyn[];
  unsigned char* smem = reinterpret_cast<unsigned char*>((reinterpret_cast<uintptr_t>(smem_dyn) + 1023) &
                                                         ~static_cast<uintptr_t>(1023));
  uint64_t* raw_full = reinterpret_cast<uint64_t*>(smem + L.bar_off);
  uint64_t* raw_empty = raw_full + kMaxStages;
  uint64_t* op_full = raw_empty + kMaxStages;   // TMA bytes of the operand stage landed
  uint64_t* cvt_full = op_full + kMaxStages;    // converters wrote the X operand(s)
  uint64_t* op_empty = cvt_full + kMaxStages;   // the MMAs reading the stage completed
  uint64_t* acc_full = op_empty + kMaxStages;
  uint64_t* acc_empty = acc_full + 2;
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(acc_empty + 2);
  __shared__ int s_abort;
  const volatile int* abort_flag = &s_abort;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const bool convert = !direct_x(L.mode);
  const int nwork = ntiles * ncb;  // (row tile, column block) work items, row tile major

  if (threadIdx.x == 0) {
    s_abort = 0;
    for (int i = 0; i < L.RS; ++i) {
      mbar_init(&raw_full[i], 1);
      mbar_init(&raw_empty[i], kConvThreads);
    }
    for (int i = 0; i < L.OS; ++i) {
      mbar_init(&op_full[i], 1);
      mbar_init(&cvt_full[i], kConvThreads);
      mbar_init(&op_empty[i], 1);
    }
    for (int i = 0; i < 2; ++i) {
      mbar_init(&acc_full[i], 1);
      mbar_init(&acc_empty[i], 128);
    }
    fence_mbar_init();
  }
  if (warp == kWarpMma) tmem_alloc(tmem_slot, L.tmem_cols);
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem_base = *tmem_slot;

  if (warp == kWarpProducer) {
    if (lane == 0) {
      int it = 0;
      bool ok = true;
      for (int w = blockIdx.x; w < nwork && ok; w += gridDim.x) {
        const int y = (w / ncb) * kBM;
        const int yb = (w % ncb) * L.N;  // rows of B = M^T: this work item's column block
        for (int kb = 0; kb < L.KB; ++kb, ++it) {
          const int os = it % L.OS;
          const uint32_t oph = (it / L.OS) & 1u;
          if (!mbar_wait(&op_empty[os], oph ^ 1u, abort_flag)) { ok = false; break; }
          unsigned char* op = smem + L.op_off + os * L.op_bytes;
          const int x = kb * L.kbe;
          if (direct_x(L.mode)) {
            const int nb = b_tiles(L.mode);
            mbar_arrive_expect_tx(&op_full[os], kXTileBytes + nb * L.b_bytes);
            tma_load_2d(op, &tmX, &op_full[os], x, y);
            tma_load_2d(op + kXTileBytes, &tmB0, &op_full[os], x, yb);
            if (nb == 3) {
              tma_load_2d(op + kXTileBytes + L.b_bytes, &tmB1, &op_full[os], x, yb);
              tma_load_2d(op + kXTileBytes + 2 * L.b_bytes, &tmB2, &op_full[os], x, yb);
            }
            continue;
          }
          const int rs = it % L.RS;
          const uint32_t rph = (it / L.RS) & 1u;
          if (!mbar_wait(&raw_empty[rs], rph ^ 1u, abort_flag)) { ok = false; break; }
          unsigned char* raw = smem + L.raw_off + rs * L.raw_bytes;
          const int nb = (L.mode == MODE_TF32X3) ? 2 : 1;  // B tiles per stage
          mbar_arrive_expect_tx(&op_full[os], nb * L.b_bytes);
          tma_load_2d(op + L.x_op_bytes, &tmB0, &op_full[os], x, yb);
          if (nb == 2) tma_load_2d(op + L.x_op_bytes + L.b_bytes, &tmB1, &op_full[os], x, yb);
          mbar_arrive_expect_tx(&raw_full[rs], L.raw_boxes * kXTileBytes);
          for (int b = 0; b < L.raw_boxes; ++b)
            tma_load_2d(raw + b * kXTileBytes, &tmX, &raw_full[rs], x + b * L.box_cols, y);
        }
      }
      if (!ok) {
        atomicExch(&s_abort, 1);
        atomicExch(&state->timeout, 3);
        // let the copies already issued land before the CTA can exit (bounded)
        for (int j = (it > L.OS ? it - L.OS : 0); j < it; ++j)
          mbar_wait(&op_full[j % L.OS], (j / L.OS) & 1u, nullptr, 50000000ull);
        if (convert)
          for (int j = (it > L.RS ? it - L.RS : 0); j < it; ++j)
            mbar_wait(&raw_full[j % L.RS], (j / L.RS) & 1u, nullptr, 50000000ull);
      }
    }
  } else if (warp == kWarpMma) {
    if (lane == 0) {
      const bool fp8 = L.mode == MODE_FP8_F32 || L.mode == MODE_FP8_BF16;
      const uint32_t id = (L.mode == MODE_TF32X3) ? idesc(FMT_TF32, FMT_TF32, kBM, L.N)
                          : fp8                   ? idesc(FMT_E4M3, FMT_E4M3, kBM, L.N)
                                                  : idesc(FMT_BF16, FMT_BF16, kBM, L.N);
      int it = 0, tcount = 0;
      bool ok = true;
      for (int w = blockIdx.x; w < nwork && ok; w += gridDim.x, ++tcount) {
        const int ab = tcount & 1;
        const uint32_t aph = (tcount >> 1) & 1u;
        if (!mbar_wait(&acc_empty[ab], aph ^ 1u, abort_flag)) { ok = false; break; }
        tc_fence_after();
        const uint32_t d_tmem = tmem_base + static_cast<uint32_t>(ab * L.N);
        for (int kb = 0; kb < L.KB; ++kb, ++it) {
          const int os = it % L.OS;
          const uint32_t oph = (it / L.OS) & 1u;
          if (!mbar_wait(&op_full[os], oph, abort_flag)) { ok = false; break; }
          if (convert && !mbar_wait(&cvt_full[os], oph, abort_flag)) { ok = false; break; }
          tc_fence_after();
          unsigned char* op = smem + L.op_off + os * L.op_bytes;
          if (L.mode == MODE_TF32X3) {
            const uint64_t ahi = sdesc_sw128(op), alo = sdesc_sw128(op + kXTileBytes);
            const uint64_t bhi = sdesc_sw128(op + 2 * kXTileBytes);
            const uint64_t blo = sdesc_sw128(op + 2 * kXTileBytes + L.b_bytes);
#pragma unroll
            for (int ks = 0; ks < 4; ++ks) {
              const uint64_t o = static_cast<uint64_t>(ks * 2);  // 32 bytes along K
              mma_tf32(d_tmem, ahi + o, bhi + o, id, (kb | ks) != 0);
              mma_tf32(d_tmem, ahi + o, blo + o, id, 1u);
              mma_tf32(d_tmem, alo + o, bhi + o, id, 1u);
            }
          } else if (L.mode == MODE_BF16X3) {
            const uint64_t a = sdesc_sw128(op);
            const uint64_t b0 = sdesc_sw128(op + kXTileBytes), b1 = sdesc_sw128(op + kXTileBytes + L.b_bytes);
            const uint64_t b2 = sdesc_sw128(op + kXTileBytes + 2 * L.b_bytes);
#pragma unroll
            for (int ks = 0; ks < 4; ++ks) {
              const uint64_t o = static_cast<uint64_t>(ks * 2);
              mma_f16(d_tmem, a + o, b0 + o, id, (kb | ks) != 0);
              mma_f16(d_tmem, a + o, b1 + o, id, 1u);
              mma_f16(d_tmem, a + o, b2 + o, id, 1u);
            }
          } else {
            const uint64_t a = sdesc_sw128(op), b = sdesc_sw128(op + kXTileBytes);
#pragma unroll
            for (int ks = 0; ks < 4; ++ks) {
              const uint64_t o = static_cast<uint64_t>(ks * 2);
              if (fp8) mma_f8(d_tmem, a + o, b + o, id, (kb | ks) != 0);
              else mma_f16(d_tmem, a + o, b + o, id, (kb | ks) != 0);
            }
          }
          mma_commit(&op_empty[os]);
        }
        if (!ok) break;
        mma_commit(&acc_full[ab]);
      }
      if (!ok) {
        atomicExch(&s_abort, 1);
        atomicExch(&state->timeout, 3);
      }
      // all MMAs issued by this thread have completed before TMEM is released
      if (it > 0) mbar_wait(&op_empty[(it - 1) % L.OS], ((it - 1) / L.OS) & 1u, nullptr, 50000000ull);
    }
  } else if (warp >= kWarpConvert0) {
    if (convert) {
      const int ct = threadIdx.x - kWarpConvert0 * 32;  // 0 .. kConvThreads-1
      int it = 0;
      bool ok = true;
      for (int w = blockIdx.x; w < nwork && ok; w += gridDim.x) {
        for (int kb = 0; kb < L.KB; ++kb, ++it) {
          const int rs = it % L.RS, os = it % L.OS;
          if (!mbar_wait(&raw_full[rs], (it / L.RS) & 1u, abort_flag)) { ok = false; break; }
          const unsigned char* raw = smem + L.raw_off + rs * L.raw_bytes;
          unsigned char* op = smem + L.op_off + os * L.op_bytes;
          if (L.mode == MODE_TF32X3) {
            // same element size and layout: chunk q of the float32 tile maps to chunk q of both
            const uint4* src = reinterpret_cast<const uint4*>(raw);
            uint4* hi = reinterpret_cast<uint4*>(op);
            uint4* lo = reinterpret_cast<uint4*>(op + kXTileBytes);
#pragma unroll
            for (int q = ct; q < static_cast<int>(kXTileBytes / 16); q += kConvThreads) {
              const uint4 v = src[q];
              uint4 h, l;
              split_tf32(v.x, h.x, l.x);
              split_tf32(v.y, h.y, l.y);
              split_tf32(v.z, h.z, l.z);
              split_tf32(v.w, h.w, l.w);
              hi[q] = h;
              lo[q] = l;
            }
          } else if (L.mode == MODE_FP8_F32 || L.mode == MODE_FP8_BF16) {
            // output row r, 16-byte chunk oc holds e4m3 elements 16oc..16oc+15 of this K-block,
            // i.e. X columns kb*128 + 16oc + t, each multiplied by its column scale first
            const float* cs = cscale + static_cast<int64_t>(kb) * 128;
#pragma unroll 2
            for (int q = ct; q < static_cast<int>(kXTileBytes / 16); q += kConvThreads) {
              const int r = q >> 3, oc = q & 7, sw = r & 7;
              float f[16];
              if (L.mode == MODE_FP8_F32) {  // four 32-column float32 boxes per K-block
                const float4* srow = reinterpret_cast<const float4*>(raw + (oc >> 1) * kXTileBytes + r * 128);
#pragma unroll
                for (int t = 0; t < 4; ++t) {
                  const float4 v = srow[((oc & 1) * 4 + t) ^ sw];
                  f[4 * t] = v.x; f[4 * t + 1] = v.y; f[4 * t + 2] = v.z; f[4 * t + 3] = v.w;
                }
              } else {  // two 64-column bfloat16 boxes per K-block
                const uint4* srow = reinterpret_cast<const uint4*>(raw + (oc >> 2) * kXTileBytes + r * 128);
#pragma unroll
                for (int t = 0; t < 2; ++t) {
                  const uint4 v = srow[((oc & 3) * 2 + t) ^ sw];
                  const uint32_t w[4] = {v.x, v.y, v.z, v.w};
#pragma unroll
                  for (int u = 0; u < 4; ++u) {
                    f[8 * t + 2 * u] = __uint_as_float(w[u] << 16);
                    f[8 * t + 2 * u + 1] = __uint_as_float(w[u] & 0xFFFF0000u);
                  }
                }
              }
              const float4* sc4 = reinterpret_cast<const float4*>(cs + oc * 16);
              uint32_t o[4];
#pragma unroll
              for (int t = 0; t < 4; ++t) {
                const float4 c = __ldg(sc4 + t);
                const __nv_fp8x2_storage_t lo2 =
                    __nv_cvt_float2_to_fp8x2(make_float2(f[4 * t] * c.x, f[4 * t + 1] * c.y), __NV_SATFINITE, __NV_E4M3);
                const __nv_fp8x2_storage_t hi2 =
                    __nv_cvt_float2_to_fp8x2(make_float2(f[4 * t + 2] * c.z, f[4 * t + 3] * c.w), __NV_SATFINITE, __NV_E4M3);
                o[t] = static_cast<uint32_t>(lo2) | (static_cast<uint32_t>(hi2) << 16);
              }
              reinterpret_cast<uint4*>(op + r * 128)[oc ^ sw] = make_uint4(o[0], o[1], o[2], o[3]);
            }
          } else {
            // output row r, 16-byte chunk oc holds bfloat16 elements 8oc..8oc+7 = float32 elements
            // of box oc/4, float32 chunks 2(oc%4) and 2(oc%4)+1; 128B swizzle: chunk c of row r
            // sits at position c ^ (r % 8).
#pragma unroll
            for (int q = ct; q < static_cast<int>(kXTileBytes / 16); q += kConvThreads) {
              const int r = q >> 3, oc = q & 7, sw = r & 7;
              const float4* srow = reinterpret_cast<const float4*>(raw + (oc >> 2) * kXTileBytes + r * 128);
              const int sc = (oc & 3) * 2;
              const float4 f0 = srow[sc ^ sw], f1 = srow[(sc + 1) ^ sw];
              const __nv_bfloat162 p0 = __floats2bfloat162_rn(f0.x, f0.y);
              const __nv_bfloat162 p1 = __floats2bfloat162_rn(f0.z, f0.w);
              const __nv_bfloat162 p2 = __floats2bfloat162_rn(f1.x, f1.y);
              const __nv_bfloat162 p3 = __floats2bfloat162_rn(f1.z, f1.w);
              uint4 o;
              o.x = *reinterpret_cast<const uint32_t*>(&p0);
              o.y = *reinterpret_cast<const uint32_t*>(&p1);
              o.z = *reinterpret_cast<const uint32_t*>(&p2);
              o.w = *reinterpret_cast<const uint32_t*>(&p3);
              reinterpret_cast<uint4*>(op + r * 128)[oc ^ sw] = o;
            }
          }
          fence_proxy_async_smem();
          mbar_arrive(&raw_empty[rs]);
          mbar_arrive(&cvt_full[os]);
        }
      }
      if (!ok) {
        atomicExch(&s_abort, 1);
        atomicExch(&state->timeout, 3);
      }
    }
  } else {  // warps 0-3: epilogue; warp w reads TMEM lanes 32w..32w+31 = tile rows 32w..32w+31
    const float post = post_scale ? *post_scale : 1.0f;
    int tcount = 0;
    bool ok = true;
    for (int w = blockIdx.x; w < nwork; w += gridDim.x, ++tcount) {
      const int tile = w / ncb;
      const int ab = tcount & 1;
      const uint32_t aph = (tcount >> 1) & 1u;
      int got = 0;
      if (lane == 0) got = mbar_wait(&acc_full[ab], aph, abort_flag) ? 1 : 0;
      got = __shfl_sync(0xFFFFFFFFu, got, 0);  // warp-uniform: tcgen05.ld is .sync.aligned
      if (!got) { ok = false; break; }
      tc_fence_after();
      const uint32_t taddr = tmem_base + (static_cast<uint32_t>(warp * 32) << 16) + static_cast<uint32_t>(ab * L.N);
      const int64_t row = static_cast<int64_t>(tile) * kBM + warp * 32 + lane;
      if (U) {  // Y = X M written out: this thread's row, columns of block w % ncb
        const int64_t col_base = static_cast<int64_t>(w % ncb) * L.N;
        float* urow = U + row * ldu + col_base;
        const bool vec = (ldu % 4 == 0) && ((reinterpret_cast<uintptr_t>(U) & 15u) == 0);
        for (int c0 = 0; c0 < L.N && col_base + c0 < ucols; c0 += 32) {
          float v[32];
          tmem_ld_32x32b_x32(taddr + static_cast<uint32_t>(c0), v);
          if (row >= n) continue;
          if (vec && col_base + c0 + 32 <= ucols) {
#pragma unroll
            for (int i = 0; i < 32; i += 4)
              *reinterpret_cast<float4*>(urow + c0 + i) = make_float4(v[i], v[i + 1], v[i + 2], v[i + 3]);
          } else {
#pragma unroll
            for (int i = 0; i < 32; ++i)
              if (col_base + c0 + i < ucols) urow[c0 + i] = v[i];
          }
        }
        tc_fence_before();
        mbar_arrive(&acc_empty[ab]);
        continue;
      }
      float sum = 0.0f;
      for (int c0 = 0; c0 < L.N; c0 += 32) {
        float v[32];
        tmem_ld_32x32b_x32(taddr + static_cast<uint32_t>(c0), v);
#pragma unroll
        for (int i = 0; i < 32; ++i) sum = fmaf(v[i], v[i], sum);
      }
      tc_fence_before();
      mbar_arrive(&acc_empty[ab]);
      if (row < n) scores[row] = sum * post;
    }
    if (!ok && lane == 0) {
      atomicExch(&s_abort, 1);
      atomicExch(&state->timeout, 3);
    }
  }

  tc_fence_before();
  __syncthreads();
  if (warp == kWarpMma) {
    tc_fence_after();
    tmem_dealloc(tmem_base, L.tmem_cols);
  }
}

// Two-tile form of the float32-accurate (3xTF32) scores for k <= 128: a work item is two
// 128-row tiles of X that share every K-block of B = M^T, so B's hi and lo tiles (the larger part
// of what each SM reads from L2 in the one-tile form) are read once per 256 rows.  X is converted
// in place: the TMA writes the float32 tile, the converters overwrite it with its tf32 high part
// and write the remainder beside it.  Stage layout (1024-byte aligned pieces): XA, XB (tiles 0, 1:
// float32, then hi), LA, LB (lo), BH, BL.  TMEM: two accumulator pairs (tiles 0, 1) of N columns,
// double-buffered across work items (4N <= 512 columns).  Warps 0-3 epilogue, 4 TMA producer,
// 5 TMEM owner and MMA issuer, 6-13 converters.  Every wait is bounded.  KBE float32 elements per
// K-block: 32 (128-byte rows, 128B swizzle) or 16 (64-byte rows, 64B swizzle: half the bytes per
// stage, so twice the stages fit and more copies are in flight).
struct Layout2T {
  int N, KB, S;
  int nbuf;  // accumulator sets in TMEM: 2 (the epilogue of one work item overlaps the next) or 1
  uint32_t b_bytes, stage_bytes, bar_off, smem_bytes, tmem_cols;
};

constexpr int kMaxStages2T = 4;

template <int KBE, int T>
__global__ void __launch_bounds__(kThreads, 1)
    score_tc2_kernel(const __grid_constant__ CUtensorMap tmX, const __grid_constant__ CUtensorMap tmBh,
                     const __grid_constant__ CUtensorMap tmBl, const Layout2T L, int64_t n, int nwork,
                     float* __restrict__ scores, DevState* __restrict__ state) {
  extern __shared__ unsigned char smem_dyn[];
  unsigned char* smem = reinterpret_cast<unsigned char*>((reinterpret_cast<uintptr_t>(smem_dyn) + 1023) &
                                                         ~static_cast<uintptr_t>(1023));
  uint64_t* full = reinterpret_cast<uint64_t*>(smem + L.bar_off);  // TMA bytes landed
  uint64_t* cvt = full + kMaxStages2T;                               // converters done
  uint64_t* empty = cvt + kMaxStages2T;                              // MMAs reading the stage done
  uint64_t* acc_full = empty + kMaxStages2T;
  uint64_t* acc_empty = acc_full + 2;
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(acc_empty + 2);
  __shared__ int s_abort;
  const volatile int* abort_flag = &s_abort;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  constexpr uint32_t kX = kBM * KBE * 4;  // one 128-row x KBE-float tile
  constexpr int kSteps = KBE / 8;         // tf32 MMAs take K = 8
  auto sdesc = [](const void* t) { return KBE == 32 ? sdesc_sw128(t) : sdesc_sw64(t); };

  if (threadIdx.x == 0) {
    s_abort = 0;
    for (int i = 0; i < L.S; ++i) {
      mbar_init(&full[i], 1);
      mbar_init(&cvt[i], kConvThreads);
      mbar_init(&empty[i], 1);
    }
    for (int i = 0; i < 2; ++i) {
      mbar_init(&acc_full[i], 1);
      mbar_init(&acc_empty[i], 128);
    }
    fence_mbar_init();
  }
  if (warp == kWarpMma) tmem_alloc(tmem_slot, L.tmem_cols);
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem_base = *tmem_slot;

  if (warp == kWarpProducer) {
    if (lane == 0) {
      int it = 0;
      bool ok = true;
      for (int w = blockIdx.x; w < nwork && ok; w += gridDim.x) {
        const int y0 = w * T * kBM;
        for (int kb = 0; kb < L.KB; ++kb, ++it) {
          const int st = it % L.S;
          if (!mbar_wait(&empty[st], ((it / L.S) & 1u) ^ 1u, abort_flag)) { ok = false; break; }
          unsigned char* stage = smem + static_cast<uint32_t>(st) * L.stage_bytes;
          const int x = kb * KBE;
          mbar_arrive_expect_tx(&full[st], T * kX + 2 * L.b_bytes);
#pragma unroll
          for (int u = 0; u < T; ++u) tma_load_2d(stage + u * kX, &tmX, &full[st], x, y0 + u * kBM);
          tma_load_2d(stage + 2 * T * kX, &tmBh, &full[st], x, 0);
          tma_load_2d(stage + 2 * T * kX + L.b_bytes, &tmBl, &full[st], x, 0);
        }
      }
      if (!ok) {
        atomicExch(&s_abort, 1);
        atomicExch(&state->timeout, 3);
        for (int j = (it > L.S ? it - L.S : 0); j < it; ++j)  // let issued copies land (bounded)
          mbar_wait(&full[j % L.S], (j / L.S) & 1u, nullptr, 50000000ull);
      }
    }
  } else if (warp == kWarpMma) {
    if (lane == 0) {
      const uint32_t id = idesc(FMT_TF32, FMT_TF32, kBM, static_cast<uint32_t>(L.N));
      int it = 0, tcount = 0;
      bool ok = true;
      for (int w = blockIdx.x; w < nwork && ok; w += gridDim.x, ++tcount) {
        const int ab = tcount % L.nbuf;
        if (!mbar_wait(&acc_empty[ab], ((tcount / L.nbuf) & 1u) ^ 1u, abort_flag)) { ok = false; break; }
        tc_fence_after();
        const uint32_t dbase = tmem_base + static_cast<uint32_t>(ab * T * L.N);
        for (int kb = 0; kb < L.KB; ++kb, ++it) {
          const int st = it % L.S;
          if (!mbar_wait(&cvt[st], (it / L.S) & 1u, abort_flag)) { ok = false; break; }
          tc_fence_after();
          unsigned char* stage = smem + static_cast<uint32_t>(st) * L.stage_bytes;
          const uint64_t bh = sdesc(stage + 2 * T * kX), bl = sdesc(stage + 2 * T * kX + L.b_bytes);
#pragma unroll
          for (int ks = 0; ks < kSteps; ++ks) {
            const uint64_t o = static_cast<uint64_t>(ks * 2);  // 32 bytes along K
            const uint32_t first = (kb | ks) != 0;
#pragma unroll
            for (int u = 0; u < T; ++u) {
              const uint32_t du = dbase + static_cast<uint32_t>(u * L.N);
              const uint64_t hu = sdesc(stage + u * kX), lu = sdesc(stage + (T + u) * kX);
              mma_tf32(du, hu + o, bh + o, id, first);
              mma_tf32(du, hu + o, bl + o, id, 1u);
              mma_tf32(du, lu + o, bh + o, id, 1u);
            }
          }
          mma_commit(&empty[st]);
        }
        if (!ok) break;
        mma_commit(&acc_full[ab]);
      }
      if (!ok) {
        atomicExch(&s_abort, 1);
        atomicExch(&state->timeout, 3);
      }
      // all MMAs issued by this thread have completed before TMEM is released
      if (it > 0) mbar_wait(&empty[(it - 1) % L.S], ((it - 1) / L.S) & 1u, nullptr, 50000000ull);
    }
  } else if (warp >= kWarpConvert0) {
    const int ct = threadIdx.x - kWarpConvert0 * 32;
    int it = 0;
    bool ok = true;
    for (int w = blockIdx.x; w < nwork && ok; w += gridDim.x) {
      for (int kb = 0; kb < L.KB; ++kb, ++it) {
        const int st = it % L.S;
        if (!mbar_wait(&full[st], (it / L.S) & 1u, abort_flag)) { ok = false; break; }
        unsigned char* stage = smem + static_cast<uint32_t>(st) * L.stage_bytes;
        // all tiles: chunk q of the X tiles (float32, the TMA's swizzled layout) -> hi in place and
        // lo at the same chunk of the lo tiles (same element size and layout)
        uint4* xs = reinterpret_cast<uint4*>(stage);
        uint4* ls = reinterpret_cast<uint4*>(stage + T * kX);
#pragma unroll 4
        for (int q = ct; q < static_cast<int>(T * kX / 16); q += kConvThreads) {
          const uint4 v = xs[q];
          uint4 h, l;
          split_tf32(v.x, h.x, l.x);
          split_tf32(v.y, h.y, l.y);
          split_tf32(v.z, h.z, l.z);
          split_tf32(v.w, h.w, l.w);
          xs[q] = h;
          ls[q] = l;
        }
        fence_proxy_async_smem();
        mbar_arrive(&cvt[st]);
      }
    }
    if (!ok) {
      atomicExch(&s_abort, 1);
      atomicExch(&state->timeout, 3);
    }
  } else {  // warps 0-3: epilogue; warp w reads TMEM lanes 32w..32w+31 = tile rows 32w..32w+31
    int tcount = 0;
    for (int w = blockIdx.x; w < nwork; w += gridDim.x, ++tcount) {
      const int ab = tcount % L.nbuf;
      int got = 0;
      if (lane == 0) got = mbar_wait(&acc_full[ab], (tcount / L.nbuf) & 1u, abort_flag) ? 1 : 0;
      got = __shfl_sync(0xFFFFFFFFu, got, 0);  // warp-uniform: tcgen05.ld is .sync.aligned
      if (!got) {
        if (lane == 0) {
          atomicExch(&s_abort, 1);
          atomicExch(&state->timeout, 3);
        }
        break;
      }
      tc_fence_after();
#pragma unroll
      for (int u = 0; u < T; ++u) {
        const uint32_t taddr = tmem_base + (static_cast<uint32_t>(warp * 32) << 16) +
                               static_cast<uint32_t>(ab * T * L.N + u * L.N);
        float sum = 0.0f;
        for (int c0 = 0; c0 < L.N; c0 += 32) {
          float v[32];
          tmem_ld_32x32b_x32(taddr + static_cast<uint32_t>(c0), v);
#pragma unroll
          for (int i = 0; i < 32; ++i) sum = fmaf(v[i], v[i], sum);
        }
        const int64_t row = (static_cast<int64_t>(w) * T + u) * kBM + warp * 32 + lane;
        if (row < n) scores[row] = sum;
      }
      tc_fence_before();
      mbar_arrive(&acc_empty[ab]);
    }
  }

  tc_fence_before();
  __syncthreads();
  if (warp == kWarpMma) {
    tc_fence_after();
    tmem_dealloc(tmem_base, L.tmem_cols);
  }
}

// Float32-accurate scores with X's low operand pieces in tensor memory, k <= 128.  X = Xhi + Xlo
// with Xhi = X truncated to tf32 (its top 19 bits) and Xlo = X - Xhi (exact in float32, below
// 2^-10 |X|).  The tf32 MMAs take A straight from the TMA's float32 tile in shared memory: the
// tensor core reads a float32 operand of kind::tf32 as its top 19 bits, which is Xhi.  The
// converters read each row of the tile once and write only what the raw tile cannot give to
// TMEM with tcgen05.st; those MMAs take A from TMEM.  K-blocks of 16 floats (64-byte rows, 64B
// swizzle).  Products, all accumulated in float32 in TMEM:
//   HYB = false (3xTF32): Xhi Mhi + Xhi Mlo (A from shared memory) + Xlo Mhi (A = tf32(Xlo) in
//               TMEM): 6 tf32 MMAs of K 8 per K-block and tile.
//   HYB = true:   Xhi Mhi in tf32 (exact products) plus bf16(Xlo) bf16(Mhi) + bf16(Xhi) bf16(Mlo)
//               in bfloat16 (2 tf32 + 2 bf16 MMAs of K 16: 2/3 of the tensor time): each dropped
//               or rounded term is below 2^-18 |x_il m_lj|.
// B = M^T is packed once per call so that one K-block of one column is one 128-byte row: its tf32
// high part (16 x 4 bytes), then either the bfloat16 high and low parts (16 x 2 bytes each) or the
// tf32 low part; one 128B-swizzled TMA box per stage carries all of B's pieces, and each product
// addresses its piece by the offset of its 32 bytes within the row.  The MMA thread issues a
// stage's shared-memory products as soon as the TMA's bytes land and the TMEM products once the
// converters are done.
// T = 2: a work item is two 128-row tiles that share each K-block of B, the whole K summed in one
//   accumulator per tile (nbuf sets of 2N columns; with two sets, which fit for k <= 64, the
//   epilogue of one item overlaps the next item's MMAs).
// T = 1, for long rows: the tensor core's float32 accumulation rounds its sums toward zero, a bias
//   that grows with the number of MMAs summed into one accumulator (about 2^-25 of the sum per
//   MMA: 1e-4 over the ~4000 MMAs of a 16800-long row).  K is cut into chunks of L.chunk K-blocks,
//   each summed into a fresh accumulator (two, ping-pong), and the epilogue adds every chunk into
//   a running sum kept in TMEM with round-to-nearest float32 additions.
// TMEM: the accumulators from column 0 (T = 1: then the running sum, N columns), then one A slot
// of 16 T columns per stage: per tile 16 columns = either tf32(Xlo) (16 tf32) or bf16(Xlo),
// bf16(Xhi) (8 columns each, two elements per column).  Converter warp w may only reach TMEM lanes
// 32 (w % 4) .. 32 (w % 4) + 31, so warp w converts rows 32 (w % 4) + lane of tile (w - 6) / 4
// (for T = 1 the warps of tile 1 only arrive).  Every wait is bounded.
struct LayoutTm {
  int N, KB, S, nbuf;           // stages (shared-memory tiles and TMEM A slots), accumulator sets
  int chunk, nchunk;            // K-blocks per accumulation chunk, chunks per work item
  uint32_t bh_bytes;            // the packed B tile (N x 128 B)
  uint32_t stage_bytes, bar_off, smem_bytes, run_col, abase, tmem_cols;
};

constexpr int kMaxStagesTm = 7;
constexpr uint32_t kXtTm = kBM * 16 * 4;  // one 128-row x 16-float tile
constexpr int kSlotTm = 16;               // TMEM A columns per tile and stage

template <bool HYB, int T, bool GROUP>
__global__ void __launch_bounds__(kThreads, 1)
    score_tm_kernel(const __grid_constant__ CUtensorMap tmX, const __grid_constant__ CUtensorMap tmBh,
                    const LayoutTm L, int64_t n, int nwork, float* __restrict__ scores,
                    DevState* __restrict__ state, const ScoreGroupJob* __restrict__ jobs, int njobs) {
  extern __shared__ unsigned char smem_dyn[];
  unsigned char* smem = reinterpret_cast<unsigned char*>((reinterpret_cast<uintptr_t>(smem_dyn) + 1023) &
                                                         ~static_cast<uintptr_t>(1023));
  uint64_t* full = reinterpret_cast<uint64_t*>(smem + L.bar_off);  // TMA bytes landed
  uint64_t* cvt = full + kMaxStagesTm;                              // A pieces in TMEM
  uint64_t* empty = cvt + kMaxStagesTm;                             // MMAs reading the stage done
  uint64_t* acc_full = empty + kMaxStagesTm;
  uint64_t* acc_empty = acc_full + 2;
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(acc_empty + 2);
  __shared__ int s_abort;
  const volatile int* abort_flag = &s_abort;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  // GROUP: work item w belongs to the job j with jobs[j].work0 <= w < jobs[j + 1].work0 and is that
  // job's item w - work0; every item is computed exactly as the one-job launch computes it
  auto job_of = [&](int w, int& lw) -> int {
    if (!GROUP) {
      lw = w;
      return 0;
    }
    int j = 0;
    while (j + 1 < njobs && w >= jobs[j + 1].work0) ++j;
    lw = w - jobs[j].work0;
    return j;
  };
  auto kb_of = [&](int j) { return GROUP ? jobs[j].KB : L.KB; };
  auto abort_all = [&](int code) {
    if (!GROUP) {
      atomicExch(&state->timeout, code);
      return;
    }
    for (int j = 0; j < njobs; ++j) atomicExch(&jobs[j].state->timeout, code);
  };

  if (threadIdx.x == 0) {
    s_abort = 0;
    for (int i = 0; i < L.S; ++i) {
      mbar_init(&full[i], 1);
      mbar_init(&cvt[i], kConvThreads);
      mbar_init(&empty[i], 1);
    }
    for (int i = 0; i < 2; ++i) {
      mbar_init(&acc_full[i], 1);
      mbar_init(&acc_empty[i], 128);
    }
    fence_mbar_init();
  }
  if (warp == kWarpMma) tmem_alloc(tmem_slot, L.tmem_cols);
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem_base = *tmem_slot;

  if (warp == kWarpProducer) {
    if (lane == 0) {
      if (GROUP)  // the jobs' tensor maps were written to global memory before the launch
        for (int j = 0; j < njobs; ++j) {
          const CUtensorMap* maps[2] = {&jobs[j].tmX, &jobs[j].tmBh};
#pragma unroll
          for (int m = 0; m < 2; ++m)
            asm volatile("fence.proxy.tensormap::generic.acquire.gpu [%0], 128;" ::"l"(maps[m]) : "memory");
        }
      int it = 0;
      bool ok = true;
      const uint32_t tx = T * kXtTm + L.bh_bytes;
      for (int w = blockIdx.x; w < nwork && ok; w += gridDim.x) {
        int lw;
        const int j = job_of(w, lw);
        const int y0 = lw * T * kBM, KB = kb_of(j);
        const CUtensorMap* mX = GROUP ? &jobs[j].tmX : &tmX;
        const CUtensorMap* mBh = GROUP ? &jobs[j].tmBh : &tmBh;
        for (int kb = 0; kb < KB; ++kb, ++it) {
          const int st = it % L.S;
          if (!mbar_wait(&empty[st], ((it / L.S) & 1u) ^ 1u, abort_flag)) { ok = false; break; }
          unsigned char* stage = smem + static_cast<uint32_t>(st) * L.stage_bytes;
          const int x = kb * 16;
          mbar_arrive_expect_tx(&full[st], tx);
#pragma unroll
          for (int u = 0; u < T; ++u) tma_load_2d(stage + u * kXtTm, mX, &full[st], x, y0 + u * kBM);
          tma_load_2d(stage + T * kXtTm, mBh, &full[st], 2 * x, 0);  // the packed B: 32 words per K-block
        }
      }
      if (!ok) {
        atomicExch(&s_abort, 1);
        abort_all(3);
        for (int j = (it > L.S ? it - L.S : 0); j < it; ++j)  // let issued copies land (bounded)
          mbar_wait(&full[j % L.S], (j / L.S) & 1u, nullptr, 50000000ull);
      }
    }
  } else if (warp == kWarpMma) {
    if (lane == 0) {
      const uint32_t idt = idesc(FMT_TF32, FMT_TF32, kBM, static_cast<uint32_t>(L.N));
      const uint32_t idb = idesc(FMT_BF16, FMT_BF16, kBM, static_cast<uint32_t>(L.N));
      // stage 0's descriptors; a stage's differ only in the start address field (address >> 4,
      // bits 0-13; shared memory is below 2^18 bytes, so no carry)
      const uint64_t x_0 = sdesc_sw64(smem);  // X's float32 tile u at + u kXtTm: A of the tf32 products
      const uint64_t bh_0 = sdesc_sw128(smem + T * kXtTm);  // packed B rows; pieces at + 0, 64, 96 bytes
      const uint64_t xt_off = static_cast<uint64_t>(kXtTm >> 4);
      int it = 0, cc = 0;  // K-blocks and accumulation chunks issued so far
      bool ok = true;
      uint32_t dbase = 0;
      for (int w = blockIdx.x; w < nwork && ok; w += gridDim.x) {
        int lw;
        const int KB = kb_of(job_of(w, lw));
        for (int kb = 0, kc = 0; kb < KB; ++kb, ++it) {  // kc: K-block within its chunk
          if (kc == 0) {                 // a fresh accumulator set for this chunk
            const int ab = cc % L.nbuf;
            if (!mbar_wait(&acc_empty[ab], ((cc / L.nbuf) & 1u) ^ 1u, abort_flag)) { ok = false; break; }
            tc_fence_after();
            dbase = tmem_base + static_cast<uint32_t>(ab * T * L.N);
          }
          const int st = it % L.S;
          const uint32_t par = (it / L.S) & 1u;
          if (!mbar_wait(&full[st], par, abort_flag)) { ok = false; break; }
          tc_fence_after();
          const uint64_t soff = static_cast<uint64_t>((static_cast<uint32_t>(st) * L.stage_bytes) >> 4);
          const uint64_t bh = bh_0 + soff, b1 = bh + 4, b2 = bh + 6;  // HYB: bf16(Mhi), bf16(Mlo); else b1 = Mlo
          // the products with A = X's raw tile (its tf32 high part): as soon as the bytes landed;
          // consecutive MMAs alternate between the tiles' accumulators
#pragma unroll
          for (int hk = 0; hk < 2; ++hk)  // the two K halves of 8 (+ 32 bytes along K)
#pragma unroll
            for (int u = 0; u < T; ++u) {
              const uint32_t du = dbase + static_cast<uint32_t>(u * L.N);
              const uint64_t xa = x_0 + soff + static_cast<uint64_t>(u) * xt_off + static_cast<uint64_t>(2 * hk);
              mma_tf32(du, xa, bh + 2 * hk, idt, (kc | hk) != 0);
            }
          if (!HYB)  // Xhi Mlo
#pragma unroll
            for (int hk = 0; hk < 2; ++hk)
#pragma unroll
              for (int u = 0; u < T; ++u) {
                const uint32_t du = dbase + static_cast<uint32_t>(u * L.N);
                const uint64_t xa = x_0 + soff + static_cast<uint64_t>(u) * xt_off + static_cast<uint64_t>(2 * hk);
                mma_tf32(du, xa, b1 + 2 * hk, idt, 1u);
              }
          if (!mbar_wait(&cvt[st], par, abort_flag)) {  // the MMAs issued above complete first
            mma_commit(&empty[st]);
            ++it;
            ok = false;
            break;
          }
          tc_fence_after();
          const uint32_t aslot = tmem_base + L.abase + static_cast<uint32_t>(st * kSlotTm * T);
#pragma unroll
          for (int pc = 0; pc < 2; ++pc)
#pragma unroll
            for (int u = 0; u < T; ++u) {
              const uint32_t du = dbase + static_cast<uint32_t>(u * L.N);
              const uint32_t a = aslot + static_cast<uint32_t>(u * kSlotTm + 8 * pc);
              if (HYB)  // bf16(Xlo) bf16(Mhi), then bf16(Xhi) bf16(Mlo)
                mma_f16_ts(du, a, pc ? b2 : b1, idb, 1u);
              else      // tf32(Xlo) Mhi, the two K halves
                mma_tf32_ts(du, a, bh + 2 * pc, idt, 1u);
            }
          mma_commit(&empty[st]);
          if (++kc == (T == 1 ? L.chunk : KB) || kb == KB - 1) {  // the chunk is summed
            mma_commit(&acc_full[cc % L.nbuf]);
            ++cc;
            kc = 0;
          }
        }
      }
      if (!ok) {
        atomicExch(&s_abort, 1);
        abort_all(3);
      }
      // all MMAs issued by this thread have completed before TMEM is released
      if (it > 0) mbar_wait(&empty[(it - 1) % L.S], ((it - 1) / L.S) & 1u, nullptr, 50000000ull);
    }
  } else if (warp >= kWarpConvert0) {
    const int u = (warp - kWarpConvert0) >> 2;  // tile
    const int q = warp & 3;                      // TMEM lane quarter
    const int r = q * 32 + lane;                 // row of the tile
    const uint32_t lane_addr = static_cast<uint32_t>(q * 32) << 16;
    int it = 0;
    bool ok = true;
    for (int w = blockIdx.x; w < nwork && ok; w += gridDim.x) {
      int lw;
      const int KB = kb_of(job_of(w, lw));
      for (int kb = 0; kb < KB; ++kb, ++it) {
        const int st = it % L.S;
        // every lane acquires the TMA's bytes (the stage, and with it its TMEM slot, was freed by
        // the MMAs before the producer refilled it); the outcome is made warp-uniform (tcgen05.st
        // is .sync.aligned)
        const bool got = mbar_wait(&full[st], (it / L.S) & 1u, abort_flag);
        if (!__all_sync(0xFFFFFFFFu, got)) { ok = false; break; }
        if (u < T) {
          // row r of the tile: 64 bytes, 16-byte chunk c stored at chunk c ^ ((r >> 1) & 3)
          const uint4* row = reinterpret_cast<const uint4*>(smem + static_cast<uint32_t>(st) * L.stage_bytes +
                                                            u * kXtTm + r * 64);
          uint32_t x[16];
#pragma unroll
          for (int c = 0; c < 4; ++c) {
            const uint4 v = row[c ^ ((r >> 1) & 3)];
            x[4 * c] = v.x;
            x[4 * c + 1] = v.y;
            x[4 * c + 2] = v.z;
            x[4 * c + 3] = v.w;
          }
          // Xhi = x with its low 13 bits cleared: what the tensor core reads from the raw tile
          uint32_t a[16];
          if (HYB) {
#pragma unroll
            for (int e = 0; e < 16; e += 2) {
              const float h0 = __uint_as_float(x[e] & 0xFFFFE000u), h1 = __uint_as_float(x[e + 1] & 0xFFFFE000u);
              const __nv_bfloat162 lp =
                  __floats2bfloat162_rn(__uint_as_float(x[e]) - h0, __uint_as_float(x[e + 1]) - h1);  // .x = element e
              const __nv_bfloat162 hp = __floats2bfloat162_rn(h0, h1);
              a[e / 2] = *reinterpret_cast<const uint32_t*>(&lp);
              a[8 + e / 2] = *reinterpret_cast<const uint32_t*>(&hp);
            }
          } else {
#pragma unroll
            for (int e = 0; e < 16; ++e)
              a[e] = rne_tf32(__float_as_uint(__uint_as_float(x[e]) - __uint_as_float(x[e] & 0xFFFFE000u)));
          }
          tmem_st_32x32b_x16(tmem_base + lane_addr + L.abase + static_cast<uint32_t>((st * T + u) * kSlotTm), a);
          tc_fence_before();
        }
        mbar_arrive(&cvt[st]);
      }
    }
    if (!ok && lane == 0) {
      atomicExch(&s_abort, 1);
      abort_all(3);
    }
  } else {  // warps 0-3: epilogue; warp w reads TMEM lanes 32w..32w+31 = tile rows 32w..32w+31
    int cc = 0;
    const uint32_t lanes = static_cast<uint32_t>(warp * 32) << 16;
    for (int w = blockIdx.x; w < nwork; w += gridDim.x) {
      float sum[T];
#pragma unroll
      for (int u = 0; u < T; ++u) sum[u] = 0.0f;
      bool ok = true;
      const int nchunk = T == 1 ? L.nchunk : 1;
      for (int ci = 0; ci < nchunk; ++ci, ++cc) {
        const int ab = cc % L.nbuf;
        int got = 0;
        if (lane == 0) got = mbar_wait(&acc_full[ab], (cc / L.nbuf) & 1u, abort_flag) ? 1 : 0;
        got = __shfl_sync(0xFFFFFFFFu, got, 0);  // warp-uniform: tcgen05.ld is .sync.aligned
        if (!got) { ok = false; break; }
        tc_fence_after();
        const bool last = ci == nchunk - 1;
#pragma unroll
        for (int u = 0; u < T; ++u) {
          const uint32_t taddr = tmem_base + lanes + static_cast<uint32_t>(ab * T * L.N + u * L.N);
          for (int c0 = 0; c0 < L.N; c0 += 32) {
            float v[32];
            tmem_ld_32x32b_x32(taddr + static_cast<uint32_t>(c0), v);
            if (T == 1 && L.nchunk > 1) {  // fold into the running sum (round to nearest)
              const uint32_t raddr = tmem_base + lanes + L.run_col + static_cast<uint32_t>(c0);
              if (ci > 0) {
                float rs[32];
                tmem_ld_32x32b_x32(raddr, rs);
#pragma unroll
                for (int i = 0; i < 32; ++i) v[i] = __fadd_rn(v[i], rs[i]);
              }
              if (!last) {
                uint32_t vb[32];
#pragma unroll
                for (int i = 0; i < 32; ++i) vb[i] = __float_as_uint(v[i]);
                tmem_st_32x32b_x32(raddr, vb);
              }
            }
            if (last)
#pragma unroll
              for (int i = 0; i < 32; ++i) sum[u] = fmaf(v[i], v[i], sum[u]);
          }
        }
        tc_fence_before();
        mbar_arrive(&acc_empty[ab]);  // the accumulators are read: the next chunk may start
      }
      if (!ok) {
        if (lane == 0) {
          atomicExch(&s_abort, 1);
          abort_all(3);
        }
        break;
      }
      int lw;
      const int j = job_of(w, lw);
      const int64_t nj = GROUP ? jobs[j].n : n;
      float* out = GROUP ? jobs[j].scores : scores;
#pragma unroll
      for (int u = 0; u < T; ++u) {
        const int64_t row = (static_cast<int64_t>(lw) * T + u) * kBM + warp * 32 + lane;
        if (row < nj) out[row] = sum[u];
      }
    }
  }

  tc_fence_before();
  __syncthreads();
  if (warp == kWarpMma) {
    tc_fence_after();
    tmem_dealloc(tmem_base, L.tmem_cols);
  }
}

// B = M^T packed for score_tm_kernel: row c holds, for each K-block b of 16, 32 words: tf32(m) for
// k = 16b .. 16b + 15, then (hyb) the bfloat16 roundings of tf32(m) and of m - tf32(m), 16 each,
// or the tf32 rounding of m - tf32(m).
__global__ void prep_b_packed_kernel(const double* __restrict__ M, int64_t d, int64_t kk, int64_t N, int64_t Kpad,
                                     int hyb, float* __restrict__ B) {
  for (int64_t e = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; e < N * Kpad;
       e += static_cast<int64_t>(gridDim.x) * blockDim.x) {
    const int64_t c = e / Kpad, k = e % Kpad;
    const double m = (c < kk && k < d) ? M[k * kk + c] : 0.0;
    const float hi = __uint_as_float(rne_tf32(__float_as_uint(static_cast<float>(m))));
    float* row = B + (c * (Kpad / 16) + k / 16) * 32;
    const int q = static_cast<int>(k % 16);
    row[q] = hi;
    if (hyb) {
      __nv_bfloat16* r16 = reinterpret_cast<__nv_bfloat16*>(row + 16);
      r16[q] = __float2bfloat16_rn(hi);
      r16[16 + q] = __float2bfloat16_rn(static_cast<float>(m - static_cast<double>(hi)));
    } else {
      row[16 + q] = __uint_as_float(rne_tf32(__float_as_uint(static_cast<float>(m - static_cast<double>(hi)))));
    }
  }
}

// B = M^T (N x Kpad, K contiguous) split into tf32-exact high parts and float32 remainders.
__global__ void prep_b_tf32_kernel(const double* __restrict__ M, int64_t d, int64_t kk, int64_t N, int64_t Kpad,
                                   float* __restrict__ Bhi, float* __restrict__ Blo) {
  for (int64_t e = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; e < N * Kpad;
       e += static_cast<int64_t>(gridDim.x) * blockDim.x) {
    const int64_t c = e / Kpad, k = e % Kpad;
    const double m = (c < kk && k < d) ? M[k * kk + c] : 0.0;
    const float hi = __uint_as_float(rne_tf32(__float_as_uint(static_cast<float>(m))));
    Bhi[e] = hi;
    Blo[e] = __uint_as_float(rne_tf32(__float_as_uint(static_cast<float>(m - static_cast<double>(hi)))));
  }
}

__global__ void prep_b_bf16_kernel(const double* __restrict__ M, int64_t d, int64_t kk, int64_t N, int64_t Kpad,
                                   __nv_bfloat16* __restrict__ B) {
  for (int64_t e = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; e < N * Kpad;
       e += static_cast<int64_t>(gridDim.x) * blockDim.x) {
    const int64_t c = e / Kpad, k = e % Kpad;
    const double m = (c < kk && k < d) ? M[k * kk + c] : 0.0;
    B[e] = __float2bfloat16_rn(static_cast<float>(m));
  }
}

// M^T as three bfloat16 pieces: m = p1 + p2 + p3 (+ a remainder below 2^-24 |m|), each the
// nearest bfloat16 to what is left.
__global__ void prep_b_bf16x3_kernel(const double* __restrict__ M, int64_t d, int64_t kk, int64_t N, int64_t Kpad,
                                     __nv_bfloat16* __restrict__ B0, __nv_bfloat16* __restrict__ B1,
                                     __nv_bfloat16* __restrict__ B2) {
  for (int64_t e = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; e < N * Kpad;
       e += static_cast<int64_t>(gridDim.x) * blockDim.x) {
    const int64_t c = e / Kpad, k = e % Kpad;
    double m = (c < kk && k < d) ? M[k * kk + c] : 0.0;
    const __nv_bfloat16 p1 = __float2bfloat16_rn(static_cast<float>(m));
    m -= static_cast<double>(__bfloat162float(p1));
    const __nv_bfloat16 p2 = __float2bfloat16_rn(static_cast<float>(m));
    m -= static_cast<double>(__bfloat162float(p2));
    B0[e] = p1;
    B1[e] = p2;
    B2[e] = __float2bfloat16_rn(static_cast<float>(m));
  }
}

Layout make_layout(int mode, int64_t kk, int64_t d) {
  Layout L{};
  L.mode = mode;
  L.N = static_cast<int>(ceil_div(kk, 32) * 32);  // whole 32-column TMEM loads in the epilogue
  const bool fp8 = mode == MODE_FP8_F32 || mode == MODE_FP8_BF16;
  L.kbe = (mode == MODE_TF32X3) ? 32 : (fp8 ? 128 : 64);  // one 128-byte operand row per K-block
  L.KB = static_cast<int>(ceil_div(d, L.kbe));
  L.b_bytes = static_cast<uint32_t>(L.N) * 128u;
  L.box_cols = (direct_x(mode) || mode == MODE_FP8_BF16) ? 64 : 32;
  L.raw_boxes = direct_x(mode) ? 0 : L.kbe / L.box_cols;
  L.x_op_bytes = (mode == MODE_TF32X3) ? 2 * kXTileBytes : kXTileBytes;
  const uint32_t budget = 226u * 1024u;  // + 1.5 KB barriers and alignment slack <= 227 KB
  L.raw_bytes = static_cast<uint32_t>(L.raw_boxes) * kXTileBytes;
  L.op_bytes = L.x_op_bytes + static_cast<uint32_t>(b_tiles(mode)) * L.b_bytes;
  if (direct_x(mode)) {
    L.OS = static_cast<int>(std::min<uint32_t>(kMaxStages, budget / L.op_bytes));
    L.RS = 1;
  } else {
    // as many operand stages as leave room for two raw stages (at most 3), then raw stages
    L.OS = static_cast<int>(std::max<uint32_t>(2, std::min<uint32_t>(3, (budget - 2 * L.raw_bytes) / L.op_bytes)));
    L.RS = static_cast<int>(std::min<uint32_t>(4, (budget - L.OS * L.op_bytes) / L.raw_bytes));
  }
  L.raw_off = 0;
  L.op_off = L.raw_bytes * static_cast<uint32_t>(direct_x(mode) ? 0 : L.RS);
  L.bar_off = L.op_off + L.op_bytes * static_cast<uint32_t>(L.OS);
  L.smem_bytes = L.bar_off + 64 * 8 + 1024;  // barriers + TMEM slot + alignment slack
  uint32_t cols = 32;
  while (cols < static_cast<uint32_t>(2 * L.N)) cols <<= 1;
  L.tmem_cols = cols;
  return L;
}

// max_i |x_ij| per column (as float bits; values are >= 0 so integer max orders them).
template <class T>
__global__ void colabsmax_kernel(const T* __restrict__ X, int64_t n, int64_t d, int64_t ldx, int64_t rows_per_cta,
                                 unsigned int* __restrict__ colmax) {
  const int64_t c = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x;
  if (c >= d) return;
  const int64_t r0 = static_cast<int64_t>(blockIdx.y) * rows_per_cta;
  const int64_t r1 = r0 + rows_per_cta < n ? r0 + rows_per_cta : n;
  float m = 0.0f;
  for (int64_t r = r0; r < r1; ++r) m = fmaxf(m, fabsf(to_float(X[r * ldx + c])));
  atomicMax(colmax + c, __float_as_uint(m));
}

// Column scales c_j = 448 / max |x_:j| (1 for empty or padded columns), and the single scale e of
// M' = diag(1/c) M: e = 448 / max |M'| and post = 1/e^2.
__global__ void fp8_scales_kernel(const unsigned int* __restrict__ colmax, const double* __restrict__ M, int64_t d,
                                  int64_t kk, int64_t Kpad, float* __restrict__ cscale, float* __restrict__ escale) {
  __shared__ float red[32];
  for (int64_t j = threadIdx.x; j < Kpad; j += blockDim.x) {
    const float a = j < d ? __uint_as_float(colmax[j]) : 0.0f;
    cscale[j] = a > 0.0f ? 448.0f / a : 1.0f;
  }
  __syncthreads();
  float m = 0.0f;
  for (int64_t e = threadIdx.x; e < d * kk; e += blockDim.x)
    m = fmaxf(m, static_cast<float>(fabs(M[e]) / static_cast<double>(cscale[e / kk])));
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) m = fmaxf(m, __shfl_xor_sync(0xFFFFFFFFu, m, o));
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = m;
  __syncthreads();
  if (threadIdx.x == 0) {
    float t = 0.0f;
    for (int w = 0; w < static_cast<int>(blockDim.x >> 5); ++w) t = fmaxf(t, red[w]);
    const float e = t > 0.0f ? 448.0f / t : 1.0f;
    escale[0] = e;
    escale[1] = 1.0f / (e * e);
  }
}

// B = e4m3(e M^T diag(1/c)) as N x Kpad bytes, K contiguous.
__global__ void prep_b_fp8_kernel(const double* __restrict__ M, int64_t d, int64_t kk, int64_t N, int64_t Kpad,
                                  const float* __restrict__ cscale, const float* __restrict__ escale,
                                  __nv_fp8_storage_t* __restrict__ B) {
  const float e = escale[0];
  for (int64_t i = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; i < N * Kpad;
       i += static_cast<int64_t>(gridDim.x) * blockDim.x) {
    const int64_t c = i / Kpad, k = i % Kpad;
    const float m = (c < kk && k < d) ? static_cast<float>(M[k * kk + c] / static_cast<double>(cscale[k])) * e : 0.0f;
    B[i] = __nv_cvt_float_to_fp8(m, __NV_SATFINITE, __NV_E4M3);
  }
}

}  // namespace

// TMEM columns, stages and shared memory of the score_tm layout (T.N set).  Two tiles: nbuf
// accumulator sets of 2N columns (two when that still leaves four A slots); one tile: two chunk
// accumulators and the running sum, 3N columns.  Then as many stages as TMEM's 512 columns and
// 227 KB of shared memory hold, at most kMaxStagesTm.
static void tm_stages(LayoutTm& T, int tiles) {
  const int slot = kSlotTm * tiles;
  T.bh_bytes = static_cast<uint32_t>(T.N) * 128u;
  T.stage_bytes = static_cast<uint32_t>(tiles) * kXtTm + T.bh_bytes;
  int acc;
  if (tiles == 2) {
    T.nbuf = (4 * T.N + 4 * slot <= 512) ? 2 : 1;
    T.run_col = 0;
    acc = T.nbuf * 2 * T.N;
  } else {
    T.nbuf = 2;
    T.run_col = static_cast<uint32_t>(2 * T.N);
    acc = 3 * T.N;
  }
  T.abase = static_cast<uint32_t>(acc);
  const uint32_t fixed = (3 * kMaxStagesTm + 4) * 8 + 8 + 1024;
  const int by_smem = static_cast<int>((227u * 1024u - fixed) / T.stage_bytes);
  T.S = std::min(kMaxStagesTm, std::min((512 - acc) / slot, by_smem));
  T.tmem_cols = 512;
  T.bar_off = static_cast<uint32_t>(T.S) * T.stage_bytes;
  T.smem_bytes = T.bar_off + fixed;
}

// Scores on the tensor cores when the shapes allow it; *used = false means the caller must
// take the SIMT kernel instead (k > 256, unaligned X, or an unsupported dtype pair).
slso_status run_scores_tc(Handle& h, Arena& ar, const void* X, int64_t n, int64_t d, int64_t ldx, int32_t xdt,
                          const double* M, int64_t kk, int32_t compute, float* scores, bool* used,
                          cudaStream_t st, const unsigned int* colmax_pre, ScoreGroupJob* group) {
  *used = false;
  int mode = -1;
  if (xdt == SLSO_F32 && compute == SLSO_F32) mode = MODE_TF32X3;
  if (xdt == SLSO_F32 && compute == SLSO_BF16) mode = MODE_BF16_CVT;
  if (xdt == SLSO_BF16 && compute == SLSO_BF16) mode = MODE_BF16;
  if (xdt == SLSO_BF16 && compute == SLSO_F32) mode = MODE_BF16X3;
  if (xdt == SLSO_F32 && compute == SLSO_FP8_E4M3) mode = MODE_FP8_F32;
  if (xdt == SLSO_BF16 && compute == SLSO_FP8_E4M3) mode = MODE_FP8_BF16;
  if (mode < 0 || kk > 256 || kk < 1) return SLSO_OK;
  const size_t esz = dtype_size(xdt);
  if (!encode_fn()) return SLSO_OK;
  if (reinterpret_cast<uintptr_t>(X) % 16 != 0 || (ldx * esz) % 16 != 0) {
    // TMA rows start on 16-byte boundaries: stage X once with its row pitch rounded up to 16
    // bytes (a strided copy at copy bandwidth, far cheaper than the SIMT product)
    const int64_t ldp = ceil_div(d * static_cast<int64_t>(esz), 16) * 16 / static_cast<int64_t>(esz);
    char* Xp = ar.take<char>(static_cast<size_t>(n) * ldp * esz);
    if (!ar.measure() && n > 0)
      SLSO_CHECK_CUDA(cudaMemcpy2DAsync(Xp, ldp * esz, X, ldx * esz, d * esz, n, cudaMemcpyDeviceToDevice, st));
    X = Xp;
    ldx = ldp;
  }
  const Layout L = make_layout(mode, kk, d);
  const int64_t Kpad = static_cast<int64_t>(L.KB) * L.kbe;
  const bool fp8 = mode == MODE_FP8_F32 || mode == MODE_FP8_BF16;
  void* B0 = nullptr;
  void* B1 = nullptr;
  void* B2 = nullptr;
  unsigned int* colmax = nullptr;
  float* cscale = nullptr;
  float* escale = nullptr;
  if (mode == MODE_TF32X3) {  // B0 also holds the packed B of the tensor-memory form (2 N Kpad words)
    B0 = ar.take<float>(2 * static_cast<size_t>(L.N) * Kpad);
    B1 = ar.take<float>(static_cast<size_t>(L.N) * Kpad);
  } else if (fp8) {
    B0 = ar.take<__nv_fp8_storage_t>(static_cast<size_t>(L.N) * Kpad);
    colmax = ar.take<unsigned int>(d);
    cscale = ar.take<float>(Kpad);
    escale = ar.take<float>(2);
  } else if (mode == MODE_BF16X3) {
    B0 = ar.take<__nv_bfloat16>(static_cast<size_t>(L.N) * Kpad);
    B1 = ar.take<__nv_bfloat16>(static_cast<size_t>(L.N) * Kpad);
    B2 = ar.take<__nv_bfloat16>(static_cast<size_t>(L.N) * Kpad);
  } else {
    B0 = ar.take<__nv_bfloat16>(static_cast<size_t>(L.N) * Kpad);
  }
  *used = true;
  if (ar.measure()) return SLSO_OK;
  const int pg = static_cast<int>(std::max<int64_t>(1, std::min<int64_t>(ceil_div(L.N * Kpad, 256), 4LL * h.num_sms)));
  CUtensorMap mX, mB0, mB1, mB2;
  bool ok;
  const CUtensorMapDataType xdt_map = (xdt == SLSO_F32) ? CU_TENSOR_MAP_DATA_TYPE_FLOAT32 : CU_TENSOR_MAP_DATA_TYPE_BFLOAT16;
  ok = make_map(&mX, xdt_map, X, d, n, ldx * esz, static_cast<uint32_t>(L.box_cols), kBM);
  // the shared-memory form sums K in one accumulator: rows longer than 2048 take the chunked form
  const bool tm = mode == MODE_TF32X3 && L.N <= 128 && (h.score_form != SLSO_SCORE_FORM_TF32X3_SMEM || d > 2048);
  if (group && !tm) return fail(SLSO_ERR_SHAPE, "internal: grouped scores need the tensor-memory form");
  const bool hyb = tm && h.score_form == SLSO_SCORE_FORM_MIXED;
  if (mode == MODE_TF32X3) {
    if (!tm) {  // the tensor-memory form packs its own pieces below
      prep_b_tf32_kernel<<<pg, 256, 0, st>>>(M, d, kk, L.N, Kpad, static_cast<float*>(B0), static_cast<float*>(B1));
      SLSO_CHECK_LAUNCH();
    }
    ok = ok && make_map(&mB0, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, B0, Kpad, L.N, Kpad * 4, 32, L.N) &&
         make_map(&mB1, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, B1, Kpad, L.N, Kpad * 4, 32, L.N);
    mB2 = mB1;
  } else if (fp8) {
    if (!colmax_pre) {  // the column maxima by a pass of their own (no sketch pass formed them)
      SLSO_CHECK_CUDA(cudaMemsetAsync(colmax, 0, sizeof(unsigned int) * d, st));
      const int64_t rows_per_cta = std::max<int64_t>(1024, ceil_div(n, 256));
      dim3 g(static_cast<unsigned>(ceil_div(d, 256)), static_cast<unsigned>(ceil_div(n, rows_per_cta)));
      if (xdt == SLSO_F32)
        colabsmax_kernel<float><<<g, 256, 0, st>>>(static_cast<const float*>(X), n, d, ldx, rows_per_cta, colmax);
      else
        colabsmax_kernel<__nv_bfloat16><<<g, 256, 0, st>>>(static_cast<const __nv_bfloat16*>(X), n, d, ldx,
                                                          rows_per_cta, colmax);
      SLSO_CHECK_LAUNCH();
    }
    fp8_scales_kernel<<<1, 1024, 0, st>>>(colmax_pre ? colmax_pre : colmax, M, d, kk, Kpad, cscale, escale);
    SLSO_CHECK_LAUNCH();
    prep_b_fp8_kernel<<<pg, 256, 0, st>>>(M, d, kk, L.N, Kpad, cscale, escale,
                                          static_cast<__nv_fp8_storage_t*>(B0));
    SLSO_CHECK_LAUNCH();
    ok = ok && make_map(&mB0, CU_TENSOR_MAP_DATA_TYPE_UINT8, B0, Kpad, L.N, Kpad, 128, L.N);
    mB1 = mB2 = mB0;
  } else if (mode == MODE_BF16X3) {
    prep_b_bf16x3_kernel<<<pg, 256, 0, st>>>(M, d, kk, L.N, Kpad, static_cast<__nv_bfloat16*>(B0),
                                             static_cast<__nv_bfloat16*>(B1), static_cast<__nv_bfloat16*>(B2));
    SLSO_CHECK_LAUNCH();
    ok = ok && make_map(&mB0, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, B0, Kpad, L.N, Kpad * 2, 64, L.N) &&
         make_map(&mB1, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, B1, Kpad, L.N, Kpad * 2, 64, L.N) &&
         make_map(&mB2, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, B2, Kpad, L.N, Kpad * 2, 64, L.N);
  } else {
    prep_b_bf16_kernel<<<pg, 256, 0, st>>>(M, d, kk, L.N, Kpad, static_cast<__nv_bfloat16*>(B0));
    SLSO_CHECK_LAUNCH();
    ok = ok && make_map(&mB0, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, B0, Kpad, L.N, Kpad * 2, 64, L.N);
    mB1 = mB2 = mB0;
  }
  if (!ok) return fail(SLSO_ERR_CUDA, "cuTensorMapEncodeTiled rejected a score operand layout");
  const int ntiles = static_cast<int>(ceil_div(n, kBM));
  if (tm) {
    // X's operand pieces in TMEM; K-blocks of 16 floats.  Rows up to 2048 long: two tiles per
    // work item, one accumulator per tile; longer rows: one tile, K summed in chunks of 512
    LayoutTm T{};
    T.N = L.N;
    T.KB = static_cast<int>(ceil_div(d, 16));
    const int tiles = T.KB > 128 ? 1 : 2;
    T.chunk = tiles == 1 ? 32 : T.KB;
    T.nchunk = static_cast<int>(ceil_div(T.KB, T.chunk));
    tm_stages(T, tiles);
    // B packed (Kpad is a multiple of 32 floats, so of 16): N rows of Kpad / 16 blocks of 32 words
    CUtensorMap mXt, mBh;
    prep_b_packed_kernel<<<pg, 256, 0, st>>>(M, d, kk, L.N, Kpad, hyb ? 1 : 0, static_cast<float*>(B0));
    SLSO_CHECK_LAUNCH();
    const bool okt = make_map(&mXt, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, X, d, n, ldx * esz, 16, kBM,
                              CU_TENSOR_MAP_SWIZZLE_64B) &&
                     make_map(&mBh, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, B0, 2 * Kpad, L.N, 2 * Kpad * 4, 32, L.N,
                              CU_TENSOR_MAP_SWIZZLE_128B);
    if (!okt) return fail(SLSO_ERR_CUDA, "cuTensorMapEncodeTiled rejected a score operand layout");
    const int nwork = (ntiles + tiles - 1) / tiles;
    if (group) {  // described for a grouped launch instead of launched
      if (tiles != 2) return fail(SLSO_ERR_SHAPE, "internal: grouped scores need rows of at most 2048");
      group->tmX = mXt;
      group->tmBh = mBh;
      group->n = n;
      group->scores = scores;
      group->state = h.state;
      group->KB = T.KB;
      group->work0 = nwork;  // the job's work items until score_group_launch numbers them
      group->N = L.N;
      group->hyb = hyb ? 1 : 0;
      return SLSO_OK;
    }
    const int gridt = std::min(nwork, h.num_sms);
    auto launch = [&](auto kern) -> slso_status {
      SLSO_TRY(raise_smem_limit(kern, T.smem_bytes));
      kern<<<gridt, kThreads, T.smem_bytes, st>>>(mXt, mBh, T, n, nwork, scores, h.state, nullptr, 0);
      SLSO_CHECK_LAUNCH();
      return SLSO_OK;
    };
    if (hyb) return tiles == 2 ? launch(score_tm_kernel<true, 2, false>) : launch(score_tm_kernel<true, 1, false>);
    return tiles == 2 ? launch(score_tm_kernel<false, 2, false>) : launch(score_tm_kernel<false, 1, false>);
  }
  if (mode == MODE_TF32X3 && L.N <= 128) {
    // two 128-row tiles per work item share each B K-block
    // K-blocks of 16 floats (64-byte rows, 64B swizzle): 4 stages of 48 KB at k = 128
    constexpr int kbe = 16;
    CUtensorMap mX16, mBh16, mBl16;
    const bool ok16 = make_map(&mX16, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, X, d, n, ldx * esz, kbe, kBM,
                               CU_TENSOR_MAP_SWIZZLE_64B) &&
                      make_map(&mBh16, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, B0, Kpad, L.N, Kpad * 4, kbe, L.N,
                               CU_TENSOR_MAP_SWIZZLE_64B) &&
                      make_map(&mBl16, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, B1, Kpad, L.N, Kpad * 4, kbe, L.N,
                               CU_TENSOR_MAP_SWIZZLE_64B);
    if (!ok16) return fail(SLSO_ERR_CUDA, "cuTensorMapEncodeTiled rejected a score operand layout");
    // row tiles per work item: B's hi and lo parts are read once per 256 rows (measured on 1M x 1024:
    // 2 tiles 1.27 ms, 4 tiles 1.29 ms: shared-memory bandwidth, not L2 ingress, bounds the kernel)
    constexpr int kT = 2;
    Layout2T L2{};
    L2.N = L.N;
    L2.KB = static_cast<int>(Kpad / kbe);
    L2.b_bytes = static_cast<uint32_t>(L.N) * kbe * 4u;
    L2.stage_bytes = 2 * kT * (kBM * kbe * 4u) + 2 * L2.b_bytes;
    L2.nbuf = (2 * kT * L.N <= 512) ? 2 : 1;
    L2.S = static_cast<int>(std::min<uint32_t>(kMaxStages2T, (226u * 1024u) / L2.stage_bytes));
    L2.bar_off = static_cast<uint32_t>(L2.S) * L2.stage_bytes;
    L2.smem_bytes = L2.bar_off + (3 * kMaxStages2T + 4) * 8 + 8 + 1024;
    uint32_t cols = 32;
    while (cols < static_cast<uint32_t>(L2.nbuf * kT * L.N)) cols <<= 1;
    L2.tmem_cols = cols;
    const int nwork = (ntiles + kT - 1) / kT;
    const int grid2 = std::min(nwork, h.num_sms);
    SLSO_TRY(raise_smem_limit(score_tc2_kernel<kbe, kT>, L2.smem_bytes));
    score_tc2_kernel<kbe, kT><<<grid2, kThreads, L2.smem_bytes, st>>>(mX16, mBh16, mBl16, L2, n, nwork, scores,
                                                                     h.state);
    SLSO_CHECK_LAUNCH();
    return SLSO_OK;
  }
  const int grid = std::min(ntiles, h.num_sms);
  SLSO_TRY(raise_smem_limit(score_tc_kernel, L.smem_bytes));
  score_tc_kernel<<<grid, kThreads, L.smem_bytes, st>>>(mX, mB0, mB1, mB2, L, n, ntiles, 1, cscale,
                                                        fp8 ? escale + 1 : nullptr, scores, nullptr, 0, 0,
                                                        h.state);
  SLSO_CHECK_LAUNCH();
  return SLSO_OK;
}


// Y = X M written to U (float32, n x ucols, row stride ldu) on the tensor cores, for M d x kk
// (row-major float64) with kk columns taken in blocks of 256: float32 X as 3xTF32, bfloat16 X
// as BF16X3 (both float32-accurate).  *used = false when the shapes need the SIMT kernel.
slso_status run_product_tc(Handle& h, Arena& ar, const void* X, int64_t n, int64_t d, int64_t ldx, int32_t xdt,
                           const double* M, int64_t kk, float* U, int64_t ldu, bool* used, cudaStream_t st) {
  *used = false;
  const int mode = (xdt == SLSO_F32) ? MODE_TF32X3 : (xdt == SLSO_BF16 ? MODE_BF16X3 : -1);
  if (mode < 0 || kk < 1) return SLSO_OK;
  const size_t esz = dtype_size(xdt);
  if (reinterpret_cast<uintptr_t>(X) % 16 != 0 || (ldx * esz) % 16 != 0) return SLSO_OK;
  if (!encode_fn()) return SLSO_OK;
  const Layout L = make_layout(mode, std::min<int64_t>(kk, 256), d);
  const int ncb = static_cast<int>(ceil_div(kk, L.N));
  const int64_t NB = static_cast<int64_t>(ncb) * L.N;  // rows of B = M^T, zero beyond kk
  const int64_t Kpad = static_cast<int64_t>(L.KB) * L.kbe;
  void* B0 = nullptr;
  void* B1 = nullptr;
  void* B2 = nullptr;
  if (mode == MODE_TF32X3) {
    B0 = ar.take<float>(static_cast<size_t>(NB) * Kpad);
    B1 = ar.take<float>(static_cast<size_t>(NB) * Kpad);
  } else {
    B0 = ar.take<__nv_bfloat16>(static_cast<size_t>(NB) * Kpad);
    B1 = ar.take<__nv_bfloat16>(static_cast<size_t>(NB) * Kpad);
    B2 = ar.take<__nv_bfloat16>(static_cast<size_t>(NB) * Kpad);
  }
  *used = true;
  if (ar.measure()) return SLSO_OK;
  const int pg = static_cast<int>(std::max<int64_t>(1, std::min<int64_t>(ceil_div(NB * Kpad, 256), 4LL * h.num_sms)));
  CUtensorMap mX, mB0, mB1, mB2;
  const CUtensorMapDataType xdt_map = (xdt == SLSO_F32) ? CU_TENSOR_MAP_DATA_TYPE_FLOAT32 : CU_TENSOR_MAP_DATA_TYPE_BFLOAT16;
  bool ok = make_map(&mX, xdt_map, X, d, n, ldx * esz, static_cast<uint32_t>(L.box_cols), kBM);
  if (mode == MODE_TF32X3) {
    prep_b_tf32_kernel<<<pg, 256, 0, st>>>(M, d, kk, NB, Kpad, static_cast<float*>(B0), static_cast<float*>(B1));
    SLSO_CHECK_LAUNCH();
    ok = ok && make_map(&mB0, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, B0, Kpad, NB, Kpad * 4, 32, L.N) &&
         make_map(&mB1, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, B1, Kpad, NB, Kpad * 4, 32, L.N);
    mB2 = mB1;
  } else {
    prep_b_bf16x3_kernel<<<pg, 256, 0, st>>>(M, d, kk, NB, Kpad, static_cast<__nv_bfloat16*>(B0),
                                             static_cast<__nv_bfloat16*>(B1), static_cast<__nv_bfloat16*>(B2));
    SLSO_CHECK_LAUNCH();
    ok = ok && make_map(&mB0, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, B0, Kpad, NB, Kpad * 2, 64, L.N) &&
         make_map(&mB1, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, B1, Kpad, NB, Kpad * 2, 64, L.N) &&
         make_map(&mB2, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, B2, Kpad, NB, Kpad * 2, 64, L.N);
  }
  if (!ok) return fail(SLSO_ERR_CUDA, "cuTensorMapEncodeTiled rejected a product operand layout");
  const int ntiles = static_cast<int>(ceil_div(n, kBM));
  const int grid = static_cast<int>(std::min<int64_t>(static_cast<int64_t>(ntiles) * ncb, h.num_sms));
  SLSO_TRY(raise_smem_limit(score_tc_kernel, L.smem_bytes));
  score_tc_kernel<<<grid, kThreads, L.smem_bytes, st>>>(mX, mB0, mB1, mB2, L, n, ntiles, ncb, nullptr, nullptr,
                                                        nullptr, U, ldu, kk, h.state);
  SLSO_CHECK_LAUNCH();
  return SLSO_OK;
}


bool score_group_eligible(const Handle& h, const void* X, int64_t d, int64_t ldx, int32_t xdt, int64_t k,
                          int32_t compute, double correct_frac) {
  return xdt == SLSO_F32 && compute == SLSO_F32 && k >= 1 && k <= 128 && d >= 1 && d <= 2048 &&
         correct_frac == 0.0 && h.score_form == SLSO_SCORE_FORM_MIXED && X != nullptr &&
         reinterpret_cast<uintptr_t>(X) % 16 == 0 && (ldx * 4) % 16 == 0 && encode_fn() != nullptr;
}

slso_status score_group_launch(Handle& h, ScoreGroupJob* host, ScoreGroupJob* dev, int njobs, cudaStream_t st) {
  if (njobs < 1 || njobs > kMaxScoreGroup) return fail(SLSO_ERR_INVALID_ARG, "grouped scores: %d jobs", njobs);
  const int N = host[0].N;
  const bool hyb = host[0].hyb != 0;
  int total = 0;
  for (int j = 0; j < njobs; ++j) {
    if (host[j].N != N || (host[j].hyb != 0) != hyb)
      return fail(SLSO_ERR_INVALID_ARG, "grouped scores need one JL width and one form");
    const int items = host[j].work0;  // run_scores_tc left the job's work items there
    host[j].work0 = total;
    total += items;
  }
  if (total == 0) return SLSO_OK;
  // the same layout as the one-job two-tile launch (it depends on N and the form only)
  LayoutTm T{};
  T.N = N;
  T.KB = 0;  // per job
  T.chunk = 0;
  T.nchunk = 1;
  tm_stages(T, 2);
  SLSO_CHECK_CUDA(cudaMemcpyAsync(dev, host, sizeof(ScoreGroupJob) * njobs, cudaMemcpyHostToDevice, st));
  const int grid = std::min(total, h.num_sms);
  auto launch = [&](auto kern) -> slso_status {
    SLSO_TRY(raise_smem_limit(kern, T.smem_bytes));
    kern<<<grid, kThreads, T.smem_bytes, st>>>(host[0].tmX, host[0].tmBh, T, 0, total, nullptr, host[0].state,
                                                dev, njobs);
    SLSO_CHECK_LAUNCH();
    return SLSO_OK;
  };
  return hyb ? launch(score_tm_kernel<true, 2, true>) : launch(score_tm_kernel<false, 2, true>);
}

}  // namespace slso
