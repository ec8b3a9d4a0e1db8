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
// All accumulation is float32 in TMEM.  Every mbarrier wait is bounded; a timeout sets an error
// word that the host reports as SLSO_ERR_TIMEOUT.
#include <cuda.h>
#include <cudaTypedefs.h>

#include <algorithm>

#include "common.cuh"
#include "tc.cuh"

namespace slso {

namespace {

using namespace tc;

enum Mode : int { MODE_TF32X3 = 0, MODE_BF16_CVT = 1, MODE_BF16 = 2 };

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
                    const __grid_constant__ CUtensorMap tmB1, const Layout L, int64_t n, int ntiles,
                    float* __restrict__ scores, DevState* __restrict__ state) {
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
  const bool convert = L.mode != MODE_BF16;

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
      for (int tile = blockIdx.x; tile < ntiles && ok; tile += gridDim.x) {
        const int y = tile * kBM;
        for (int kb = 0; kb < L.KB; ++kb, ++it) {
          const int os = it % L.OS;
          const uint32_t oph = (it / L.OS) & 1u;
          if (!mbar_wait(&op_empty[os], oph ^ 1u, abort_flag)) { ok = false; break; }
          unsigned char* op = smem + L.op_off + os * L.op_bytes;
          const int x = kb * L.kbe;
          if (L.mode == MODE_BF16) {
            mbar_arrive_expect_tx(&op_full[os], kXTileBytes + L.b_bytes);
            tma_load_2d(op, &tmX, &op_full[os], x, y);
            tma_load_2d(op + kXTileBytes, &tmB0, &op_full[os], x, 0);
            continue;
          }
          const int rs = it % L.RS;
          const uint32_t rph = (it / L.RS) & 1u;
          if (!mbar_wait(&raw_empty[rs], rph ^ 1u, abort_flag)) { ok = false; break; }
          unsigned char* raw = smem + L.raw_off + rs * L.raw_bytes;
          if (L.mode == MODE_TF32X3) {
            mbar_arrive_expect_tx(&op_full[os], 2 * L.b_bytes);
            tma_load_2d(op + 2 * kXTileBytes, &tmB0, &op_full[os], x, 0);
            tma_load_2d(op + 2 * kXTileBytes + L.b_bytes, &tmB1, &op_full[os], x, 0);
            mbar_arrive_expect_tx(&raw_full[rs], kXTileBytes);
            tma_load_2d(raw, &tmX, &raw_full[rs], x, y);
          } else {  // bfloat16 operands from float32 X: two 32-column float32 boxes per K-block
            mbar_arrive_expect_tx(&op_full[os], L.b_bytes);
            tma_load_2d(op + kXTileBytes, &tmB0, &op_full[os], x, 0);
            mbar_arrive_expect_tx(&raw_full[rs], 2 * kXTileBytes);
            tma_load_2d(raw, &tmX, &raw_full[rs], x, y);
            tma_load_2d(raw + kXTileBytes, &tmX, &raw_full[rs], x + 32, y);
          }
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
      const uint32_t id = (L.mode == MODE_TF32X3) ? idesc(FMT_TF32, FMT_TF32, kBM, L.N)
                                                  : idesc(FMT_BF16, FMT_BF16, kBM, L.N);
      int it = 0, tcount = 0;
      bool ok = true;
      for (int tile = blockIdx.x; tile < ntiles && ok; tile += gridDim.x, ++tcount) {
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
          } else {
            const uint64_t a = sdesc_sw128(op), b = sdesc_sw128(op + kXTileBytes);
#pragma unroll
            for (int ks = 0; ks < 4; ++ks) {
              const uint64_t o = static_cast<uint64_t>(ks * 2);
              mma_f16(d_tmem, a + o, b + o, id, (kb | ks) != 0);
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
      for (int tile = blockIdx.x; tile < ntiles && ok; tile += gridDim.x) {
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
    int tcount = 0;
    bool ok = true;
    for (int tile = blockIdx.x; tile < ntiles; tile += gridDim.x, ++tcount) {
      const int ab = tcount & 1;
      const uint32_t aph = (tcount >> 1) & 1u;
      int got = 0;
      if (lane == 0) got = mbar_wait(&acc_full[ab], aph, abort_flag) ? 1 : 0;
      got = __shfl_sync(0xFFFFFFFFu, got, 0);  // warp-uniform: tcgen05.ld is .sync.aligned
      if (!got) { ok = false; break; }
      tc_fence_after();
      const uint32_t taddr = tmem_base + (static_cast<uint32_t>(warp * 32) << 16) + static_cast<uint32_t>(ab * L.N);
      float sum = 0.0f;
      for (int c0 = 0; c0 < L.N; c0 += 32) {
        float v[32];
        tmem_ld_32x32b_x32(taddr + static_cast<uint32_t>(c0), v);
#pragma unroll
        for (int i = 0; i < 32; ++i) sum = fmaf(v[i], v[i], sum);
      }
      tc_fence_before();
      mbar_arrive(&acc_empty[ab]);
      const int64_t row = static_cast<int64_t>(tile) * kBM + warp * 32 + lane;
      if (row < n) scores[row] = sum;
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

using EncodeTiled = PFN_cuTensorMapEncodeTiled_v12000;

EncodeTiled encode_fn() {
  static EncodeTiled fn = nullptr;
  if (!fn) {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<EncodeTiled>(p);
  }
  return fn;
}

// Row-major (outer x inner) matrix with row pitch `pitch_bytes`, 128B swizzle, zero fill outside.
bool make_map(CUtensorMap* m, CUtensorMapDataType dt, const void* base, uint64_t inner, uint64_t outer,
              uint64_t pitch_bytes, uint32_t box_inner, uint32_t box_outer) {
  EncodeTiled fn = encode_fn();
  if (!fn) return false;
  cuuint64_t dims[2] = {inner, outer};
  cuuint64_t strides[1] = {pitch_bytes};
  cuuint32_t box[2] = {box_inner, box_outer};
  cuuint32_t es[2] = {1, 1};
  return fn(m, dt, 2, const_cast<void*>(base), dims, strides, box, es, CU_TENSOR_MAP_INTERLEAVE_NONE,
            CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
            CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

Layout make_layout(int mode, int64_t kk, int64_t d) {
  Layout L{};
  L.mode = mode;
  L.N = static_cast<int>(ceil_div(kk, 32) * 32);  // whole 32-column TMEM loads in the epilogue
  L.kbe = (mode == MODE_TF32X3) ? 32 : 64;
  L.KB = static_cast<int>(ceil_div(d, L.kbe));
  L.b_bytes = static_cast<uint32_t>(L.N) * 128u;
  const uint32_t budget = 226u * 1024u;  // + 1.5 KB barriers and alignment slack <= 227 KB
  if (mode == MODE_TF32X3) {
    L.raw_bytes = kXTileBytes;
    L.op_bytes = 2 * kXTileBytes + 2 * L.b_bytes;
    L.OS = static_cast<int>(std::max<uint32_t>(2, std::min<uint32_t>(3, (budget - 2 * L.raw_bytes) / L.op_bytes)));
    L.RS = static_cast<int>(std::min<uint32_t>(4, (budget - L.OS * L.op_bytes) / L.raw_bytes));
  } else if (mode == MODE_BF16_CVT) {
    L.raw_bytes = 2 * kXTileBytes;
    L.op_bytes = kXTileBytes + L.b_bytes;
    L.OS = static_cast<int>(std::min<uint32_t>(4, budget / 2 / L.op_bytes));
    L.RS = static_cast<int>(std::min<uint32_t>(4, (budget - L.OS * L.op_bytes) / L.raw_bytes));
  } else {
    L.raw_bytes = 0;
    L.op_bytes = kXTileBytes + L.b_bytes;
    L.OS = static_cast<int>(std::min<uint32_t>(kMaxStages, budget / L.op_bytes));
    L.RS = 1;
  }
  L.raw_off = 0;
  L.op_off = L.raw_bytes * static_cast<uint32_t>(mode == MODE_BF16 ? 0 : L.RS);
  L.bar_off = L.op_off + L.op_bytes * static_cast<uint32_t>(L.OS);
  L.smem_bytes = L.bar_off + 64 * 8 + 1024;  // barriers + TMEM slot + alignment slack
  uint32_t cols = 32;
  while (cols < static_cast<uint32_t>(2 * L.N)) cols <<= 1;
  L.tmem_cols = cols;
  return L;
}

}  // namespace

// Scores on the tensor cores when the shapes allow it; *used = false means the caller must
// take the SIMT kernel instead (k > 256, unaligned X, or an unsupported dtype pair).
slso_status run_scores_tc(Handle& h, Arena& ar, const void* X, int64_t n, int64_t d, int64_t ldx, int32_t xdt,
                          const double* M, int64_t kk, int32_t compute, float* scores, bool* used,
                          cudaStream_t st) {
  *used = false;
  int mode = -1;
  if (xdt == SLSO_F32 && compute == SLSO_F32) mode = MODE_TF32X3;
  if (xdt == SLSO_F32 && compute == SLSO_BF16) mode = MODE_BF16_CVT;
  if (xdt == SLSO_BF16 && compute == SLSO_BF16) mode = MODE_BF16;
  if (mode < 0 || kk > 256 || kk < 1) return SLSO_OK;
  const size_t esz = dtype_size(xdt);
  if (reinterpret_cast<uintptr_t>(X) % 16 != 0 || (ldx * esz) % 16 != 0) return SLSO_OK;
  if (!encode_fn()) return SLSO_OK;
  const Layout L = make_layout(mode, kk, d);
  const int64_t Kpad = static_cast<int64_t>(L.KB) * L.kbe;
  void* B0 = nullptr;
  void* B1 = nullptr;
  if (mode == MODE_TF32X3) {
    B0 = ar.take<float>(static_cast<size_t>(L.N) * Kpad);
    B1 = ar.take<float>(static_cast<size_t>(L.N) * Kpad);
  } else {
    B0 = ar.take<__nv_bfloat16>(static_cast<size_t>(L.N) * Kpad);
  }
  *used = true;
  if (ar.measure()) return SLSO_OK;
  const int pg = static_cast<int>(std::max<int64_t>(1, std::min<int64_t>(ceil_div(L.N * Kpad, 256), 4LL * h.num_sms)));
  CUtensorMap mX, mB0, mB1;
  bool ok;
  if (mode == MODE_TF32X3) {
    prep_b_tf32_kernel<<<pg, 256, 0, st>>>(M, d, kk, L.N, Kpad, static_cast<float*>(B0), static_cast<float*>(B1));
    SLSO_CHECK_LAUNCH();
    ok = make_map(&mX, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, X, d, n, ldx * 4, 32, kBM) &&
         make_map(&mB0, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, B0, Kpad, L.N, Kpad * 4, 32, L.N) &&
         make_map(&mB1, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, B1, Kpad, L.N, Kpad * 4, 32, L.N);
  } else {
    prep_b_bf16_kernel<<<pg, 256, 0, st>>>(M, d, kk, L.N, Kpad, static_cast<__nv_bfloat16*>(B0));
    SLSO_CHECK_LAUNCH();
    if (mode == MODE_BF16_CVT)
      ok = make_map(&mX, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, X, d, n, ldx * 4, 32, kBM);
    else
      ok = make_map(&mX, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, X, d, n, ldx * 2, 64, kBM);
    ok = ok && make_map(&mB0, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, B0, Kpad, L.N, Kpad * 2, 64, L.N);
    mB1 = mB0;
  }
  if (!ok) return fail(SLSO_ERR_CUDA, "cuTensorMapEncodeTiled rejected a score operand layout");
  const int ntiles = static_cast<int>(ceil_div(n, kBM));
  const int grid = std::min(ntiles, h.num_sms);
  SLSO_CHECK_CUDA(cudaFuncSetAttribute(score_tc_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       static_cast<int>(L.smem_bytes)));
  score_tc_kernel<<<grid, kThreads, L.smem_bytes, st>>>(mX, mB0, mB1, L, n, ntiles, scores, h.state);
  SLSO_CHECK_LAUNCH();
  return SLSO_OK;
}

}  // namespace slso
