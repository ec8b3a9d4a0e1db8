// Tensor-core Gram matrix G = SX^T SX for the Gram route of R (Algorithm 2/3 step 2), float64-class
// accurate, on the bfloat16 tcgen05 path with exact integer accumulation (an Ozaki-type split).
//
// Column j of SX is scaled by 2^-e_j (its largest entry in [1/2, 1)) and rounded to 55 fractional
// bits, a' = F 2^-55 with |F| < 2^55 (within 2^-56 of the column's maximum).  F is cut into eight
// signed 7-bit digits, F = sum_p d_p 2^(49 - 7p), each rounded to nearest from the remainder, so
// that |d_p| <= 64 and bfloat16 holds every digit exactly.  Slice p stores E_p = d_p 2^(21 - 7p)
// (exact), so for two columns
//   a'_i a'_j = sum_(p, q) d_p(i) d_q(j) 2^(-12 - 7(p + q)),
// and a product E_p E_q = d_p d_q 2^(42 - 7(p + q)) depends on the digit order t = p + q only.  The
// 36 pairs with t <= 7 are kept; the others lie near 2^-56 of the leading term.
//
// Exactness: a float32 accumulator holds a sum of products of one order t exactly while the
// integer sum S_t = sum d_p d_q stays within 2^24 in magnitude: every product is a multiple of
// 2^(42 - 7t) and every partial sum is then representable, whatever the order of the additions
// inside the tensor core (measured bit-exact).  With |d_p d_q| <= 2^12 and at most 8 pairs of one
// order, a window of 512 rows of SX keeps every order within 2^24 (8 x 512 x 2^12), so each order
// has its own accumulator and nothing is rounded: also orders 3..7 matter when rows are
// heavy-tailed (a row far below its columns' maxima has small leading digits, and then its middle
// digits dominate).  After every window the epilogue warps read the eight accumulators from TMEM
// and add their exact integers to two int64 running sums per entry,
//   T_hi = sum 2^21 S_0 + 2^14 S_1 + 2^7 S_2 + S_3,   T_lo = sum 2^21 S_4 + 2^14 S_5 + 2^7 S_6 + S_7
// (each below 2^53 for s <= 2^20), and G_ij = 2^(e_i + e_j - 33) (T_hi + 2^-28 T_lo), rounded once
// per entry.  Integer sums are exact in any order, so G does not depend on how the rows are split.
//
// gram_tc_kernel: one 128 x 64 tile of the lower triangle of G over a range of rows of SX per CTA
// (576 threads, one CTA per SM):
//   warps 0-15 epilogue: warp w reads TMEM lanes 32 (w % 4).. (tile rows) and columns
//              16 (w / 4).. of each accumulator; two int64 running sums per entry in registers.
//   warp 16    TMA producer: per stage the eight A slices (128 columns of SX x 16 rows) and eight B
//              slices (64 columns x 16 rows) in four 128B-swizzled boxes (slices 0-3 and 4-7 of A
//              and of B, each row 128 bytes = 4 slices x 16 values); four stages of 48 KB.
//   warp 17    TMEM owner (eight 64-column accumulators) and MMA issuer: 36 tcgen05.mma
//              (kind::f16, bfloat16, M = 128, N = 64, K = 16) per stage.
// Every mbarrier wait is bounded; a timeout sets DevState::timeout.
#include <cuda_bf16.h>

#include <algorithm>
#include <cmath>

#include "common.cuh"
#include "tc.cuh"
#include "tmap.cuh"

namespace slso {

namespace {

using namespace tc;

constexpr int kThreadsG = 576;
constexpr int kBMg = 128;   // tile rows (columns i of SX)
constexpr int kBNg = 64;    // tile columns (columns j of SX)
constexpr int kKBg = 16;    // rows of SX per stage: one 32-byte bfloat16 row per slice tile
constexpr int kSlices = 8;  // 7-bit digits of the 56-bit fixed-point value
constexpr int kOrders = 8;  // accumulators: one per digit order 0..7
constexpr int kWinRows = 512;  // rows of SX per exact window
constexpr int kKbPerWin = kWinRows / kKBg;
constexpr int kStagesG = 4;  // four stages of 48 KB: more of the L2 ingress in flight than two of 96 KB
constexpr int kEpiWarpsG = 16;
constexpr int kWarpProdG = 16, kWarpMmaG = 17;
constexpr uint32_t kASliceBytes = kBMg * kKBg * 2;  // 4 KB: one slice of the A tile
constexpr uint32_t kBSliceBytes = kBNg * kKBg * 2;  // 2 KB
constexpr uint32_t kAGroupBytes = 4 * kASliceBytes;  // four slices' K-block rows of 128 bytes (16 KB)
constexpr uint32_t kBGroupBytes = 4 * kBSliceBytes;  // 8 KB
constexpr uint32_t kStageBytesG = kSlices * (kASliceBytes + kBSliceBytes);
constexpr uint32_t kBarOffG = kStagesG * kStageBytesG;
constexpr uint32_t kSmemG = kBarOffG + (2 * kStagesG + 2) * 8 + 16 + 1024;
constexpr uint32_t kTmemColsG = kOrders * kBNg;  // 512
constexpr int kPairs = 36;
constexpr int kTimeoutIdG = 6;
constexpr int kSplitBalanceSms = 152;  // GB300's SM count: fixed, so the plan does not depend on the device
constexpr int64_t kMaxRowsTc = int64_t(1) << 20;  // keeps |T_hi|, |T_lo| < 2^53

// The digit pairs (p, q), p + q <= 7, by order t = p + q: pair index pr = t (t + 1) / 2 + p; the
// first pair of each order starts its accumulator.  Compile-time functions of the (unrolled) pair
// index, so that the MMA issuer spends no instructions on them.
__host__ __device__ constexpr int pair_order(int pr) {
  int t = 0;
  while ((t + 1) * (t + 2) / 2 <= pr) ++t;
  return t;
}
__host__ __device__ constexpr int pair_p(int pr) { return pr - pair_order(pr) * (pair_order(pr) + 1) / 2; }
static_assert(pair_order(35) == 7 && pair_p(35) == 7 && pair_p(6) == 0 && pair_order(6) == 3, "pair table");

// rint(a 2^(55 - e)) for |a| < 2^e, from a's bits (integer operations only: the float64 pipe is
// narrow on this part).  Round half away from zero; non-finite a sets bad.
__device__ __forceinline__ long long fixed55(double a, int e, bool& bad) {
  const unsigned long long u = static_cast<unsigned long long>(__double_as_longlong(a));
  const int ex = static_cast<int>((u >> 52) & 0x7FFu);
  if (ex == 0x7FF) {
    bad = true;
    return 0;
  }
  long long m = static_cast<long long>(u & ((1ull << 52) - 1));
  int E;  // |a| = m 2^E
  if (ex == 0) {
    E = 1 - 1075;
  } else {
    m |= 1ll << 52;
    E = ex - 1075;
  }
  const int sh = E + 55 - e;
  long long F;
  if (sh >= 0) {
    F = m * (1ll << sh);  // |F| < 2^55 by the choice of e
  } else {
    const int rs = -sh;
    F = rs >= 60 ? 0 : ((m + (1ll << (rs - 1))) >> rs);
  }
  return (u >> 63) ? -F : F;
}

// Slices E_p (p < 8) of the scaled SX, transposed and interleaved: column j of SX is row j of a
// dpad x (8 sp) bfloat16 matrix (rows j >= d are zero) that holds, for each K-block of 16 rows of
// SX, the 16 values of slice 0, then of slice 1, ..., slice 7 (256 bytes); sp, the padded number of
// rows of SX, is a multiple of 64.  A 128-byte TMA box then carries four slices of one K-block.
// Block (x: row block, y: column block): 64 rows x 32 columns of SX; threads (32, 8): a warp reads
// 32 consecutive float64 of a row, each thread 8 rows (loads issued first); the block writes each
// column's 1 KB run (4 K-blocks x 8 slices x 16) with a warp on 128 consecutive bytes.
constexpr int kSliceRows = 64;
__global__ void __launch_bounds__(256) gram_slice_kernel(const double* __restrict__ SX, int64_t s, int d, int dpad,
                                                         int64_t sp, const int* __restrict__ cexp,
                                                         __nv_bfloat16* __restrict__ E, int* __restrict__ bad_flag) {
  // [p][column][row], rows of 66 values; slice p at p kPStride, so that the warps' reads of four
  // slices' runs fall on different banks (kPStride is 8 words past a multiple of 32 words)
  constexpr int kRowS = kSliceRows + 2, kPStride = 32 * kRowS + 16;
  __shared__ __align__(16) __nv_bfloat16 tile[kSlices * kPStride];
  const int j0 = blockIdx.y * 32;
  const int64_t i0 = static_cast<int64_t>(blockIdx.x) * kSliceRows;
  const int tx = threadIdx.x, ty = threadIdx.y;
  bool bad = false;
  const int j = j0 + tx;
  const int e = j < d ? cexp[j] : 0;
  constexpr int kPer = kSliceRows / 8;
  double xv[kPer];
#pragma unroll
  for (int k = 0; k < kPer; ++k) {
    const int64_t i = i0 + ty + 8 * k;
    xv[k] = (j < d && i < s) ? SX[i * d + j] : 0.0;
  }
#pragma unroll
  for (int k = 0; k < kPer; ++k) {
    const int rr = ty + 8 * k;
    const int64_t i = i0 + rr;
    long long F = 0;
    if (j < d && i < s) F = fixed55(xv[k], e, bad);
    // balanced base-128 digits of F = sum_p d_p 2^(49 - 7p), d_7..d_1 in [-64, 63], |d_0| <= 64,
    // from the bottom in 32-bit arithmetic: the low 28 bits give d_7..d_4 and a carry into the
    // high part, which gives d_3..d_0
    int dg[kSlices];
    int x = static_cast<int>(static_cast<unsigned int>(F) & 0x0FFFFFFFu);
#pragma unroll
    for (int p = kSlices - 1; p >= 4; --p) {
      dg[p] = ((x + 64) & 127) - 64;
      x = (x - dg[p]) >> 7;  // exact division; the carry out of the last step is 0 or 1
    }
    int y = static_cast<int>(F >> 28) + x;  // |y| < 2^27 + 1
#pragma unroll
    for (int p = 3; p >= 1; --p) {
      dg[p] = ((y + 64) & 127) - 64;
      y = (y - dg[p]) >> 7;
    }
    dg[0] = y;  // |F| < 2^55 keeps it within [-64, 64]
#pragma unroll
    for (int p = 0; p < kSlices; ++p) {
      // E_p = d_p 2^(21 - 7p), exact in float32 and in bfloat16 (|d_p| <= 64), without conversion
      // instructions: the float with the bits of 2^23 + 2^22 + d_p is exactly 1.5 2^23 + d_p, one
      // FMA with the power of two takes 1.5 2^23 back off exactly, and the product's low 16 bits
      // are zero (at most 7 significant bits), so its upper half is the bfloat16
      const float scale = __int_as_float((127 + 21 - 7 * p) << 23);  // 2^(21 - 7p)
      const float v = fmaf(__int_as_float(0x4B400000 + dg[p]), scale, -12582912.0f * scale);
      tile[p * kPStride + tx * kRowS + rr] = __ushort_as_bfloat16(static_cast<unsigned short>(__float_as_uint(v) >> 16));
    }
  }
  __syncthreads();
  // column j0 + cc: 512 values from E[(j0 + cc) 8 sp + 8 i0]; value o is slice (o / 16) % 8 of row
  // 16 (o / 128) + o % 16 of the block
  for (int cc = ty; cc < 32; cc += 8) {
    __nv_bfloat16* out = E + static_cast<int64_t>(j0 + cc) * 8 * sp + 8 * i0;
#pragma unroll
    for (int m = 0; m < 8; ++m) {
      const int o = 2 * (tx + 32 * m);
      const int p = (o >> 4) & 7, r = ((o >> 7) << 4) + (o & 15);
      *reinterpret_cast<__nv_bfloat162*>(out + o) =
          *reinterpret_cast<const __nv_bfloat162*>(&tile[p * kPStride + cc * kRowS + r]);
    }
  }
  if (__syncthreads_or(bad) && tx == 0 && ty == 0) atomicOr(bad_flag, 1);
}

// t-th tile (I, J) of the 128 x 64 tiling of G's lower triangle: row blocks I of 128, then the
// column blocks J < min(2I + 2, nbJ) that reach the diagonal.
__device__ __forceinline__ void tc_tile(int t, int nbJ, int& I, int& J) {
  int i = 0;
  while (true) {
    const int cnt = min(2 * i + 2, nbJ);
    if (t < cnt) break;
    t -= cnt;
    ++i;
  }
  I = i;
  J = t;
}

__device__ __forceinline__ void tmem_ld_x16(uint32_t taddr, uint32_t* r) {
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 "
      "{%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
        "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
      : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
}

// CTA = (split q, tile t): blockIdx.x = q tiles + t.  Rows [q kc, min((q + 1) kc, s)) of SX in
// windows of 256.  part[blockIdx.x][128][64][2]: the int64 sums (T_hi, T_lo) of the tile over those rows.
__global__ void __launch_bounds__(kThreadsG, 1)
    gram_tc_kernel(const __grid_constant__ CUtensorMap tmA, const __grid_constant__ CUtensorMap tmB, int64_t s,
                   int dpad, int tiles, int nbJ, int64_t kc, long long* __restrict__ part,
                   DevState* __restrict__ state) {
  extern __shared__ unsigned char smem_dyn[];
  unsigned char* smem = reinterpret_cast<unsigned char*>((reinterpret_cast<uintptr_t>(smem_dyn) + 1023) &
                                                         ~static_cast<uintptr_t>(1023));
  uint64_t* full = reinterpret_cast<uint64_t*>(smem + kBarOffG);  // TMA bytes of the stage landed
  uint64_t* empty = full + kStagesG;                               // the MMAs reading it completed
  uint64_t* acc_full = empty + kStagesG;                           // the window is accumulated
  uint64_t* acc_empty = acc_full + 1;                              // the epilogue has read it
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(acc_empty + 1);
  __shared__ int s_abort;
  const volatile int* abort_flag = &s_abort;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int q = blockIdx.x / tiles, t = blockIdx.x % tiles;
  int I, J;
  tc_tile(t, nbJ, I, J);
  const int64_t r0 = static_cast<int64_t>(q) * kc;
  const int64_t r1 = r0 + kc < s ? r0 + kc : s;
  const int kb0 = static_cast<int>(r0 / kKBg);
  const int nkb = r1 > r0 ? static_cast<int>((r1 - r0 + kKBg - 1) / kKBg) : 0;
  const int nwin = (nkb + kKbPerWin - 1) / kKbPerWin;

  if (threadIdx.x == 0) {
    s_abort = 0;
    for (int i = 0; i < kStagesG; ++i) {
      mbar_init(&full[i], 1);
      mbar_init(&empty[i], 1);
    }
    mbar_init(acc_full, 1);
    mbar_init(acc_empty, kEpiWarpsG);
    fence_mbar_init();
  }
  if (warp == kWarpMmaG) tmem_alloc(tmem_slot, kTmemColsG);
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem_base = *tmem_slot;

  if (warp == kWarpProdG) {
    if (lane == 0) {
      int kb = 0;
      bool ok = true;
      for (; kb < nkb; ++kb) {
        const int st = kb % kStagesG;
        if (!mbar_wait(&empty[st], ((kb / kStagesG) & 1u) ^ 1u, abort_flag)) {
          ok = false;
          break;
        }
        unsigned char* stage = smem + static_cast<uint32_t>(st) * kStageBytesG;
        mbar_arrive_expect_tx(&full[st], kStageBytesG);
        const int x = (kb0 + kb) * kKBg * kSlices;  // the K-block's 128 values (8 slices x 16)
#pragma unroll
        for (int g = 0; g < 2; ++g) {  // slices 4g .. 4g + 3: one 128-byte box row per column
          tma_load_2d(stage + g * kAGroupBytes, &tmA, &full[st], x + 64 * g, I * kBMg);
          tma_load_2d(stage + 2 * kAGroupBytes + g * kBGroupBytes, &tmB, &full[st], x + 64 * g, J * kBNg);
        }
      }
      if (!ok) {
        atomicExch(&s_abort, 1);
        atomicExch(&state->timeout, kTimeoutIdG);
        for (int j = (kb > kStagesG ? kb - kStagesG : 0); j < kb; ++j)  // let issued copies land (bounded)
          mbar_wait(&full[j % kStagesG], (j / kStagesG) & 1u, nullptr, 50000000ull);
      }
    }
  } else if (warp == kWarpMmaG) {
    if (lane == 0) {
      const uint32_t id = idesc(FMT_BF16, FMT_BF16, kBMg, kBNg);
      int kb = 0;
      bool ok = true;
      for (int w = 0; w < nwin && ok; ++w) {
        if (!mbar_wait(acc_empty, (w & 1u) ^ 1u, abort_flag)) {
          ok = false;
          break;
        }
        tc_fence_after();
        const int kb_end = min(nkb, (w + 1) * kKbPerWin);
        for (int kw = 0; kb < kb_end; ++kb, ++kw) {
          const int st = kb % kStagesG;
          if (!mbar_wait(&full[st], (kb / kStagesG) & 1u, abort_flag)) {
            ok = false;
            break;
          }
          tc_fence_after();
          unsigned char* stage = smem + static_cast<uint32_t>(st) * kStageBytesG;
          // the slices' descriptors differ from the stage's first ones only in the start address
          // field (address >> 4, bits 0-13; every address here is below 2^18, so no carry): slice
          // p sits in group p / 4 at 32 (p % 4) bytes into each 128-byte row
          const uint64_t a0 = sdesc_sw128(stage), b0 = sdesc_sw128(stage + 2 * kAGroupBytes);
#pragma unroll
          for (int ks = 0; ks < kKBg / 16; ++ks) {
            const uint64_t o = static_cast<uint64_t>(ks * 2);  // 32 bytes along K
#pragma unroll
            for (int pr = 0; pr < kPairs; ++pr) {
              const int ord = pair_order(pr), p = pair_p(pr), qq = ord - p;
              // the first pair of each order starts its accumulator in the window's first K-step
              const bool first = p == 0;
              const uint32_t acc = (kw | ks) != 0 || !first;
              const uint64_t a = a0 + static_cast<uint64_t>((p >> 2) * (kAGroupBytes >> 4) + (p & 3) * 2) + o;
              const uint64_t bd = b0 + static_cast<uint64_t>((qq >> 2) * (kBGroupBytes >> 4) + (qq & 3) * 2) + o;
              mma_f16(tmem_base + static_cast<uint32_t>(ord * kBNg), a, bd, id, acc);
            }
          }
          mma_commit(&empty[st]);
        }
        if (ok) mma_commit(acc_full);
      }
      if (!ok) {
        atomicExch(&s_abort, 1);
        atomicExch(&state->timeout, kTimeoutIdG);
      }
      // every MMA issued by this thread has completed before TMEM is released
      if (kb > 0) mbar_wait(&empty[(kb - 1) % kStagesG], ((kb - 1) / kStagesG) & 1u, nullptr, 50000000ull);
    }
  } else {  // epilogue warps 0-15
    const int lg = warp & 3, cq = warp >> 2;
    const uint32_t lane_off = static_cast<uint32_t>(lg * 32) << 16;
    long long Th[16], Tl[16];
#pragma unroll
    for (int c = 0; c < 16; ++c) Th[c] = Tl[c] = 0;
    bool ok = true;
    for (int w = 0; w < nwin; ++w) {
      int got = 0;
      if (lane == 0) got = mbar_wait(acc_full, w & 1u, abort_flag) ? 1 : 0;
      got = __shfl_sync(0xFFFFFFFFu, got, 0);  // warp-uniform: tcgen05.ld is .sync.aligned
      if (!got) {
        ok = false;
        break;
      }
      tc_fence_after();
      const uint32_t taddr = tmem_base + lane_off + static_cast<uint32_t>(cq * 16);
      // accumulator t holds 2^(42 - 7t) S_t exactly, |S_t| <= 2^24
#pragma unroll
      for (int t = 0; t < kOrders; ++t) {
        uint32_t v[16];
        tmem_ld_x16(taddr + static_cast<uint32_t>(t * kBNg), v);
        const float unscale = __int_as_float((127 - 42 + 7 * t) << 23);  // 2^(7t - 42)
        const long long wgt = 1ll << (7 * (3 - (t & 3)));
#pragma unroll
        for (int c = 0; c < 16; ++c) {
          const long long S = __float2int_rn(__uint_as_float(v[c]) * unscale);
          if (t < 4) Th[c] += S * wgt;
          else Tl[c] += S * wgt;
        }
      }
      tc_fence_before();
      __syncwarp();
      if (lane == 0) mbar_arrive(acc_empty);
    }
    if (ok) {
      long long* dst = part + ((static_cast<int64_t>(blockIdx.x) * kBMg + lg * 32 + lane) * kBNg + cq * 16) * 2;
#pragma unroll
      for (int c = 0; c < 16; ++c) *reinterpret_cast<longlong2*>(dst + 2 * c) = make_longlong2(Th[c], Tl[c]);
    } else if (lane == 0) {
      atomicExch(&s_abort, 1);
      atomicExch(&state->timeout, kTimeoutIdG);
    }
  }

  tc_fence_before();
  __syncthreads();
  if (warp == kWarpMmaG) {
    tc_fence_after();
    tmem_dealloc(tmem_base, kTmemColsG);
  }
}

// L[i d + j] (j <= i) = 2^(e_i + e_j - 33) (T_hi + 2^-28 T_lo) with the sums over splits; a
// non-finite SX entry writes NaN on the diagonal, so that the Cholesky breaks down and the route
// closes.  Opens the route.
__global__ void gram_tc_reduce_kernel(const long long* __restrict__ part, int tiles, int splits, int d, int nbJ,
                                      const int* __restrict__ cexp, const int* __restrict__ bad_flag,
                                      double* __restrict__ L, DevState* __restrict__ st) {
  const int64_t total = static_cast<int64_t>(d) * d;
  const bool bad = *bad_flag != 0;
  for (int64_t e = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; e < total;
       e += static_cast<int64_t>(gridDim.x) * blockDim.x) {
    const int i = static_cast<int>(e / d), j = static_cast<int>(e % d);
    if (j > i) continue;
    const int I = i / kBMg, J = j / kBNg;
    int t = 0;
    for (int r = 0; r < I; ++r) t += min(2 * r + 2, nbJ);
    t += J;
    const int64_t off = (static_cast<int64_t>(i - I * kBMg) * kBNg + (j - J * kBNg)) * 2;
    long long Th = 0, Tl = 0;
    for (int qq = 0; qq < splits; ++qq) {
      const longlong2 v = *reinterpret_cast<const longlong2*>(part + (static_cast<int64_t>(qq) * tiles + t) *
                                                                          (kBMg * kBNg * 2) + off);
      Th += v.x;
      Tl += v.y;
    }
    double v = ldexp(static_cast<double>(Th) + ldexp(static_cast<double>(Tl), -28), cexp[i] + cexp[j] - 33);
    if (bad && i == j) v = nan("");
    L[e] = v;
  }
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    st->gram_ok = 1;
    st->gram_tried = 1;
    st->gram_resid = 0.0;
  }
}

}  // namespace

bool gram_tc_applies(int64_t s, int64_t d) { return encode_fn() != nullptr && s < kMaxRowsTc && d >= 1; }

void gram_tc_take(Arena& ar, int64_t s, int64_t d, GramTcWork* w) {
  w->dpad = static_cast<int>(ceil_div(d, kBMg) * kBMg);
  w->sp = ceil_div(s, kSliceRows) * kSliceRows;
  const int nbI = static_cast<int>(ceil_div(d, kBMg));
  w->nbJ = static_cast<int>(ceil_div(d, kBNg));
  int tiles = 0;
  for (int i = 0; i < nbI; ++i) tiles += std::min(2 * i + 2, w->nbJ);
  w->tiles = tiles;
  // splits: the smallest count (each split at least two windows) whose CTAs fill GB300's SMs within
  // 6% of even, else the most even one
  const int64_t wins = ceil_div(s, kWinRows);
  double best = 1e30;
  int best_s = 1;
  for (int S = 1; S <= 16 && S <= std::max<int64_t>(1, wins / 2); ++S) {
    const int64_t items = static_cast<int64_t>(tiles) * S;
    const double waste = static_cast<double>(ceil_div(items, kSplitBalanceSms) * kSplitBalanceSms) /
                         static_cast<double>(items);
    if (waste < 1.06) {
      best_s = S;
      break;
    }
    if (waste < best) {
      best = waste;
      best_s = S;
    }
  }
  w->splits = best_s;
  w->kc = ceil_div(ceil_div(s, best_s), kWinRows) * kWinRows;
  w->E = ar.take<__nv_bfloat16>(static_cast<size_t>(kSlices) * w->dpad * w->sp);
  w->part = ar.take<long long>(static_cast<size_t>(w->splits) * tiles * kBMg * kBNg * 2);
  w->bad = ar.take<int>(1);
}

slso_status run_gram_tc(Handle& h, const GramTcWork& w, const double* SX, int64_t s, int64_t d, const int* cexp,
                        double* L, cudaStream_t st) {
  const int d_i = static_cast<int>(d);
  SLSO_CHECK_CUDA(cudaMemsetAsync(w.bad, 0, sizeof(int), st));
  const dim3 gs(static_cast<unsigned>(w.sp / kSliceRows), static_cast<unsigned>(w.dpad / 32));
  gram_slice_kernel<<<gs, dim3(32, 8), 0, st>>>(SX, s, d_i, w.dpad, w.sp, cexp, w.E, w.bad);
  SLSO_CHECK_LAUNCH();
  CUtensorMap mA, mB;
  const uint64_t inner = static_cast<uint64_t>(kSlices) * w.sp;  // values per column of SX
  bool ok = make_map(&mA, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, w.E, inner, w.dpad, inner * 2, 64, kBMg,
                     CU_TENSOR_MAP_SWIZZLE_128B) &&
            make_map(&mB, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, w.E, inner, w.dpad, inner * 2, 64, kBNg,
                     CU_TENSOR_MAP_SWIZZLE_128B);
  if (!ok) return fail(SLSO_ERR_CUDA, "cuTensorMapEncodeTiled failed for the Gram slices");
  SLSO_TRY(raise_smem_limit(gram_tc_kernel, kSmemG));
  gram_tc_kernel<<<static_cast<unsigned>(w.tiles * w.splits), kThreadsG, kSmemG, st>>>(
      mA, mB, s, w.dpad, w.tiles, w.nbJ, w.kc, w.part, h.state);
  SLSO_CHECK_LAUNCH();
  const int64_t total = d * d;
  const unsigned rb = static_cast<unsigned>(std::min<int64_t>(ceil_div(total, 256), static_cast<int64_t>(h.num_sms) * 8));
  gram_tc_reduce_kernel<<<rb, 256, 0, st>>>(w.part, w.tiles, w.splits, d_i, w.nbJ, cexp, w.bad, L, h.state);
  SLSO_CHECK_LAUNCH();
  return SLSO_OK;
}

}  // namespace slso
