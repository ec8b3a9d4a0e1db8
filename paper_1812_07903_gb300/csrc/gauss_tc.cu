// Tensor-core Gaussian sketch SX = (1/sqrt(s)) G X (Sec. 2.1, Gaussian projection) on sm_103a.
//
// G (s x n, bfloat16-valued N(0,1) entries from Philox, four per block) is never formed whole.
// The rows of X are taken in chunks of Kc, and for each chunk:
//   gauss_gen_kernel   writes G[:, chunk] (s x Kc bfloat16, K contiguous), each entry once;
//   xt_split_kernel    writes X[chunk, :]^T (d x Kc bfloat16, K contiguous): one piece for
//                      bfloat16 X, three for float32 X (x = x1 + x2 + x3 exactly, each piece a
//                      bfloat16), and flags non-finite values of X;
//   gauss_tc_kernel    computes each 128 x NT tile of G[:, chunk] X[chunk, :] with tcgen05.mma
//                      (kind::f16; bfloat16 products are exact) and adds it, times 1/sqrt(s),
//                      into SX in float64.
// Accumulation: the tensor core's float32 accumulation loses up to ~2^-24 of the running sum per
// MMA step, with a consistent sign, so its error grows with the number of steps (measured ~1e-4
// relative over 32768 rows).  The K range of a chunk is therefore cut into sub-chunks of at most
// ~32 MMA steps, each accumulated from zero in one of two TMEM accumulators; the epilogue warps
// add each finished sub-chunk into float32 running sums held in registers (round-to-nearest
// adds, unbiased) while the MMAs fill the other accumulator, and only the chunk total goes to
// SX in float64.
// Chunks are added in order and every SX element belongs to one CTA per chunk, so the result is
// deterministic.  CTAs that share a row block of G are adjacent in launch order, so a G tile is
// fetched from HBM once and re-read from L2 by the other column tiles.
//
// gauss_tc_kernel<NT>, one 128 x NT output tile per CTA (320 threads):
//   warps 0-7  epilogue: warp w reads TMEM lanes 32(w%4).. (tile rows) and columns
//              (w/4)*NT/2 .. +NT/2 with tcgen05.ld 32x32b; thread = tile row.
//   warp 8     TMA producer: G tile (128 rows x 64 K) and P X^T tiles (NT rows x 64 K) per stage.
//   warp 9     TMEM owner (2*NT columns) and MMA issuer (one thread).
// Every mbarrier wait is bounded; a timeout sets DevState::timeout (SLSO_ERR_TIMEOUT).
#include <cuda_bf16.h>

#include <algorithm>
#include <cmath>

#include "common.cuh"
#include "tc.cuh"
#include "tmap.cuh"

namespace slso {

namespace {

using namespace tc;

constexpr int kGThreads = 320;
constexpr int kGBM = 128;        // tile rows (rows of SX = rows of G)
constexpr int kGKB = 64;         // K elements per stage (one 128-byte bfloat16 operand row)
constexpr int kGMaxStages = 6;
constexpr int kGEpiWarps = 8;
constexpr int kGWarpProducer = 8, kGWarpMma = 9;
constexpr uint32_t kATileBytes = kGBM * 128;
constexpr int64_t kChunkRows = 32768;  // rows of X per chunk (G chunk s*Kc*2 bytes)
constexpr int kStepsPerSub = 32;       // MMA steps accumulated in float32 by the tensor core

struct GLayout {
  int P;            // X pieces: 1 (bfloat16 X) or 3 (float32 X)
  int NT;           // tile columns = accumulator columns (power of two, 64..256)
  int KB;           // K-blocks per chunk
  int KBS;          // K-blocks per sub-chunk
  int S;            // pipeline stages
  uint32_t b_bytes, stage_bytes, bar_off, smem_bytes;
};

// 32 lanes x 16 columns of 32-bit accumulators (thread t of the warp gets lane base + t).
__device__ __forceinline__ void tmem_ld_32x32b_x16(uint32_t taddr, float* v) {
  uint32_t r[16];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 "
      "{%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
        "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
      : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
  for (int i = 0; i < 16; ++i) v[i] = __uint_as_float(r[i]);
}

template <int NT>
__global__ void __launch_bounds__(kGThreads, 1)
    gauss_tc_kernel(const __grid_constant__ CUtensorMap tmA, const __grid_constant__ CUtensorMap tmB0,
                    const __grid_constant__ CUtensorMap tmB1, const __grid_constant__ CUtensorMap tmB2,
                    const GLayout L, int64_t s, int64_t d, double scale, int first, double* __restrict__ SX,
                    DevState* __restrict__ state) {
  constexpr int CW = NT / 2;  // columns per epilogue warp
  extern __shared__ unsigned char smem_dyn[];
  unsigned char* smem = reinterpret_cast<unsigned char*>((reinterpret_cast<uintptr_t>(smem_dyn) + 1023) &
                                                         ~static_cast<uintptr_t>(1023));
  uint64_t* full = reinterpret_cast<uint64_t*>(smem + L.bar_off);  // TMA bytes of the stage landed
  uint64_t* empty = full + kGMaxStages;                             // the MMAs reading it completed
  uint64_t* acc_full = empty + kGMaxStages;                         // [2] sub-chunk accumulated
  uint64_t* acc_empty = acc_full + 2;                               // [2] epilogue folded it
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(acc_empty + 2);
  __shared__ int s_abort;
  const volatile int* abort_flag = &s_abort;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int n0 = blockIdx.x * NT, m0 = blockIdx.y * kGBM;
  const int nsub = (L.KB + L.KBS - 1) / L.KBS;

  if (threadIdx.x == 0) {
    s_abort = 0;
    for (int i = 0; i < L.S; ++i) {
      mbar_init(&full[i], 1);
      mbar_init(&empty[i], 1);
    }
    for (int i = 0; i < 2; ++i) {
      mbar_init(&acc_full[i], 1);
      mbar_init(&acc_empty[i], kGEpiWarps);
    }
    fence_mbar_init();
  }
  if (warp == kGWarpMma) tmem_alloc(tmem_slot, 2u * NT);
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem_base = *tmem_slot;

  if (warp == kGWarpProducer) {
    if (lane == 0) {
      int kb = 0;
      bool ok = true;
      for (; kb < L.KB; ++kb) {
        const int st = kb % L.S;
        const uint32_t ph = (kb / L.S) & 1u;
        if (!mbar_wait(&empty[st], ph ^ 1u, abort_flag)) {
          ok = false;
          break;
        }
        unsigned char* stage = smem + static_cast<uint32_t>(st) * L.stage_bytes;
        mbar_arrive_expect_tx(&full[st], L.stage_bytes);
        const int x = kb * kGKB;
        tma_load_2d(stage, &tmA, &full[st], x, m0);
        tma_load_2d(stage + kATileBytes, &tmB0, &full[st], x, n0);
        if (L.P == 3) {
          tma_load_2d(stage + kATileBytes + L.b_bytes, &tmB1, &full[st], x, n0);
          tma_load_2d(stage + kATileBytes + 2 * L.b_bytes, &tmB2, &full[st], x, n0);
        }
      }
      if (!ok) {
        atomicExch(&s_abort, 1);
        atomicExch(&state->timeout, 4);
        // let the copies already issued land before the CTA can exit (bounded)
        for (int j = (kb > L.S ? kb - L.S : 0); j < kb; ++j)
          mbar_wait(&full[j % L.S], (j / L.S) & 1u, nullptr, 50000000ull);
      }
    }
  } else if (warp == kGWarpMma) {
    if (lane == 0) {
      const uint32_t id = idesc(FMT_BF16, FMT_BF16, kGBM, static_cast<uint32_t>(NT));
      int kb = 0;
      bool ok = true;
      for (int q = 0; q < nsub && ok; ++q) {
        const int b = q & 1;
        if (!mbar_wait(&acc_empty[b], ((q >> 1) & 1u) ^ 1u, abort_flag)) {
          ok = false;
          break;
        }
        tc_fence_after();
        const uint32_t d_tmem = tmem_base + static_cast<uint32_t>(b * NT);
        const int kb_end = (kb + L.KBS < L.KB) ? kb + L.KBS : L.KB;
        for (int k = 0; kb < kb_end; ++kb, ++k) {
          const int st = kb % L.S;
          if (!mbar_wait(&full[st], (kb / L.S) & 1u, abort_flag)) {
            ok = false;
            break;
          }
          tc_fence_after();
          unsigned char* stage = smem + static_cast<uint32_t>(st) * L.stage_bytes;
          const uint64_t a = sdesc_sw128(stage);
#pragma unroll
          for (int ks = 0; ks < 4; ++ks) {
            const uint64_t o = static_cast<uint64_t>(ks * 2);  // 32 bytes along K
            for (int p = 0; p < L.P; ++p) {
              const uint64_t bd = sdesc_sw128(stage + kATileBytes + p * L.b_bytes);
              mma_f16(d_tmem, a + o, bd + o, id, (k | ks | p) != 0);
            }
          }
          mma_commit(&empty[st]);
        }
        if (ok) mma_commit(&acc_full[b]);
      }
      if (!ok) {
        atomicExch(&s_abort, 1);
        atomicExch(&state->timeout, 4);
      }
      // every MMA issued by this thread has completed before TMEM is released
      if (kb > 0) mbar_wait(&empty[(kb - 1) % L.S], ((kb - 1) / L.S) & 1u, nullptr, 50000000ull);
    }
  } else {  // epilogue warps 0-7
    const int lg = warp & 3, half = warp >> 2;
    const uint32_t lane_off = static_cast<uint32_t>(lg * 32) << 16;
    float hsum[CW];
#pragma unroll
    for (int i = 0; i < CW; ++i) hsum[i] = 0.0f;
    bool ok = true;
    for (int q = 0; q < nsub; ++q) {
      const int b = q & 1;
      int got = 0;
      if (lane == 0) got = mbar_wait(&acc_full[b], (q >> 1) & 1u, abort_flag) ? 1 : 0;
      got = __shfl_sync(0xFFFFFFFFu, got, 0);  // warp-uniform: tcgen05.ld is .sync.aligned
      if (!got) {
        ok = false;
        break;
      }
      tc_fence_after();
      const uint32_t taddr = tmem_base + lane_off + static_cast<uint32_t>(b * NT + half * CW);
      // 16 columns per load keeps the running sums (CW registers) plus one load within the
      // 168 registers a 320-thread block gets
#pragma unroll
      for (int c0 = 0; c0 < CW; c0 += 16) {
        float v[16];
        tmem_ld_32x32b_x16(taddr + static_cast<uint32_t>(c0), v);
#pragma unroll
        for (int i = 0; i < 16; ++i) hsum[c0 + i] += v[i];
      }
      tc_fence_before();
      __syncwarp();
      if (lane == 0) mbar_arrive(&acc_empty[b]);
    }
    if (ok) {
      // Write-back through shared memory (the pipeline stages are idle: every load has been
      // consumed by the MMAs that the last acc_full commit waited for).  Thread = row writes its
      // sums into a padded per-warp region; then the warp reads one row at a time with lanes
      // across columns, so the float64 read-add-write of SX is coalesced.
      float* region = reinterpret_cast<float*>(smem) + static_cast<size_t>(warp) * 32 * (CW + 1);
#pragma unroll
      for (int i = 0; i < CW; ++i) region[lane * (CW + 1) + i] = hsum[i];
      __syncwarp();
      const int64_t col_base = static_cast<int64_t>(n0) + half * CW;
      for (int r = 0; r < 32; ++r) {
        const int64_t row = static_cast<int64_t>(m0) + lg * 32 + r;
        if (row >= s) break;  // same r in every lane
        double* dst = SX + row * d;
        for (int c = lane; c < CW; c += 32) {
          const int64_t col = col_base + c;
          if (col < d) {
            const double add = static_cast<double>(region[r * (CW + 1) + c]) * scale;
            dst[col] = first ? add : dst[col] + add;
          }
        }
      }
    } else if (lane == 0) {
      atomicExch(&s_abort, 1);
      atomicExch(&state->timeout, 4);
    }
  }

  tc_fence_before();
  __syncthreads();
  if (warp == kGWarpMma) {
    tc_fence_after();
    tmem_dealloc(tmem_base, 2u * NT);
  }
}

// G[:, k0 : k0 + Kc] (s x Kc, row pitch Kc) in bfloat16; columns at or beyond n are zero.
// Entries whose float32 value lies near a bfloat16 rounding midpoint (about 1 in 2000) are queued
// in shared memory and rounded from the float64 evaluation once at least a block's worth has
// collected, so the float64 pipe (slow on this part) runs full warps rarely instead of stalling
// a warp for every such entry.
constexpr int kGenThreads = 256;
constexpr int kGenQueue = 2048;  // > kGenThreads - 1 + 4 * kGenThreads: one pass never overflows

__global__ void __launch_bounds__(kGenThreads) gauss_gen_kernel(uint64_t seed, int64_t s, int64_t n, int64_t row0,
                                                                int64_t k0, int64_t Kc,
                                                                __nv_bfloat16* __restrict__ Gc) {
  __shared__ uint32_t q_w0[kGenQueue], q_w1[kGenQueue];
  __shared__ int64_t q_at[kGenQueue];
  __shared__ int q_len;
  if (threadIdx.x == 0) q_len = 0;
  __syncthreads();
  auto drain = [&](int cnt) {
    for (int i = threadIdx.x; i < cnt; i += kGenThreads)
      Gc[q_at[i]] = __float2bfloat16_rn(bf16_round_f64(box_muller_f64(q_w0[i], q_w1[i])));
    __syncthreads();
    if (threadIdx.x == 0) q_len = 0;
    __syncthreads();
  };
  // grid: x over the Kc/4 Philox blocks of a row (grid-stride), y over rows of G (grid-stride);
  // no 64-bit division per block
  const int qn = static_cast<int>(Kc / 4);
  const int qstride = gridDim.x * kGenThreads;
  for (int64_t j = blockIdx.y; j < s; j += gridDim.y) {
    for (int q0 = blockIdx.x * kGenThreads; q0 < qn; q0 += qstride) {  // block-uniform
      const int q = q0 + threadIdx.x;
      if (q < qn) {
        const int64_t col = k0 + 4 * static_cast<int64_t>(q);  // k0 is a multiple of 4
        const int64_t at = j * Kc + 4 * static_cast<int64_t>(q);
        float g[4] = {0.0f, 0.0f, 0.0f, 0.0f};
        if (col < n) {
          // column row0 + col of G (row0 a multiple of 4): the block's row in the whole X
          const Gauss4 b = gaussian_block4_f32(seed, static_cast<uint32_t>(j), static_cast<uint64_t>(row0 + col) >> 2);
#pragma unroll
          for (int e = 0; e < 4; ++e) {
            if (col + e >= n) continue;
            if (!bf16_near_midpoint(b.z[e])) {
              g[e] = b.z[e];
            } else {
              const int slot = atomicAdd(&q_len, 1);
              if (slot < kGenQueue) {
                q_w0[slot] = b.w0[e];
                q_w1[slot] = b.w1[e];
                q_at[slot] = at + e;
              } else {
                g[e] = bf16_round_f64(box_muller_f64(b.w0[e], b.w1[e]));
              }
            }
          }
        }
        // queued entries are written here as 0 and overwritten by the drain (same block, after a barrier)
        const __nv_bfloat162 lo = __floats2bfloat162_rn(g[0], g[1]);
        const __nv_bfloat162 hi = __floats2bfloat162_rn(g[2], g[3]);
        uint2 o;
        o.x = *reinterpret_cast<const uint32_t*>(&lo);
        o.y = *reinterpret_cast<const uint32_t*>(&hi);
        *reinterpret_cast<uint2*>(Gc + at) = o;
      }
      __syncthreads();
      const int cnt = q_len < kGenQueue ? q_len : kGenQueue;
      __syncthreads();  // every thread has read q_len before anyone appends again
      if (cnt >= kGenThreads) drain(cnt);
    }
  }
  __syncthreads();
  const int cnt = q_len < kGenQueue ? q_len : kGenQueue;
  __syncthreads();
  if (cnt > 0) drain(cnt);
}

// X[k0 : k0 + Kc, :]^T as P bfloat16 pieces (piece p at XT + p*d*Kc, row c = column c of X, row
// pitch Kc); rows of X at or beyond n give zeros.  For float32 x: x1 = bf16(x), x2 = bf16(x - x1),
// x3 = bf16(x - x1 - x2) with x = x1 + x2 + x3 exactly (each remainder is exact in float32 and
// the last one has at most 8 significant bits).
template <typename T>
__global__ void __launch_bounds__(256) xt_split_kernel(const T* __restrict__ X, int64_t n, int64_t d, int64_t ldx,
                                                       int64_t k0, int64_t Kc, int P,
                                                       __nv_bfloat16* __restrict__ XT,
                                                       DevState* __restrict__ state) {
  __shared__ float tile[32][33];
  const int64_t c0 = static_cast<int64_t>(blockIdx.x) * 32, r0 = static_cast<int64_t>(blockIdx.y) * 32;
  bool bad = false;
  for (int rr = threadIdx.y; rr < 32; rr += blockDim.y) {
    const int64_t r = r0 + rr, c = c0 + threadIdx.x;
    float v = 0.0f;
    if (k0 + r < n && c < d) {
      v = to_float(X[(k0 + r) * ldx + c]);
      bad |= !isfinite(v);
    }
    tile[rr][threadIdx.x] = v;
  }
  __syncthreads();
  for (int cc = threadIdx.y; cc < 32; cc += blockDim.y) {
    const int64_t c = c0 + cc, r = r0 + threadIdx.x;
    if (c < d) {
      const float v = tile[threadIdx.x][cc];
      const __nv_bfloat16 x1 = __float2bfloat16_rn(v);
      __nv_bfloat16* dst = XT + c * Kc + r;
      dst[0] = x1;
      if (P == 3) {
        const float r1 = v - __bfloat162float(x1);
        const __nv_bfloat16 x2 = __float2bfloat16_rn(r1);
        const float r2 = r1 - __bfloat162float(x2);
        dst[d * Kc] = x2;
        dst[2 * d * Kc] = __float2bfloat16_rn(r2);
      }
    }
  }
  if (__syncthreads_or(bad) && threadIdx.x == 0 && threadIdx.y == 0) atomicOr(&state->nonfinite, 1);
}

// Tile width: the widest power of two (<= 256 for one piece, <= 128 for three, so that at least
// three stages fit; >= 64 so each epilogue warp reads at least 32 columns... or 16 at 32) whose
// padding of d stays within 15%.
int choose_nt(int64_t d, int P) {
  const int maxnt = (P == 1) ? 256 : 128;
  for (int nt = maxnt; nt > 32; nt >>= 1)
    if (ceil_div(d, nt) * nt * 100 <= d * 115) return nt;
  return 32;
}

GLayout make_glayout(int P, int NT, int64_t Kc) {
  GLayout L{};
  L.P = P;
  L.NT = NT;
  L.KB = static_cast<int>(Kc / kGKB);
  L.KBS = std::max(1, kStepsPerSub / (4 * P));  // 4 MMAs (K = 16 each) per K-block and piece
  L.b_bytes = static_cast<uint32_t>(NT) * 128u;
  L.stage_bytes = kATileBytes + static_cast<uint32_t>(P) * L.b_bytes;
  const uint32_t budget = 220u * 1024u;
  L.S = static_cast<int>(std::min<uint32_t>(kGMaxStages, budget / L.stage_bytes));
  L.bar_off = static_cast<uint32_t>(L.S) * L.stage_bytes;
  L.smem_bytes = L.bar_off + (2 * kGMaxStages + 5) * 8 + 1024;  // barriers, TMEM slot, 1 KB alignment
  return L;
}

template <int NT>
slso_status launch_gauss_tc(const dim3& grid, const GLayout& L, const CUtensorMap& mA, const CUtensorMap* mB,
                            int64_t s, int64_t d, double scale, int first, double* SX, DevState* state,
                            cudaStream_t st) {
  SLSO_TRY(raise_smem_limit(gauss_tc_kernel<NT>, L.smem_bytes));
  gauss_tc_kernel<NT><<<grid, kGThreads, L.smem_bytes, st>>>(mA, mB[0], mB[1], mB[2], L, s, d, scale, first, SX,
                                                             state);
  SLSO_CHECK_LAUNCH();
  return SLSO_OK;
}

}  // namespace

slso_status run_gauss_tc(Handle& h, Arena& ar, const void* X, int64_t n, int64_t d, int64_t ldx, int32_t xdt,
                         int64_t s, uint64_t seed, int64_t row0, bool accumulate, double* SX, cudaStream_t st,
                         bool* used) {
  *used = false;
  if (xdt != SLSO_F32 && xdt != SLSO_BF16) return SLSO_OK;
  if (row0 % 4 != 0 || !encode_fn()) return SLSO_OK;
  const int P = (xdt == SLSO_BF16) ? 1 : 3;
  const int NT = choose_nt(d, P);
  const int64_t Kc = std::min<int64_t>(kChunkRows, ceil_div(n, kGKB) * kGKB);
  const GLayout L = make_glayout(P, NT, Kc);
  if (L.S < 2) return SLSO_OK;
  // two chunk buffers: the side stream generates chunk i + 1 while the tensor cores take chunk i
  __nv_bfloat16* Gc[2];
  __nv_bfloat16* XT[2];
  for (int b = 0; b < 2; ++b) {
    Gc[b] = ar.take<__nv_bfloat16>(static_cast<size_t>(s) * Kc);
    XT[b] = ar.take<__nv_bfloat16>(static_cast<size_t>(P) * d * Kc);
  }
  *used = true;
  if (ar.measure()) return SLSO_OK;

  CUtensorMap mA[2], mB[2][3];
  bool ok = true;
  for (int b = 0; b < 2; ++b) {
    ok = ok && make_map(&mA[b], CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, Gc[b], Kc, s, Kc * 2, kGKB, kGBM);
    for (int p = 0; p < 3; ++p)
      ok = ok && make_map(&mB[b][p], CU_TENSOR_MAP_DATA_TYPE_BFLOAT16,
                          XT[b] + static_cast<size_t>(p < P ? p : 0) * d * Kc, Kc, d, Kc * 2, kGKB,
                          static_cast<uint32_t>(NT));
  }
  if (!ok) return fail(SLSO_ERR_CUDA, "cuTensorMapEncodeTiled failed for the Gaussian sketch operands");
  const double scale = 1.0 / std::sqrt(static_cast<double>(s));
  const dim3 grid_tc(static_cast<unsigned>(ceil_div(d, NT)), static_cast<unsigned>(ceil_div(s, kGBM)));
  const dim3 grid_xt(static_cast<unsigned>(ceil_div(d, 32)), static_cast<unsigned>(Kc / 32));
  // generator grid: enough blocks per row for the row's Kc/4 Philox blocks, rows spread over y
  const unsigned gen_x = static_cast<unsigned>(ceil_div(Kc / 4, kGenThreads));
  const unsigned gen_y = static_cast<unsigned>(std::max<int64_t>(
      1, std::min<int64_t>(s, ceil_div(int64_t(h.num_sms) * 8, static_cast<int64_t>(gen_x)))));
  const dim3 grid_gen(gen_x, gen_y);
  // Producer stream: the handle's side stream, forked from st (it starts after everything st holds)
  // and joined back (st waits for each chunk it consumes, the last one included); without a side
  // stream every launch goes to st in the same order.
  const bool two = h.side != nullptr && n > Kc;
  cudaStream_t ps = two ? h.side : st;
  if (two) {
    SLSO_CHECK_CUDA(cudaEventRecord(h.ev_fork, st));
    SLSO_CHECK_CUDA(cudaStreamWaitEvent(ps, h.ev_fork, 0));
  }
  int64_t i = 0;
  for (int64_t k0 = 0; k0 < n; k0 += Kc, ++i) {
    const int b = static_cast<int>(i & 1);
    if (two && i >= 2) SLSO_CHECK_CUDA(cudaStreamWaitEvent(ps, h.ev_free[b], 0));  // chunk i - 2 consumed
    gauss_gen_kernel<<<grid_gen, kGenThreads, 0, ps>>>(seed, s, n, row0, k0, Kc, Gc[b]);
    SLSO_CHECK_LAUNCH();
    if (xdt == SLSO_F32)
      xt_split_kernel<float><<<grid_xt, dim3(32, 8), 0, ps>>>(static_cast<const float*>(X), n, d, ldx, k0, Kc, P,
                                                              XT[b], h.state);
    else
      xt_split_kernel<__nv_bfloat16><<<grid_xt, dim3(32, 8), 0, ps>>>(static_cast<const __nv_bfloat16*>(X), n, d,
                                                                      ldx, k0, Kc, P, XT[b], h.state);
    SLSO_CHECK_LAUNCH();
    if (two) {
      SLSO_CHECK_CUDA(cudaEventRecord(h.ev_ready[b], ps));
      SLSO_CHECK_CUDA(cudaStreamWaitEvent(st, h.ev_ready[b], 0));
    }
    const int first = (k0 == 0 && !accumulate) ? 1 : 0;
    switch (NT) {
      case 256: SLSO_TRY(launch_gauss_tc<256>(grid_tc, L, mA[b], mB[b], s, d, scale, first, SX, h.state, st)); break;
      case 128: SLSO_TRY(launch_gauss_tc<128>(grid_tc, L, mA[b], mB[b], s, d, scale, first, SX, h.state, st)); break;
      case 64: SLSO_TRY(launch_gauss_tc<64>(grid_tc, L, mA[b], mB[b], s, d, scale, first, SX, h.state, st)); break;
      default: SLSO_TRY(launch_gauss_tc<32>(grid_tc, L, mA[b], mB[b], s, d, scale, first, SX, h.state, st)); break;
    }
    if (two) SLSO_CHECK_CUDA(cudaEventRecord(h.ev_free[b], st));
  }
  return SLSO_OK;
}

}  // namespace slso
