// Stable LSD radix sort of (key, u32 value) pairs and the "dec" ordering of scores
// (Algorithm 4 step 4, policy "dec" of Sec. 5.2).
//
// Three launches per 8-bit digit, with no inter-CTA waiting:
//   hist    each tile of 4096 keys counts its digits          -> hist[digit][tile]
//   scan    one CTA per digit: exclusive prefix over the tiles in place, and the digit's total
//   scatter each tile adds the exclusive prefix of the digit totals to its row of offsets, ranks
//           its keys stably (warp match + per-warp counters), places them in shared memory in
//           digit order and writes every digit's run to offset[digit][tile] + rank with
//           consecutive threads on consecutive addresses (keys, then values, through one buffer).
// Stability: tiles are contiguous and ordered, warps own contiguous 512-key runs inside a
// tile, and a warp walks its run 32 keys at a time in index order.
#include "common.cuh"

namespace slso {

namespace {

constexpr int kThreads = 256;
constexpr int kWarps = kThreads / 32;
constexpr int kItems = 16;                    // per thread
constexpr int kTile = kThreads * kItems;      // 4096 keys per CTA
constexpr int kWarpRun = 32 * kItems;         // 512 consecutive keys per warp
constexpr int kRadix = 256;
static_assert(kThreads == kRadix, "the scatter kernel computes one digit's start per thread");

template <class K>
__global__ void __launch_bounds__(kThreads) radix_hist_kernel(const K* __restrict__ keys,
                                                              int64_t n, int shift,
                                                              uint32_t* __restrict__ hist,
                                                              int ntiles) {
  __shared__ uint32_t cnt[kRadix];
  for (int i = threadIdx.x; i < kRadix; i += kThreads) cnt[i] = 0;
  __syncthreads();
  const int64_t base = static_cast<int64_t>(blockIdx.x) * kTile;
#pragma unroll 4
  for (int t = 0; t < kItems; ++t) {
    const int64_t idx = base + t * kThreads + threadIdx.x;
    if (idx < n) atomicAdd(&cnt[static_cast<uint32_t>(keys[idx] >> shift) & 0xFFu], 1u);
  }
  __syncthreads();
  for (int i = threadIdx.x; i < kRadix; i += kThreads)
    hist[static_cast<int64_t>(i) * ntiles + blockIdx.x] = cnt[i];
}

// One CTA per digit: hist[digit][.] becomes its exclusive prefix over the tiles (in tile order),
// totals[digit] the digit's count.
__global__ void __launch_bounds__(256) radix_scan_digit_kernel(uint32_t* __restrict__ hist, int ntiles,
                                                               uint32_t* __restrict__ totals) {
  __shared__ uint32_t wsum[8];
  const int t = threadIdx.x, lane = t & 31, w = t >> 5;
  uint32_t* row = hist + static_cast<int64_t>(blockIdx.x) * ntiles;
  const int per = (ntiles + 255) / 256;
  const int i0 = t * per, i1 = i0 + per < ntiles ? i0 + per : ntiles;
  uint32_t sum = 0;
  for (int i = i0; i < i1; ++i) sum += row[i];
  uint32_t x = sum;  // inclusive scan over the warp
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const uint32_t y = __shfl_up_sync(0xFFFFFFFFu, x, o);
    if (lane >= o) x += y;
  }
  if (lane == 31) wsum[w] = x;
  __syncthreads();
  uint32_t before = 0;
  for (int v = 0; v < w; ++v) before += wsum[v];
  uint32_t run = before + x - sum;  // exclusive
  for (int i = i0; i < i1; ++i) {
    const uint32_t c = row[i];
    row[i] = run;
    run += c;
  }
  if (t == 255) totals[blockIdx.x] = before + x;
}

template <class K>
__global__ void __launch_bounds__(kThreads) radix_scatter_kernel(
    const K* __restrict__ kin, const uint32_t* __restrict__ vin, K* __restrict__ kout,
    uint32_t* __restrict__ vout, int64_t n, int shift, const uint32_t* __restrict__ offs,
    const uint32_t* __restrict__ totals, int ntiles) {
  __shared__ uint32_t wcnt[kWarps][kRadix];
  __shared__ uint32_t gofs[kRadix];
  __shared__ uint32_t lstart[kRadix];
  __shared__ uint32_t wtot[kWarps];
  __shared__ __align__(16) unsigned char sbuf[kTile * sizeof(K)];  // the tile in digit order
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  for (int i = threadIdx.x; i < kWarps * kRadix; i += kThreads) (&wcnt[0][0])[i] = 0;
  // the digits' start: exclusive prefix of the totals (kThreads == kRadix: one digit per thread)
  {
    const uint32_t tot = totals[threadIdx.x];
    uint32_t x = tot;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const uint32_t y = __shfl_up_sync(0xFFFFFFFFu, x, o);
      if (lane >= o) x += y;
    }
    if (lane == 31) wtot[warp] = x;
    __syncthreads();
    uint32_t before = 0;
    for (int v = 0; v < warp; ++v) before += wtot[v];
    gofs[threadIdx.x] = before + x - tot + offs[static_cast<int64_t>(threadIdx.x) * ntiles + blockIdx.x];
  }
  __syncthreads();

  const int64_t base = static_cast<int64_t>(blockIdx.x) * kTile + warp * kWarpRun;
  const uint32_t lt_mask = (1u << lane) - 1u;
  K key[kItems];
  uint32_t val[kItems], rank[kItems];
#pragma unroll
  for (int r = 0; r < kItems; ++r) {
    const int64_t idx = base + r * 32 + lane;
    const bool valid = idx < n;
    const unsigned active = __ballot_sync(0xFFFFFFFFu, valid);
    key[r] = valid ? kin[idx] : K(0);
    val[r] = valid ? vin[idx] : 0u;
    rank[r] = 0;
    if (valid) {
      const uint32_t dg = static_cast<uint32_t>(key[r] >> shift) & 0xFFu;
      const unsigned peers = __match_any_sync(active, dg);
      const uint32_t before = wcnt[warp][dg];
      __syncwarp(active);
      if (lane == __ffs(peers) - 1) wcnt[warp][dg] = before + __popc(peers);
      __syncwarp(active);
      rank[r] = before + __popc(peers & lt_mask);
    }
  }
  __syncthreads();
  // exclusive prefix over warps for every digit, and the tile-local start of every digit (the
  // exclusive prefix of the tile's digit counts; one digit per thread)
  {
    const int dg = threadIdx.x;
    uint32_t run = 0;
    for (int w = 0; w < kWarps; ++w) {
      const uint32_t c = wcnt[w][dg];
      wcnt[w][dg] = run;
      run += c;
    }
    uint32_t x = run;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const uint32_t y = __shfl_up_sync(0xFFFFFFFFu, x, o);
      if (lane >= o) x += y;
    }
    if (lane == 31) wtot[warp] = x;  // the digit starts' use of wtot ended at the barrier above
    __syncthreads();
    uint32_t before = 0;
    for (int v = 0; v < warp; ++v) before += wtot[v];
    lstart[dg] = before + x - run;
  }
  __syncthreads();
  // tile-local position of every key: the digit's start, then the warps before, then the rank
  K* kbuf = reinterpret_cast<K*>(sbuf);
#pragma unroll
  for (int r = 0; r < kItems; ++r) {
    const int64_t idx = base + r * 32 + lane;
    if (idx < n) {
      const uint32_t dg = static_cast<uint32_t>(key[r] >> shift) & 0xFFu;
      rank[r] += lstart[dg] + wcnt[warp][dg];
      kbuf[rank[r]] = key[r];
    }
  }
  __syncthreads();
  const int64_t t0 = static_cast<int64_t>(blockIdx.x) * kTile;
  const int tn = static_cast<int>(n - t0 < kTile ? n - t0 : kTile);  // keys in this tile
  uint32_t dgs[kItems];
#pragma unroll
  for (int i = 0; i < kItems; ++i) {
    const int p = i * kThreads + threadIdx.x;
    if (p < tn) {
      const K k = kbuf[p];
      const uint32_t dg = static_cast<uint32_t>(k >> shift) & 0xFFu;
      dgs[i] = dg;
      kout[gofs[dg] + static_cast<uint32_t>(p) - lstart[dg]] = k;
    }
  }
  __syncthreads();
  uint32_t* vbuf = reinterpret_cast<uint32_t*>(sbuf);
#pragma unroll
  for (int r = 0; r < kItems; ++r)
    if (base + r * 32 + lane < n) vbuf[rank[r]] = val[r];
  __syncthreads();
#pragma unroll
  for (int i = 0; i < kItems; ++i) {
    const int p = i * kThreads + threadIdx.x;
    if (p < tn) vout[gofs[dgs[i]] + static_cast<uint32_t>(p) - lstart[dgs[i]]] = vbuf[p];
  }
}

template <class K>
slso_status radix_sort_impl(Arena& ar, K* keys, uint32_t* vals, int64_t n, int bits,
                            cudaStream_t st, K** kres, uint32_t** vres) {
  const int ntiles = static_cast<int>(ceil_div(n, kTile));
  K* kalt = ar.template take<K>(n);
  uint32_t* valt = ar.template take<uint32_t>(n);
  uint32_t* hist = ar.template take<uint32_t>(static_cast<size_t>(kRadix) * ntiles);
  uint32_t* totals = ar.template take<uint32_t>(kRadix);
  if (ar.measure()) return SLSO_OK;
  K* ka = keys;
  K* kb = kalt;
  uint32_t* va = vals;
  uint32_t* vb = valt;
  const int passes = (bits + 7) / 8;
  for (int p = 0; p < passes; ++p) {
    const int shift = 8 * p;
    radix_hist_kernel<K><<<ntiles, kThreads, 0, st>>>(ka, n, shift, hist, ntiles);
    SLSO_CHECK_LAUNCH();
    radix_scan_digit_kernel<<<kRadix, 256, 0, st>>>(hist, ntiles, totals);
    SLSO_CHECK_LAUNCH();
    radix_scatter_kernel<K><<<ntiles, kThreads, 0, st>>>(ka, va, kb, vb, n, shift, hist, totals, ntiles);
    SLSO_CHECK_LAUNCH();
    K* tk = ka; ka = kb; kb = tk;
    uint32_t* tv = va; va = vb; vb = tv;
  }
  *kres = ka;
  *vres = va;
  return SLSO_OK;
}

__global__ void keys_from_f32_kernel(const float* __restrict__ sc, int64_t n, uint32_t* __restrict__ k,
                                     uint32_t* __restrict__ v) {
  for (int64_t i = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; i < n;
       i += static_cast<int64_t>(gridDim.x) * blockDim.x) {
    k[i] = desc_key_f32(sc[i]);
    v[i] = static_cast<uint32_t>(i);
  }
}

__global__ void keys_from_f64_kernel(const double* __restrict__ sc, int64_t n,
                                     unsigned long long* __restrict__ k, uint32_t* __restrict__ v) {
  for (int64_t i = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; i < n;
       i += static_cast<int64_t>(gridDim.x) * blockDim.x) {
    k[i] = desc_key_f64(sc[i]);
    v[i] = static_cast<uint32_t>(i);
  }
}

__global__ void widen_order_kernel(const uint32_t* __restrict__ v, int64_t n, int64_t* __restrict__ o) {
  for (int64_t i = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; i < n;
       i += static_cast<int64_t>(gridDim.x) * blockDim.x)
    o[i] = static_cast<int64_t>(v[i]);
}

}  // namespace

slso_status radix_sort_u32(Arena& ar, uint32_t* keys, uint32_t* vals, int64_t n, int bits,
                           cudaStream_t st, uint32_t** keys_out, uint32_t** vals_out) {
  return radix_sort_impl<uint32_t>(ar, keys, vals, n, bits, st, keys_out, vals_out);
}

slso_status radix_sort_u64(Arena& ar, unsigned long long* keys, uint32_t* vals, int64_t n,
                           int bits, cudaStream_t st, unsigned long long** keys_out,
                           uint32_t** vals_out) {
  return radix_sort_impl<unsigned long long>(ar, keys, vals, n, bits, st, keys_out, vals_out);
}

slso_status order_scores(Handle& h, Arena& ar, const void* scores, int32_t sdt, int64_t n,
                         int64_t* order, cudaStream_t st) {
  const int grid = static_cast<int>(std::min<int64_t>(ceil_div(n, 256), 4LL * h.num_sms * 8));
  uint32_t* vals = ar.take<uint32_t>(n);
  uint32_t* vres = nullptr;
  if (sdt == SLSO_F32) {
    uint32_t* keys = ar.take<uint32_t>(n);
    uint32_t* kres = nullptr;
    if (!ar.measure()) {
      keys_from_f32_kernel<<<grid, 256, 0, st>>>(static_cast<const float*>(scores), n, keys, vals);
      SLSO_CHECK_LAUNCH();
    }
    SLSO_TRY(radix_sort_u32(ar, keys, vals, n, 32, st, &kres, &vres));
  } else {
    unsigned long long* keys = ar.take<unsigned long long>(n);
    unsigned long long* kres = nullptr;
    if (!ar.measure()) {
      keys_from_f64_kernel<<<grid, 256, 0, st>>>(static_cast<const double*>(scores), n, keys, vals);
      SLSO_CHECK_LAUNCH();
    }
    SLSO_TRY(radix_sort_u64(ar, keys, vals, n, 64, st, &kres, &vres));
  }
  if (ar.measure()) return SLSO_OK;
  widen_order_kernel<<<grid, 256, 0, st>>>(vres, n, order);
  SLSO_CHECK_LAUNCH();
  return SLSO_OK;
}

}  // namespace slso
