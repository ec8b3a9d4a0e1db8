// Internal definitions shared by the CUDA translation units of libslso.
#pragma once

#include <cuda.h>
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <cstddef>
#include <cstdint>
#include <type_traits>

#include "slso.h"

namespace slso {

// ------------------------------------------------------------------ errors
slso_status fail(slso_status st, const char* fmt, ...);

#define SLSO_CHECK_CUDA(expr)                                                                  \
  do {                                                                                         \
    cudaError_t e_ = (expr);                                                                   \
    if (e_ != cudaSuccess)                                                                     \
      return ::slso::fail(SLSO_ERR_CUDA, "%s failed: %s (%s:%d)", #expr, cudaGetErrorString(e_), \
                          __FILE__, __LINE__);                                                 \
  } while (0)

// Every kernel launch is followed by exactly one SLSO_CHECK_LAUNCH (cooperative launches call
// note_launch), which also counts the launch for slso_profile_read.
void note_launch();
#define SLSO_CHECK_LAUNCH()      \
  do {                           \
    ::slso::note_launch();       \
    SLSO_CHECK_CUDA(cudaGetLastError()); \
  } while (0)

#define SLSO_TRY(expr)              \
  do {                              \
    slso_status s_ = (expr);        \
    if (s_ != SLSO_OK) return s_;   \
  } while (0)

// ------------------------------------------------------------------ device status words
// One per handle, in device memory.  Kernels only ever set fields (never wait on them).
struct DevState {
  int32_t nonfinite;     // X held NaN/Inf
  int32_t need_svd;      // certification failed: take the SVD route
  int32_t timeout;       // a bounded wait gave up (id of the kernel)
  int32_t rank;          // numerical rank r
  int32_t rotations;     // Jacobi: rotations applied in the current sweep
  int32_t sweeps;        // Jacobi: sweeps run
  int32_t gram_ok;       // Gram route: 1 while its factor stands (the Householder kernels then return)
  int32_t gram_tried;    // Gram route attempted
  double sigma_max;      // sigma_1 (SVD route)
  double sigma_min_kept; // sigma_r (SVD route)
  double score_sum;
  double tau;
  double fro_r;          // ||R||_F
  double fro_rinv;       // ||R^-1||_F
  double gram_resid;     // Gram route: probe estimate of ||R^-T SX^T SX R^-1 - I||_F (NaN: breakdown)
  int32_t m_ready;       // M = R^-1 Pi already written by the float-float Gram route
  int32_t gemm_gate;     // 1: M is formed from R^-1 by the float64 product (certified, not yet written)
};

// ------------------------------------------------------------------ scratch arena
// Every internal run function first takes all of its buffers from an Arena and only then
// launches.  Run once with a measuring arena to size the pool, then for real.
class Arena {
 public:
  Arena(char* base, size_t cap, bool measure) : base_(base), cap_(cap), off_(0), measure_(measure) {}
  template <class T>
  T* take(size_t count) {
    size_t off = (off_ + 255) & ~size_t(255);
    off_ = off + count * sizeof(T);
    if (measure_ || off_ > cap_) return nullptr;
    return reinterpret_cast<T*>(base_ + off);
  }
  bool measure() const { return measure_; }
  size_t used() const { return off_; }
  bool overflow() const { return off_ > cap_; }

 private:
  char* base_;
  size_t cap_;
  size_t off_;
  bool measure_;
};

// Stage timing for slso_profile / slso_profile_read: event pairs recorded on the caller's
// stream around each stage, summed when read.
enum Stage {
  ST_SKETCH = 0, ST_QR = 1, ST_SOLVE = 2, ST_SCORES = 3, ST_ORDER = 4, ST_COPY = 5, ST_SYRK = 6, ST_CHOL = 7,
  ST_COUNT = 8
};

struct ProfRecord {
  int stage;
  cudaEvent_t a, b;
};

struct Handle {
  int device = 0;
  int num_sms = 0;
  char* pool = nullptr;
  size_t pool_cap = 0;
  size_t pool_limit = 0;           // 0: no cap (slso_set_pool_limit)
  DevState* state = nullptr;       // device
  DevState* state_host = nullptr;  // pinned mirror for info
  bool prof = false;
  ProfRecord* recs = nullptr;      // capacity kProfCap
  int nrec = 0;
  int open_rec = -1;
  long long launches_at_enable = 0;
  int score_form = 0;              // float32 scores, k <= 128: SLSO_SCORE_FORM_* (slso_set_score_form)
  // A second stream forked from and joined back into the call's stream (producer work that
  // overlaps the tensor-core kernels: the Gaussian sketch's G and X^T chunks), with its events.
  cudaStream_t side = nullptr;
  cudaEvent_t ev_fork = nullptr, ev_ready[2] = {nullptr, nullptr}, ev_free[2] = {nullptr, nullptr};
};

// Create / release the handle's side stream and events (no-ops when already done / absent).
cudaError_t side_stream_create(Handle& h);
void side_stream_release(Handle& h);
constexpr int kProfCap = 4096;

// Begin / end a timed stage on stream st (no-ops unless profiling is on).
void prof_begin(Handle& h, const Arena& ar, int stage, cudaStream_t st);
void prof_end(Handle& h, const Arena& ar, cudaStream_t st);

slso_status ensure_pool(Handle& h, size_t bytes);

// Raise fn's dynamic shared-memory limit on the current device to at least `bytes`, never lowering
// it.  The limit belongs to the function, not to a launch: every call, host thread and captured
// graph shares it, so setting it to one call's size would make a concurrent or later launch with
// more shared memory fail.
slso_status raise_smem_limit(const void* fn, size_t bytes);
template <class F>
slso_status raise_smem_limit(F* fn, size_t bytes) {
  return raise_smem_limit(reinterpret_cast<const void*>(fn), bytes);
}
slso_status check_handle(slso_handle* hp, Handle** out);

inline int64_t ceil_div(int64_t a, int64_t b) { return (a + b - 1) / b; }
// Largest d (columns of X): R^-1's column-at-a-time kernel keeps d doubles in shared memory.
constexpr int64_t kMaxD = 24576;
inline size_t dtype_size(int32_t dt) {
  switch (dt) {
    case SLSO_F64: return 8;
    case SLSO_F32: return 4;
    case SLSO_BF16: return 2;
    case SLSO_FP8_E4M3: return 1;
    default: return 0;
  }
}

// ------------------------------------------------------------------ Philox4x32-10
// Salmon, Moraes, Dror, Shaw, SC'11: two 32x32->64 multiplies per round, Weyl key bumps.
struct U32x4 {
  uint32_t x, y, z, w;
};

__device__ __forceinline__ U32x4 philox(uint32_t c0, uint32_t c1, uint32_t c2, uint32_t c3,
                                        uint64_t key) {
  uint32_t k0 = static_cast<uint32_t>(key), k1 = static_cast<uint32_t>(key >> 32);
#pragma unroll
  for (int r = 0; r < 10; ++r) {
    if (r) {
      k0 += 0x9E3779B9u;
      k1 += 0xBB67AE85u;
    }
    const uint32_t lo0 = 0xD2511F53u * c0, hi0 = __umulhi(0xD2511F53u, c0);
    const uint32_t lo1 = 0xCD9E8D57u * c2, hi1 = __umulhi(0xCD9E8D57u, c2);
    const uint32_t n0 = hi1 ^ c1 ^ k0, n2 = hi0 ^ c3 ^ k1;
    c0 = n0;
    c1 = lo1;
    c2 = n2;
    c3 = lo0;
  }
  return {c0, c1, c2, c3};
}

enum : uint32_t {
  TAG_COUNTSKETCH = 1,
  TAG_SRHT_SIGN = 2,
  TAG_SRHT_SAMPLE = 3,
  TAG_GAUSSIAN = 4,
  TAG_JL = 5,
  TAG_OSNAP = 7,
  TAG_PROBE = 8
};

// ------------------------------------------------------------------ Box-Muller
// Normal deviate sqrt(-2 ln u1) cos(2 pi u2), u1 = (w0+1) 2^-32, u2 = w1 2^-32, evaluated from
// exact arguments: ln u1 through log1p(-m 2^-32), m = 2^32-1-w0, when w0 >= 2^31; the angle is
// reduced to its octant o = w1 >> 29 and an exact fraction c in [0,1] so that the cosine is
// +-sin or +-cos of (pi/4) c.
__device__ __forceinline__ double box_muller_f64(uint32_t w0, uint32_t w1) {
  const double ln_u1 = (w0 >= 0x80000000u)
                           ? log1p(-static_cast<double>(0xFFFFFFFFu - w0) * 0x1p-32)
                           : log((static_cast<double>(w0) + 1.0) * 0x1p-32);
  const double rho = sqrt(-2.0 * ln_u1);
  const uint32_t oct = w1 >> 29;
  const bool odd = oct & 1u;
  const uint32_t f = w1 & 0x1FFFFFFFu;
  const uint32_t ci = odd ? (0x20000000u - f) : f;  // exact integer in [0, 2^29]
  const double arg = static_cast<double>(ci) * 0x1p-31;  // (pi/4) c = pi * arg
  const double sn = sinpi(arg), cs = cospi(arg);
  const uint32_t q = odd ? (oct + 1) >> 1 : oct >> 1;
  double v;
  switch (q) {
    case 0: v = cs; break;
    case 1: v = odd ? sn : -sn; break;
    case 2: v = -cs; break;
    case 3: v = odd ? -sn : sn; break;
    default: v = cs; break;
  }
  return rho * v;
}

// Same formula in float32: a few ulp from the exact value (each factor within ~2 ulp).
__device__ __forceinline__ float box_muller_f32(uint32_t w0, uint32_t w1) {
  const float ln_u1 = (w0 >= 0x80000000u)
                          ? log1pf(-static_cast<float>(0xFFFFFFFFu - w0) * 0x1p-32f)
                          : logf((static_cast<float>(w0) + 1.0f) * 0x1p-32f);
  const float rho = sqrtf(-2.0f * ln_u1);
  const uint32_t oct = w1 >> 29;
  const bool odd = oct & 1u;
  const uint32_t f = w1 & 0x1FFFFFFFu;
  const uint32_t ci = odd ? (0x20000000u - f) : f;
  const float arg = static_cast<float>(ci) * 0x1p-31f;
  const float sn = sinpif(arg), cs = cospif(arg);
  const uint32_t q = odd ? (oct + 1) >> 1 : oct >> 1;
  float v;
  switch (q) {
    case 0: v = cs; break;
    case 1: v = odd ? sn : -sn; break;
    case 2: v = -cs; break;
    case 3: v = odd ? -sn : sn; break;
    default: v = cs; break;
  }
  return rho * v;
}

// Round a float64 to bfloat16 (8 significant bits), nearest-even, in one step on the bits.
__device__ __forceinline__ float bf16_round_f64(double x) {
  unsigned long long b = static_cast<unsigned long long>(__double_as_longlong(x));
  const unsigned long long lsb = (b >> 45) & 1ull;
  b = (b + ((1ull << 44) - 1ull) + lsb) & ~((1ull << 45) - 1ull);
  return static_cast<float>(__longlong_as_double(static_cast<long long>(b)));
}

// bfloat16 value of the float64 normal deviate BoxMuller(w0, w1), given its float32 evaluation
// z, with the rounding decided exactly as float64 rounding would decide it.  The float32
// evaluation is within 4 float32 ulp of the exact value (logf / log1pf <= 1 ulp, sqrtf exact,
// sinpif / cospif <= 1 ulp, plus the roundings of their arguments and of the product); when it
// lies further than kBf16Margin float32 ulp from a bfloat16 rounding midpoint its nearest-even
// rounding equals that of the exact value, otherwise the float64 evaluation decides.
constexpr int kBf16Margin = 16;

__device__ __forceinline__ bool bf16_near_midpoint(float z) {
  const int dist = static_cast<int>(__float_as_uint(z) & 0xFFFFu) - 0x8000;
  return dist <= kBf16Margin && dist >= -kBf16Margin;
}

__device__ __forceinline__ float bf16_decide(float z, uint32_t w0, uint32_t w1) {
  if (!bf16_near_midpoint(z)) return __bfloat162float(__float2bfloat16_rn(z));
  return bf16_round_f64(box_muller_f64(w0, w1));
}

__device__ __forceinline__ float gaussian_bf16_value(uint32_t w0, uint32_t w1) {
  return bf16_decide(box_muller_f32(w0, w1), w0, w1);
}

// Gaussian sketch entries.  Four consecutive columns i = 4b..4b+3 of row j share the Philox
// block (lo b, hi b, j, TAG_GAUSSIAN): columns 4b, 4b+1 are the cosine and sine normals of the
// Box-Muller pair (w0, w1), columns 4b+2, 4b+3 those of (w2, w3).  sin(2 pi w 2^-32) is the
// cosine of the word w - 2^30 (mod 2^32), which keeps the exact-argument evaluation.
constexpr uint32_t kQuarterTurnWord = 0x40000000u;

__device__ __forceinline__ float gaussian_entry(uint64_t seed, uint32_t row_j, uint64_t col_i) {
  const uint64_t blk = col_i >> 2;
  const U32x4 w = philox(static_cast<uint32_t>(blk), static_cast<uint32_t>(blk >> 32), row_j, TAG_GAUSSIAN, seed);
  const uint32_t r = static_cast<uint32_t>(col_i & 3u);
  const uint32_t wa = r < 2 ? w.x : w.z;
  uint32_t wb = r < 2 ? w.y : w.w;
  if (r & 1u) wb -= kQuarterTurnWord;
  return gaussian_bf16_value(wa, wb);
}

// float32 sqrt(-2 ln u1), u1 = (w+1) 2^-32 (log1p near 1, as in box_muller_f32).
__device__ __forceinline__ float bm_radius_f32(uint32_t w) {
  const float ln_u1 = (w >= 0x80000000u) ? log1pf(-static_cast<float>(0xFFFFFFFFu - w) * 0x1p-32f)
                                         : logf((static_cast<float>(w) + 1.0f) * 0x1p-32f);
  return sqrtf(-2.0f * ln_u1);
}

// Signed +-sin / +-cos of the reduced angle for octant o (same selection as box_muller_f32).
__device__ __forceinline__ float bm_quarter(uint32_t oct, float sn, float cs) {
  const bool odd = oct & 1u;
  const uint32_t q = odd ? (oct + 1) >> 1 : oct >> 1;
  switch (q) {
    case 0: return cs;
    case 1: return odd ? sn : -sn;
    case 2: return -cs;
    case 3: return odd ? -sn : sn;
    default: return cs;
  }
}

// float32 cos and sin of 2 pi w 2^-32 from one reduced argument: the word w - 2^30 has octant
// o - 2 (mod 8) and the same fraction, hence the same sinpi/cospi values.
__device__ __forceinline__ void bm_cos_sin_f32(uint32_t w, float& c, float& s) {
  const uint32_t oct = w >> 29;
  const uint32_t f = w & 0x1FFFFFFFu;
  const uint32_t ci = (oct & 1u) ? (0x20000000u - f) : f;
  float sn, cs;
  sincospif(static_cast<float>(ci) * 0x1p-31f, &sn, &cs);
  c = bm_quarter(oct, sn, cs);
  s = bm_quarter((oct - 2u) & 7u, sn, cs);
}

// The four entries G[j, 4b..4b+3] in float32 (z) with the words each came from; the caller
// rounds them with bf16_decide (or defers the entries with bf16_near_midpoint set).
struct Gauss4 {
  float z[4];
  uint32_t w0[4], w1[4];
};

__device__ __forceinline__ Gauss4 gaussian_block4_f32(uint64_t seed, uint32_t row_j, uint64_t blk) {
  const U32x4 w = philox(static_cast<uint32_t>(blk), static_cast<uint32_t>(blk >> 32), row_j, TAG_GAUSSIAN, seed);
  const float ra = bm_radius_f32(w.x), rb = bm_radius_f32(w.z);
  float ca, sa, cb, sb;
  bm_cos_sin_f32(w.y, ca, sa);
  bm_cos_sin_f32(w.w, cb, sb);
  Gauss4 g;
  g.z[0] = ra * ca;
  g.z[1] = ra * sa;
  g.z[2] = rb * cb;
  g.z[3] = rb * sb;
  g.w0[0] = g.w0[1] = w.x;
  g.w0[2] = g.w0[3] = w.z;
  g.w1[0] = w.y;
  g.w1[1] = w.y - kQuarterTurnWord;
  g.w1[2] = w.w;
  g.w1[3] = w.w - kQuarterTurnWord;
  return g;
}

// ------------------------------------------------------------------ small helpers
__device__ __forceinline__ float to_float(float v) { return v; }
__device__ __forceinline__ float to_float(__nv_bfloat16 v) { return __bfloat162float(v); }
__device__ __forceinline__ float to_float(double v) { return static_cast<float>(v); }

__device__ __forceinline__ float to_float_or_double(float v) { return v; }
__device__ __forceinline__ float to_float_or_double(__nv_bfloat16 v) { return __bfloat162float(v); }
__device__ __forceinline__ double to_float_or_double(double v) { return v; }

// Knuth's TwoSum: hi + lo accumulates x with the rounding error of every add kept in lo.
__device__ __forceinline__ void two_sum_acc(float& hi, float& lo, float x) {
  const float s = hi + x;
  const float bp = s - hi;
  const float err = (hi - (s - bp)) + (x - bp);
  hi = s;
  lo += err;
}

__device__ __forceinline__ void comp_add(float& hi, float& lo, float x) { two_sum_acc(hi, lo, x); }
__device__ __forceinline__ void comp_add(double& hi, double& lo, double x) {
  hi += x;
  (void)lo;
}

// Descending-order radix keys: NaN -> all ones (last); -0 -> +0.
__device__ __forceinline__ uint32_t desc_key_f32(float f) {
  if (isnan(f)) return 0xFFFFFFFFu;
  if (f == 0.0f) f = 0.0f;
  const uint32_t u = __float_as_uint(f);
  const uint32_t ord = (u & 0x80000000u) ? ~u : (u | 0x80000000u);
  return ~ord;
}
__device__ __forceinline__ unsigned long long desc_key_f64(double f) {
  if (isnan(f)) return ~0ull;
  if (f == 0.0) f = 0.0;
  const unsigned long long u = static_cast<unsigned long long>(__double_as_longlong(f));
  const unsigned long long ord = (u >> 63) ? ~u : (u | (1ull << 63));
  return ~ord;
}

// Bounded spin on a flag written by another CTA of the same (co-resident) grid.
// Returns false after ~`limit` polls; the caller records a timeout and bails out.
__device__ __forceinline__ bool wait_flag_geq(const volatile int* flag, int value, long long limit) {
  for (long long it = 0; it < limit; ++it) {
    if (*flag >= value) return true;
    __nanosleep(64);
  }
  return *flag >= value;
}

}  // namespace slso

// ------------------------------------------------------------------ cross-TU host interface
namespace slso {

// sort.cu
slso_status radix_sort_u32(Arena& ar, uint32_t* keys, uint32_t* vals, int64_t n, int bits,
                           cudaStream_t st, uint32_t** keys_out, uint32_t** vals_out);
slso_status radix_sort_u64(Arena& ar, unsigned long long* keys, uint32_t* vals, int64_t n,
                           int bits, cudaStream_t st, unsigned long long** keys_out,
                           uint32_t** vals_out);
slso_status order_scores(Handle& h, Arena& ar, const void* scores, int32_t sdt, int64_t n,
                         int64_t* order, cudaStream_t st);

// sketch.cu
// nnz: OSNAP's nonzeros per column of S (ignored by the other kinds).
constexpr int kOsnapDefaultNnz = 4;
// A block of rows of a larger X (the streamed entry point): the block is rows row0 .. row0 + n - 1
// of an X with n_total rows (the sketch's hash, sign and Gaussian counters use those global
// indices), and with accumulate its sketch is added to SX.  SRHT needs row0 to be a multiple of
// 8192 and the sampled rows of H drawn once for n_total (srht_sample_rows).
struct SketchBlock {
  int64_t row0 = 0;
  int64_t n_total = 0;  // 0: the block is the whole X
  bool accumulate = false;
  const uint32_t* srht_rows = nullptr;
  // CountSketch / OSNAP of float32 or bfloat16 X: also max_i |X_ij| per column j into colmax (float
  // bits; the caller zeroes it), for the FP8 scores' column scales
  unsigned int* colmax = nullptr;
};
slso_status run_sketch(Handle& h, Arena& ar, const void* X, int64_t n, int64_t d, int64_t ldx,
                       int32_t xdt, int32_t kind, int64_t s, uint64_t seed, int nnz, double* SX,
                       cudaStream_t st, const SketchBlock* blk = nullptr);
slso_status srht_sample_rows(Handle& h, Arena& ar, int64_t n_total, int64_t s, uint64_t seed,
                             const uint32_t** rows, cudaStream_t st);

// solve.cu
struct SolveOut {
  double* M = nullptr;      // d x kk row-major float64 (kk = k, or d when k = 0)
  double* sigma = nullptr;  // d (SVD route / sketched SVD)
  double* V = nullptr;      // d x d row-major (column j = v_j)
  double* R = nullptr;      // d x d row-major
  int64_t kk = 0;
};
// mode 0: leverage (certified inverse or SVD); mode 1: sketched SVD only (always SVD).
// gram (mode 0 only): try the Gram route for R first (gram.cu), Householder when it fails.
slso_status run_solve(Handle& h, Arena& ar, const double* SX, int64_t s, int64_t d, double tau,
                      int64_t k, uint64_t seed_pi, int mode, SolveOut* out, cudaStream_t st,
                      bool gram = false);

// gram.cu: R of SX from the Cholesky factor of G = SX^T SX, with a probe check.
// gram_take takes the buffers (call before the arena's measuring return); run_gram_factor writes
// L = R^T (d x d row-major lower triangle, i.e. R column-major) into L and sets state->gram_ok;
// run_gram_check (after R^-1, column-major, is in Rinv) clears gram_ok when the probe estimate
// of ||R^-T SX^T SX R^-1 - I||_F exceeds kGramTol.
constexpr double kGramTol = 1e-8;
// gram_tc.cu: G = SX^T SX on the tensor cores from six exact bfloat16 digit slices of the scaled
// columns (float64-class accuracy), written like the float-float SYRK's reduction into L.
struct GramTcWork {
  __nv_bfloat16* E = nullptr;  // 6 dpad x sp slices, K (rows of SX) contiguous
  long long* part = nullptr;   // split partial tiles (128 x 64 int64 sums)
  int* bad = nullptr;          // a non-finite SX entry was met
  int dpad = 0, nbJ = 0, tiles = 0, splits = 1;
  int64_t sp = 0, kc = 0;
};
bool gram_tc_applies(int64_t s, int64_t d);
void gram_tc_take(Arena& ar, int64_t s, int64_t d, GramTcWork* w);
slso_status run_gram_tc(Handle& h, const GramTcWork& w, const double* SX, int64_t s, int64_t d, const int* cexp,
                        double* L, cudaStream_t st);
struct GramWork {
  double* part = nullptr;   // split-K partial tiles of the Gram matrix
  double* Z = nullptr;      // d x P probes
  double* Y = nullptr;      // d x P
  double* W = nullptr;      // s x P
  double* vpart = nullptr;  // row-chunk partials of SX^T W
  double* V = nullptr;      // d x P
  double* eres = nullptr;   // d per-row squared residuals
  double* ldiag = nullptr;  // the factored 32 x 32 diagonal blocks of the Cholesky factor
  unsigned long long* colmax = nullptr;  // per column max |SX| (float64 bits)
  int* cexp = nullptr;      // per column scale exponent e_j
  double* cscale = nullptr; // 2^-e_j
  float* xh = nullptr;      // SX 2^-e_j split into float32 parts xh + xl (s x d row-major)
  float* xl = nullptr;
  bool use_tc = false;      // G from the tensor-core route (gram_tc.cu) instead of the float-float SYRK
  GramTcWork tc;
  bool use_ff = false;      // Cholesky, R^-1, M and the probe check in float-float (chol_ff.cu)
  float2* Aff = nullptr;    // d x d float-float working matrices of chol_ff
  float2* Xff = nullptr;
  unsigned int* cbar = nullptr;
  float2* Dbuf = nullptr;   // 2 x 32 x 32: the lookahead's diagonal block
  float2* Outff = nullptr;  // d x (k + 4): X'^T [Pi | Z]
  float2* Yff = nullptr;    // d x P: X'^T Z
  float2* Wff = nullptr;    // s x P
  float2* vff = nullptr;    // row-chunk partials of SX'^T W
  float2* Vff = nullptr;    // d x P
  int splits = 1, tiles = 0, vchunks = 1;
  int64_t kc = 0;
};
// k: the JL width of the call (0: none), for the float-float route's right-hand sides.
GramWork gram_take(Handle& h, Arena& ar, int64_t s, int64_t d, int64_t k = 0);
// With g.use_ff the factor's inverse is written to Rinv (column-major R^-1) as well, and
// *rinv_done is set; otherwise the caller forms R^-1 from L.
// Pi (d x k, k > 0, or NULL) is generated before the call, on st or on another stream whose event
// pi_ready st waits for once G is formed: with g.use_ff, M = R^-1 Pi is written too
// (state->m_ready).
slso_status run_gram_factor(Handle& h, const Arena& ar, const GramWork& g, const double* SX, int64_t s,
                            int64_t d, double* L, double* Rinv, bool* rinv_done, const double* Pi, int64_t k,
                            double* M, cudaStream_t st, cudaEvent_t pi_ready = nullptr);
// chol_ff.cu: L (G's lower triangle in, R^T out) and Rinv from the float-float Cholesky.
bool chol_ff_applies(int64_t d);
slso_status run_chol_ff(Handle& h, double* L, const int* cexp, int64_t d, float2* A, float2* X, double* Rinv,
                        const double* Pi, int64_t k, const double* Z, double* M, float2* Yff, unsigned int* bar,
                        float2* Dbuf, float2* Out, cudaStream_t st);
slso_status run_probe_ff(Handle& h, const double* SX, int64_t s, int64_t d, const int* cexp, const float2* X,
                         const float2* Yff, float2* Wff, float2* vpart, int chunks, float2* Vff, const double* Z,
                         double* eres, cudaStream_t st);
// G = SX^T SX alone: its lower triangle into L (d x d row-major); run_gram_full also writes the
// whole symmetric G (d x d row-major).
slso_status run_gram_matrix(Handle& h, const Arena& ar, const GramWork& g, const double* SX, int64_t s,
                            int64_t d, double* L, cudaStream_t st);
slso_status run_gram_full(Handle& h, const Arena& ar, const GramWork& g, const double* SX, int64_t s, int64_t d,
                          double* L, double* G, cudaStream_t st);
slso_status run_gram_check(Handle& h, const GramWork& g, const double* SX, int64_t s, int64_t d,
                           const double* Rinv, cudaStream_t st);

// api.cu: argument checks and the leverage plan shared with the server
double default_tau(int64_t s, int64_t d);
slso_status check_x(const void* X, int64_t n, int64_t d, int64_t ldx, int32_t xdt);
slso_status check_params(const slso_params* p, int64_t n, int64_t d);
bool use_gram(const slso_params* p);  // the Gram route is tried for this leverage call
// Every slso_info field from a call's device status words.
void info_from_state(const DevState& d, slso_info* info);
slso_status leverage_plan(Handle& h, Arena& ar, const void* X, int64_t n, int64_t d, int64_t ldx,
                          int32_t xdt, const slso_params* p, void* scores, cudaStream_t st);
// leverage_plan up to M (sketch and solve): M (d x kk) and the FP8 column maxima (or NULL).
slso_status leverage_solve(Handle& h, Arena& ar, const void* X, int64_t n, int64_t d, int64_t ldx,
                           int32_t xdt, const slso_params* p, cudaStream_t st, const double** M, int64_t* kk,
                           const unsigned int** colmax);

// Approximate left singular vectors U = X V_r Sigma_r^-1 of the sketched SVD (basis.cu).
slso_status approx_u_plan(Handle& h, Arena& ar, const void* X, int64_t n, int64_t d, int64_t ldx, int32_t xdt,
                          const slso_params* p, void* U, int64_t ldu, cudaStream_t st);
// Orderings of Algorithm 4 step 4 (policy dec, swr or swor) into order (int64, n).
slso_status sample_order(Handle& h, Arena& ar, const void* scores, int32_t sdt, int64_t n, int32_t policy,
                         uint64_t seed, int64_t* order, cudaStream_t st);
// Tensor-core Gaussian sketch for float32 / bfloat16 X; *used = false when it does not apply
// (float64 X or no tensor-map support), and the SIMT kernels run instead.
// row0: the first row's index in the whole X (a multiple of 4); accumulate adds to SX.
slso_status run_gauss_tc(Handle& h, Arena& ar, const void* X, int64_t n, int64_t d, int64_t ldx, int32_t xdt,
                         int64_t s, uint64_t seed, int64_t row0, bool accumulate, double* SX, cudaStream_t st,
                         bool* used);
// One job of a grouped score launch (the serving path): the tensor maps of its X and of its
// packed B, its rows, scores and device status, its K-blocks, its first global work item (before
// score_group_launch numbers the items: its count of work items), its JL width and form.
struct ScoreGroupJob {
  CUtensorMap tmX, tmBh;
  int64_t n;
  float* scores;
  DevState* state;
  int KB, work0, N, hyb;
};
constexpr int kMaxScoreGroup = 8;

// score_tc.cu: tensor-core scores; *used = false when the shapes need the SIMT kernel
// colmax_pre (FP8 only, optional): the column maxima of |X| already formed by the sketch pass.
// With group != nullptr, a float32 score product that takes the two-tile tensor-memory kernel is
// prepared exactly as for its own launch (same scratch, same B pieces) and described in *group
// instead of launched.
slso_status run_scores_tc(Handle& h, Arena& ar, const void* X, int64_t n, int64_t d, int64_t ldx, int32_t xdt,
                          const double* M, int64_t kk, int32_t compute, float* scores, bool* used,
                          cudaStream_t st, const unsigned int* colmax_pre = nullptr,
                          ScoreGroupJob* group = nullptr);
// Whether a leverage call's scores can join a grouped launch: float32 X and compute, k in
// [1, 128], d <= 2048, 16-byte aligned rows, no correction pass, the default score form.
bool score_group_eligible(const Handle& h, const void* X, int64_t d, int64_t ldx, int32_t xdt, int64_t k,
                          int32_t compute, double correct_frac);
// The scratch and preparation of scores_typed for such a call, with the product described in *job
// (state: h.state); *sums receives the score-sum scratch that score_group_sum needs afterwards.
slso_status score_group_add(Handle& h, Arena& ar, const void* X, int64_t n, int64_t d, int64_t ldx, const double* M,
                            int64_t kk, float* scores, ScoreGroupJob* job, double** sums, cudaStream_t st);
// One launch over the described jobs (all with the same N and form): work items numbered job by
// job; the descriptors are copied from host (pinned, kept until the launch has run) to device.
slso_status score_group_launch(Handle& h, ScoreGroupJob* host, ScoreGroupJob* dev, int njobs, cudaStream_t st);
// The score sum of one grouped job (into h.state), as the one-job path forms it.
slso_status score_group_sum(Handle& h, const float* scores, int64_t n, double* sums, cudaStream_t st);

// Y = X M (M d x kk row-major float64) written to U (float32, row stride ldu) on the tensor cores
// for float32 / bfloat16 X (score_tc.cu); *used = false when the SIMT kernel must run instead.
slso_status run_product_tc(Handle& h, Arena& ar, const void* X, int64_t n, int64_t d, int64_t ldx, int32_t xdt,
                           const double* M, int64_t kk, float* U, int64_t ldu, bool* used, cudaStream_t st);

// score.cu
// state->score_sum = the sum of n scores (F32 or F64), in a fixed order.
slso_status score_sum(Handle& h, Arena& ar, const void* scores, int32_t sdt, int64_t n, cudaStream_t st);
slso_status run_scores(Handle& h, Arena& ar, const void* X, int64_t n, int64_t d, int64_t ldx,
                       int32_t xdt, const double* M, int64_t kk, int32_t compute, void* scores,
                       double correct_frac, cudaStream_t st, const unsigned int* colmax_pre = nullptr);

}  // namespace slso
