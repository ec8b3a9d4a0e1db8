/*
 * slso.h -- C ABI of the GB300 (sm_103a) Sketched Leverage Score Ordering library.
 *
 * Method: Chin & Liang, "An Empirical Evaluation of Sketched SVD and its Application to
 * Leverage Score Ordering" (ACML 2018).  Leverage scores (Sec. 2.2) of a tall data matrix
 * X (n x d) are approximated by sketch-and-solve (Algorithm 2, with the truncation of
 * Algorithm 3), and the scores induce the "dec" training order of Algorithm 4 / Sec. 5.2.
 *
 * Conventions shared by every entry point
 * ---------------------------------------
 * - Matrices are row-major.  X has n rows of d elements with leading dimension ldx >= d
 *   (elements, not bytes).  All array arguments are caller-owned DEVICE pointers unless
 *   the name ends in _host; the library never frees them or keeps them past the call.
 * - Work is enqueued asynchronously on `stream` (a cudaStream_t passed as void*; NULL is
 *   the legacy default stream).  Device outputs are valid once the stream has run.
 *   When a host `info` pointer is passed, the call synchronises `stream` before it
 *   returns so that `info` is filled; pass NULL to keep the call fully asynchronous.
 * - Scratch memory comes from the handle's own device pool (cudaMalloc, grown on demand
 *   and kept until slso_destroy).  A handle must be used by one host thread and one
 *   stream at a time.
 * - Every call returns an slso_status.  Argument, shape and dtype errors are detected
 *   on the host before anything is enqueued.  slso_last_error() returns a message for
 *   the calling thread's last failure.  No entry point throws or aborts.
 * - Random draws use Philox4x32-10 (Salmon et al., SC'11) keyed by the 64-bit seeds, with
 *   the counter layouts given beside each entry point; results depend only on the seeds,
 *   the inputs and the shapes, not on the GPU or the launch configuration.
 */
#ifndef SLSO_H
#define SLSO_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  SLSO_OK = 0,
  SLSO_ERR_INVALID_ARG = 1, /* NULL pointer, negative size, unknown enum value       */
  SLSO_ERR_SHAPE = 2,       /* sizes violate a shape rule (e.g. s < d)               */
  SLSO_ERR_DTYPE = 3,       /* dtype not supported for that argument                 */
  SLSO_ERR_OOM = 4,         /* the handle's device pool could not grow               */
  SLSO_ERR_CUDA = 5,        /* a CUDA runtime call failed (message has the detail)   */
  SLSO_ERR_NONFINITE = 6,   /* input held NaN or Inf (reported through slso_info)    */
  SLSO_ERR_TIMEOUT = 7,     /* a bounded device-side wait gave up                    */
  SLSO_ERR_BUSY = 8,        /* serving: no slot or memory free for the job           */
  SLSO_ERR_NOT_FOUND = 9,   /* serving: unknown ticket                               */
  SLSO_ERR_CANCELLED = 10   /* serving: the job was cancelled before it was admitted */
} slso_status;

typedef enum { SLSO_F64 = 0, SLSO_F32 = 1, SLSO_BF16 = 2, SLSO_FP8_E4M3 = 3 } slso_dtype;

/* Sketch families of Sec. 2.1 / Sec. 3.1.2, normalised so that E[S^T S] = I:
 *  COUNTSKETCH  S[h(i), i] = sign(i); h, sign from Philox counter (lo i, hi i, 0, 1):
 *               h = (w0 * s) >> 32, sign = 1 - 2 (w1 & 1).
 *  SRHT         sqrt(n_pad/s) P (H/sqrt(n_pad)) D on X zero-padded to n_pad = 2^ceil(log2 n)
 *               rows; D_i = 1 - 2 (w0 & 1) at counter (lo i, hi i, 0, 2); P keeps the s rows
 *               j with the smallest (w0 at counter (lo j, hi j, 0, 3), j), in ascending j.
 *  GAUSSIAN     (1/sqrt(s)) G, G_ji = bf16_rne(g) with four consecutive columns i sharing one
 *               Philox block: b = floor(i / 4), counter (lo b, hi b, j, 4); i mod 4 = 0, 1 take
 *               the cosine and sine normals of the Box-Muller pair (w0, w1), i mod 4 = 2, 3 those
 *               of (w2, w3); BoxMuller(w0, w1) = sqrt(-2 ln((w0+1) 2^-32)) cos(2 pi w1 2^-32) and
 *               the sine normal is the cosine of the angle word shifted by 2^30; the bf16
 *               rounding is decided on the float64 value. */
/* OSNAP (Sec. 3.1.2, a variant of CountSketch): z blocks of s/z rows, one +-1/sqrt(z) per block in
 * each column of S, bucket b s/z + ((w0 s/z) >> 32), sign 1 - 2 (w1 & 1) from Philox at counter
 * (lo i, hi i, b, 7); z = slso_params.nnz (0: 4); slso_sketch uses z = 4. */
typedef enum { SLSO_COUNTSKETCH = 0, SLSO_SRHT = 1, SLSO_GAUSSIAN = 2, SLSO_OSNAP = 3 } slso_sketch_kind;

/* Sampling policies of Algorithm 4 step 4 (Sec. 5.2) on P = scores / sum(scores). */
typedef enum { SLSO_POLICY_DEC = 0, SLSO_POLICY_SWR = 1, SLSO_POLICY_SWOR = 2 } slso_policy;

/* The factor R of SX (Algorithm 2/3 step 2).  With R_jj > 0 and SX of full column rank R is unique,
 * so both give the same R up to rounding.
 *  HOUSEHOLDER  unpivoted Householder QR of SX, float64 (orthogonality error ~ kappa(SX) u).
 *  AUTO         for compute != F64: the Gram route first, R = chol(SX^T SX), kept only when a
 *               check with 4 seeded Gaussian probes z (Philox at counter (lo c, hi c, q, 8))
 *               estimates ||R^-T SX^T SX R^-1 - I||_F <= 1e-8 (its error grows like kappa(SX)^2 u;
 *               the relative error of every score is at most that norm); otherwise, and always
 *               for compute = F64, Householder.  Decided on the device; slso_info reports it.
 *               G = SX^T SX comes from exact digit products on the tensor cores (slso_gram; a
 *               float-float SYRK on the float32 pipe where the tensor route does not apply), and
 *               the Cholesky factor, R^-1, M = R^-1 Pi and the probe check are computed in
 *               float-float arithmetic (pairs of float32 values, ~2^-48).  Its scratch (the digit slices of SX, 16 dpad s bytes, or the float32
 *               split, 8 s d bytes, plus O(d^2)) is taken whether or not the route stands;
 *               slso_workspace_size includes it. */
typedef enum { SLSO_FACTOR_AUTO = 0, SLSO_FACTOR_HOUSEHOLDER = 1 } slso_factor;

typedef struct slso_handle slso_handle;

typedef struct {
  int32_t kind;        /* slso_sketch_kind                                                   */
  int32_t compute;     /* dtype of the X.M contraction: F64, F32 (3xTF32-accurate), BF16, FP8 */
  int64_t s;           /* sketch rows, d <= s (SRHT: s <= n_pad)                             */
  int64_t k;           /* JL width; 0 means Pi = I (Algorithm 3 exactly); k <= 4096           */
  uint64_t seed_S;     /* seed of the sketch S                                                */
  uint64_t seed_Pi;    /* seed of Pi: Pi_jc = BoxMuller(w0, w1)/sqrt(k) at counter
                          (lo c, hi c, j, 5)                                                  */
  double tau;          /* relative rank threshold: keep sigma_j > tau sigma_1; < 0 selects
                          max(s, d) 2^-52 (float64 numerical rank)                            */
  double correct_frac; /* BF16/FP8 only: rescore the top ceil(frac n) rows in float32; 0 = off */
  int32_t nnz;         /* OSNAP: nonzeros per column of S (1..64, s divisible by it); 0 = 4     */
  int32_t factor;      /* how R of SX is formed: SLSO_FACTOR_AUTO or SLSO_FACTOR_HOUSEHOLDER    */
} slso_params;

typedef struct {
  int64_t rank;          /* numerical rank r of SX (Algorithm 3 step 3)                       */
  double sigma_max;      /* sigma_1(SX); NaN when the certified full-rank route was taken     */
  double sigma_min_kept; /* sigma_r(SX); NaN on the certified route                          */
  double score_sum;      /* sum of the returned scores (normaliser of P, Algorithm 4 step 3)  */
  double tau;            /* the threshold actually used                                       */
  int32_t nonfinite;     /* 1 if X held NaN or Inf                                            */
  int32_t svd_route;     /* 1: R^+ from the SVD of R; 0: rank d certified, R^+ = R^-1          */
  int32_t svd_sweeps;    /* float64 one-sided Jacobi sweeps of the SVD of R (after the float32
                            preconditioning sweeps when d >= 64); 0 when it did not run          */
  int32_t gram_route;    /* 1: R from the Gram route; 0: Householder QR                          */
  double gram_resid;     /* the Gram route's probe estimate of ||R^-T SX^T SX R^-1 - I||_F; NaN
                            when its Cholesky broke down or the route was not tried              */
} slso_info;

/* Library / handle ------------------------------------------------------------------ */
const char* slso_version(void);
const char* slso_last_error(void);
slso_status slso_create(slso_handle** handle, int device);
slso_status slso_destroy(slso_handle* handle);
/* Device bytes the handle's pool needs for slso_leverage + slso_order on these shapes. */
slso_status slso_workspace_size(const slso_params* params, int64_t n, int64_t d, size_t* bytes);

/* Sketch SX = S X  (Algorithm 2/3 step 1; Sec. 2.1 definition of the sketches).
 * X: n x d (ldx) of dtype xdt in {F64, F32, BF16}.  SX: s x d float64, row-major, dense.
 * CountSketch sums each bucket's rows in ascending row order with compensated float32
 * (float64 for F64 X); SRHT and Gaussian accumulate partial sums in float32 (float64
 * for F64 X) merged in float64 in a fixed order, so the result is deterministic.
 * Errors: SHAPE if n < 1, d < 1, s < 1, ldx < d, (SRHT) s > n_pad, or (OSNAP, z = 4) s not a
 * multiple of 4. */
slso_status slso_sketch(slso_handle* handle, const void* X, int64_t n, int64_t d, int64_t ldx,
                        int32_t xdt, int32_t kind, int64_t s, uint64_t seed_S, double* SX,
                        void* stream);

/* Sketched SVD (title; Algorithm 2/3 steps 2-3): unpivoted Householder QR of SX (s x d,
 * float64, s >= d) with R_jj >= 0, then the SVD of R by one-sided Jacobi.  For d >= 64 float32
 * sweeps on float32(R) first give a basis V32; Q = V32 (V32^T V32)^(-1/2) (series, float64) and
 * the float64 sweeps run on R Q with V starting at Q, so the result is float64-accurate:
 * sigma (d, descending) are the singular values of SX and V (d x d, row-major, column j
 * the j-th right singular vector) its right singular vectors.  R (d x d) is written when
 * non-NULL.  rank = #{sigma_j > tau sigma_1} (tau < 0: max(s, d) 2^-52) goes to info.
 * Householder step j: no reflection when the subcolumn below the diagonal is exactly 0;
 * otherwise beta = -sign(alpha) ||A[j:, j]|| with sign(+-0) = +1. */
slso_status slso_sketched_svd(slso_handle* handle, const double* SX, int64_t s, int64_t d,
                              double tau, double* sigma, double* V, double* R, slso_info* info,
                              void* stream);

/* Gram matrix G = SX^T SX (d x d float64, row-major, symmetric) as the float32 compute path's
 * Gram route forms it for R (R^T R = G at full column rank; Algorithm 2/3 step 2).  Each column j
 * of SX (s x d float64, row-major, s >= 1) is scaled by 2^-e_j, its largest entry then in [1/2, 1),
 * rounded to 55 fractional bits and cut into eight signed 7-bit digits; the 36 digit products of
 * order <= 7 run on the tensor cores (bfloat16, float32 accumulation, one accumulator per order) in
 * 512-row windows in which every partial sum is an exact integer, and the windows are added as
 * exact int64 sums, so G is deterministic and, for integer-valued columns with at most 55
 * significant bits below their scale, exact.  Where the tensor route does not apply (s >= 2^20) a
 * float-float SYRK on the float32 pipe forms G instead.  SX, G: caller-owned device memory;
 * asynchronous on stream.
 * Errors: SHAPE unless 1 <= d <= 24576 and 1 <= s < 2^31; INVALID_ARG for NULL pointers. */
slso_status slso_gram(slso_handle* handle, const double* SX, int64_t s, int64_t d, double* G, void* stream);

/* Approximate leverage scores (Algorithm 3 with the JL projection Pi):
 *   SX = S X;  R = householder_R(SX);  r = #{sigma_j(R) > tau sigma_1};
 *   M = R^+_tau Pi = V_r Sigma_r^-1 U_R,r^T Pi  (Pi = I when k = 0);
 *   scores_i = ||x_i M||^2.
 * With params->factor = SLSO_FACTOR_AUTO and compute != F64, R is first taken as the Cholesky
 * factor of SX^T SX (the same R at full column rank); it stands only when its probe check
 * passes, else the Householder R is computed instead (slso_factor; info->gram_route and
 * info->gram_resid report which).
 * When ||R||_F ||R^-1||_F < 1e-3 / tau the rank is certified to be d and R^+_tau = R^-1
 * exactly, so the SVD is skipped (info->svd_route = 0).  scores: n values, float64 when
 * compute == F64, else float32.  compute F32 evaluates X.M to float32 accuracy on the
 * tensor cores (three TF32 products); BF16 and FP8 round X and M (FP8 with per-column
 * scales of X folded into M) and accumulate in float32.
 * Errors: SHAPE as for slso_sketch plus k > 4096 or s < d; DTYPE for an unsupported
 * (xdt, compute) pair; INVALID_ARG for an unknown factor. */
slso_status slso_leverage(slso_handle* handle, const void* X, int64_t n, int64_t d, int64_t ldx,
                          int32_t xdt, const slso_params* params, void* scores, slso_info* info,
                          void* stream);

/* Approximate left singular vectors (Algorithm 2 step 3; Algorithm 3 step 4, read without
 * the transpose): sketch SX = S X (params: kind, s, seed_S, tau; k, seed_Pi, compute and
 * correct_frac are not used), sketched SVD SX = U' Sigma V^T (float64 QR + Jacobi SVD of R),
 * r = #{sigma_j > tau sigma_1}, then U = X V_r Sigma_r^-1 (tensor cores, float32-accurate split
 * operands, for F32 / BF16 X; float64 for F64 X).  U is n x d row-major with leading
 * dimension ldu >= d, float64 for F64 X, float32 otherwise; columns r .. d-1 are zero.  Column j
 * is defined up to the sign of the singular vector v_j (as for any SVD).  ||U_i||^2 is row i's
 * score of slso_leverage with k = 0.  Errors as slso_leverage, plus SHAPE for ldu < d. */
slso_status slso_approx_u(slso_handle* handle, const void* X, int64_t n, int64_t d, int64_t ldx,
                          int32_t xdt, const slso_params* params, void* U, int64_t ldu, slso_info* info,
                          void* stream);

/* Policy "dec" of Sec. 5.2 (Algorithm 4 step 4): order[0..n) lists row indices by strictly
 * decreasing score; equal scores (with -0 == +0) by increasing index; NaN last.  A stable
 * LSD radix argsort on the 32-bit (F32 scores) or 64-bit (F64 scores) orderable key. */
slso_status slso_order(slso_handle* handle, const void* scores, int32_t sdt, int64_t n,
                       int64_t* order, void* stream);

/* The end-to-end call of slso_rank_rows_host for `count` host matrices of the same shape and
 * type (X_host[i], scores_host[i], order_host[i]; info[i] when info is non-NULL), pipelined:
 * item i+1's host-to-device copy and item i-1's device-to-host copies run on two internal
 * streams while item i computes on `stream`, with two device buffers for X and for the
 * outputs.  Every kernel runs on `stream`, in item order.  Synchronous: returns when every
 * output is in host memory.  Host buffers should be pinned for the copies to overlap.
 * Errors: as slso_rank_rows_host, checked for every item before anything is launched; a
 * device-side condition (timeout, non-finite X) is reported for the first item it hit, after
 * every item has run. */
slso_status slso_rank_rows_host_batch(slso_handle* handle, int64_t count, const void* const* X_host,
                                      int64_t n, int64_t d, int64_t ldx, int32_t xdt,
                                      const slso_params* params, void* const* scores_host,
                                      int64_t* const* order_host, slso_info* info, void* stream);

/* Out-of-core X: slso_rank_rows_host for a HOST matrix that need not fit in device memory.  X is
 * streamed through the device twice in blocks of rows.  Pass 1 copies each block in and adds its
 * sketch to SX; the hash, sign and Gaussian counters use the rows' indices in the whole X, so SX
 * equals slso_sketch's up to the float64 rounding of the block sums.  The solve runs once.  Pass 2
 * copies the blocks in again, last block first (the two blocks still on the device are not copied
 * again), and scores them.  Copies run on a stream of the call's own, overlapped with the compute
 * of the neighbouring block.
 *   X_host       n x d host matrix, row stride ldx (pinned memory lets the copies overlap compute)
 *   block_rows   rows per block: at least 65536, rounded down to a power of two (0: 262144)
 *   scores_host  n scores, F64 when params->compute == SLSO_F64, else F32; order_host n int64
 * Device memory: two blocks (block_rows x d elements each), SX, and O(n) for the scores and the
 * order, plus scratch; independent of n x d.
 * params->correct_frac must be 0 (a correction pass would need a third pass over X).  With compute
 * FP8 the per-column scales are taken per block.
 * Errors: as slso_rank_rows_host; INVALID_ARG for correct_frac != 0 or block_rows < 0.
 * Synchronous: returns after the copies out have finished. */
slso_status slso_rank_rows_streamed(slso_handle* handle, const void* X_host, int64_t n, int64_t d,
                                    int64_t ldx, int32_t xdt, const slso_params* params,
                                    int64_t block_rows, void* scores_host, int64_t* order_host,
                                    slso_info* info, void* stream);

/* Orderings of Algorithm 4 step 4 (Sec. 5.2) from the scores (device, F32 or F64, n of
 * them) into order[0..n) (device, int64), on the given stream; seed selects the draws (one
 * seed per training epoch).  Weights are the scores; NaN, infinite or negative scores weigh 0.
 *   SLSO_POLICY_DEC   the "dec" order, exactly as slso_order (seed unused).
 *   SLSO_POLICY_SWOR  "dec, swor": the order of n successive draws without replacement, each
 *                     point drawn with probability proportional to its score among those not
 *                     yet drawn (Efraimidis-Spirakis keys log(u_i)/l_i sorted decreasingly).
 *                     Weight-0 points follow all others in increasing index, NaN scores last.
 *   SLSO_POLICY_SWR   "dec, swr": n draws with replacement, in draw order: draw t is the
 *                     smallest i whose cumulative score exceeds u_t times the total (points
 *                     can repeat).  When no score is positive and finite every entry is -1.
 * u_t = (m + 1/2) 2^-52, m = w0 2^20 + (w1 >> 12) from Philox4x32-10 at counter
 * (lo t, hi t, 0, 6) with key seed.  Scratch from the handle's pool.
 * Errors: INVALID_ARG (NULL pointers, unknown policy), SHAPE (n < 1 or n >= 2^31), DTYPE. */
slso_status slso_sample_order(slso_handle* handle, const void* scores, int32_t sdt, int64_t n,
                              int32_t policy, uint64_t seed, int64_t* order, void* stream);

/* End-to-end call with HOST buffers: copies X_host (pinned or pageable) to the device,
 * runs slso_leverage + slso_order, copies scores (float32, or float64 for F64 compute)
 * and order back.  Synchronous.  Device buffers come from the handle's pool. */
slso_status slso_rank_rows_host(slso_handle* handle, const void* X_host, int64_t n, int64_t d,
                                int64_t ldx, int32_t xdt, const slso_params* params,
                                void* scores_host, int64_t* order_host, slso_info* info,
                                void* stream);

/* Serving: continuous batching of leverage-score and sketched-SVD jobs ----------------------
 * A server owns `slots` CUDA streams on one device and a worker thread.  slso_server_submit
 * queues a job without blocking; the worker admits queued jobs in arrival order whenever a slot
 * is free and the job's scratch footprint (exactly what slso_workspace_size would report for
 * it) fits in `mem_budget_bytes` beside the jobs already running.  Admitted jobs run
 * concurrently, each on its own stream with stream-ordered scratch; jobs that arrive while
 * others run are admitted as slots and memory free up.  Results are identical to running the
 * job alone with slso_leverage (+ slso_order) or slso_sketched_svd.  All device pointers in a
 * job stay owned by the caller and must stay valid until the job has been polled. */
typedef struct slso_server slso_server;
typedef enum { SLSO_JOB_LEVERAGE = 0, SLSO_JOB_SKETCHED_SVD = 1 } slso_job_kind;
typedef struct {
  int32_t job;          /* slso_job_kind                                                        */
  int32_t xdt;          /* leverage: dtype of X                                                  */
  const void* X;        /* leverage: X (n x d, ldx); sketched SVD: SX (n = s rows x d, float64)  */
  int64_t n, d, ldx;
  slso_params params;   /* leverage: all fields; sketched SVD: only tau is read                  */
  void* scores;         /* leverage: n scores (float64 when compute == F64, else float32)        */
  int64_t* order;       /* leverage: n row indices in "dec" order, or NULL                       */
  double* sigma;        /* sketched SVD: d singular values, V (d x d), R (d x d or NULL)         */
  double* V;
  double* R;
} slso_job;

/* slots in [1, 64]; the budget bounds the summed scratch of running jobs. */
slso_status slso_server_create(slso_server** server, int device, int slots, size_t mem_budget_bytes);
/* Waits for running jobs; jobs still queued finish with SLSO_ERR_BUSY.  Unpolled results are freed. */
slso_status slso_server_destroy(slso_server* server);
/* Validates the job (same errors as the direct entry points) and queues it.  BUSY when the
 * job alone needs more scratch than the whole budget, or the server is shutting down. */
slso_status slso_server_submit(slso_server* server, const slso_job* job, int64_t* ticket);
/* Waits up to timeout_ms for the job.  Returns TIMEOUT if it is not finished (poll again),
 * NOT_FOUND for an unknown or already collected ticket; otherwise OK with the job's own status,
 * its info, and times_ms[0..2] = {queued, admitted to done, submit to done} when non-NULL.
 * A finished job is forgotten once polled. */
slso_status slso_server_poll(slso_server* server, int64_t ticket, int timeout_ms, slso_status* job_status,
                             slso_info* info, double* times_ms);
/* Cancels a job that is still queued (not yet admitted): it finishes with SLSO_ERR_CANCELLED,
 * which slso_server_poll reports.  BUSY when the job is already running or finished,
 * NOT_FOUND for an unknown or collected ticket. */
slso_status slso_server_cancel(slso_server* server, int64_t ticket);
/* counters[0..3] = {submitted, admitted, completed, queued}; bytes of scratch in use. */
slso_status slso_server_stats(slso_server* server, int64_t* counters, size_t* mem_in_use);
/* The first `count` of {submitted, admitted, completed, queued, scratch bytes in use, graphs
 * instantiated, graphs updated in place, leverage jobs run without a graph, grouped score
 * launches, jobs run in them} (zeros beyond).
 * From the second job of a shape (n, d, ldx, dtype, params, order or not) on, leverage jobs are
 * recorded into CUDA graphs by stream capture; each slot keeps the graphs of its 8 most recent
 * shapes with their workspace, within a quarter of the memory budget, and a job of a cached
 * shape updates that graph's arguments in place and replays it.
 * Grouped launches: when a slot frees up and the queue's head is a small leverage job (float32 X
 * and compute, 1 <= k <= 128, d <= 2048, n <= 2^17, 16-byte aligned rows, no correction pass), up
 * to 8 consecutive queued jobs of that kind with the same JL width (k rounded up to 32) that fit
 * the budget are admitted together: each job's sketch and solve run on the slot's stream, then
 * one persistent tensor-core launch computes all their scores from device-side job descriptors
 * (each row exactly as the job's own launch computes it), then each job's score sum and order. */
slso_status slso_server_counters(slso_server* server, int64_t* counters, int32_t count);

/* Ordering that allocates nothing (the paper has no counterpart; this exists for callers).
 * Some callers cannot call cudaMalloc where they need an ordering: a process whose device
 * memory is entirely owned by another framework's caching allocator, a service that forbids
 * allocation after start-up so that its footprint and latency stay fixed, or code running
 * while someone else records a CUDA graph.  slso_order_static computes exactly what slso_order
 * computes, takes no handle, and uses as scratch one file-scope __device__ array sized for
 * n <= 1048576 (2^20) scores, about 24.3 MB that every GPU loading the library keeps until the
 * process exits.  scores: n values of dtype sdt (F32 or F64) on the current device; order: n
 * int64 row indices.  Errors: SHAPE for n < 1 or n > 2^20, DTYPE, INVALID_ARG for NULL
 * pointers.  The first call on each device looks up the array's device address (with that
 * device current); make that first call before any stream capture.  All calls share the one
 * array, so calls that can overlap on the GPU (different streams, no ordering between them)
 * race and must be serialised by the caller; nothing in the array needs to start at zero. */
slso_status slso_order_static(const void* scores, int32_t sdt, int64_t n, int64_t* order, void* stream);

/* Caps the handle's device pool at `bytes` (0: no cap).  A call whose scratch would need more
 * fails with SLSO_ERR_OOM before launching anything, as a real allocation failure does; lowering
 * the cap below the current pool frees nothing until the pool next grows.  Used to give a
 * caller a fixed footprint and to exercise allocation-failure paths. */
slso_status slso_set_pool_limit(slso_handle* handle, size_t bytes);

/* Operand form of the float32 score product X M (Algorithm 3 step 4) for k <= 128 on the tensor
 * cores (float32 X, compute SLSO_F32).  X = Xhi + Xlo and M = Mhi + Mlo with tf32 high parts;
 * all forms accumulate in float32 and keep Y = X M on the SM.
 *   SLSO_SCORE_FORM_MIXED (default): Xhi Mhi in tf32 plus bf16(Xlo) bf16(Mhi) + bf16(Xhi)
 *     bf16(Mlo) in bfloat16, X's pieces in tensor memory; every rounded or dropped term is below
 *     2^-18 |x_il m_lj|.
 *   SLSO_SCORE_FORM_TF32X3: Xhi Mhi + Xhi Mlo + Xlo Mhi in tf32, X's pieces in tensor memory
 *     (below 2^-21 |x_il m_lj|).
 *   SLSO_SCORE_FORM_TF32X3_SMEM: the same products with X's pieces in shared memory.
 * The choice holds for later calls on the handle; other shapes and precisions ignore it.
 * Unknown forms: SLSO_ERR_INVALID_ARG. */
#define SLSO_SCORE_FORM_MIXED 0
#define SLSO_SCORE_FORM_TF32X3 1
#define SLSO_SCORE_FORM_TF32X3_SMEM 2
slso_status slso_set_score_form(slso_handle* handle, int32_t form);

/* Self-test of the bounded device-side waits every kernel relies on (no GPU fault involved):
 * what = 0 runs the ready-flag wait of the QR on a flag that nothing sets, what = 1 the
 * mbarrier wait of the tensor-core kernels on a barrier that nothing completes, each limited to
 * about limit_us microseconds (1 .. 10^7).  The expected outcome is SLSO_ERR_TIMEOUT after the
 * limit, with the CUDA context still usable; SLSO_OK would mean the wait did not run out. */
slso_status slso_selftest_wait(slso_handle* handle, int32_t what, int64_t limit_us, void* stream);

/* Instrumentation (no counterpart in the paper).  slso_profile(h, 1) resets and starts
 * recording a CUDA event pair around every stage each call enqueues on its stream:
 * 0 sketch, 1 Householder QR, 2 rest of the small solve (certificate, R^-1 or SVD, M),
 * 3 scores (X.M + row norms), 4 ordering, 5 host<->device copies, 6 the Gram route's SYRK
 * (G = SX^T SX), 7 the rest of the Gram route (Cholesky, R^-1, probe check).  A stage may be
 * recorded more than once per call (calls counts records, not calls of the API).
 * slso_profile_read waits for the recorded events and returns per-stage milliseconds and record
 * counts (arrays of SLSO_STAGES) and the number of kernels this library launched (in this
 * process) since slso_profile was called.  Recording stops after 4096 stages. */
#define SLSO_STAGES 8
slso_status slso_profile(slso_handle* handle, int enable);
slso_status slso_profile_read(slso_handle* handle, double* stage_ms, int64_t* stage_calls,
                              int64_t* launches);

#ifdef __cplusplus
}
#endif

#endif /* SLSO_H */
