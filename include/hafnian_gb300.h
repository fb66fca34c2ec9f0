/*
 * hafnian_gb300.h -- C ABI of the GB300 (sm_103a) hafnian / loop-hafnian
 * library.
 *
 * What is computed.  For an n x n complex (or real) symmetric matrix A:
 *   haf(A)  = sum over perfect matchings M of prod_{(i,j) in M} A_ij
 *             (Sec. 2, eq. hafA);
 *   lhaf(A) = the same sum over single-pair matchings, in which a vertex may
 *             also be matched to itself with weight A_ii (Sec. 2, lhaf
 *             definition).
 * Both are evaluated with the signed subset sum of Sec. 3.2 (eq. main):
 *   haf(A) = sum_{Z subset of the n/2 pairs} (-1)^{n/2-|Z|} f(Z),
 * where f(Z) is the lambda^{n/2} coefficient of the trace generating
 * function of Sec. 3.3 (eq. poly, eq. haffinal; for lhaf the q(lambda,B,v)
 * function).  The library obtains f(Z) = [lambda^{n/2}] det(I - lambda B)^{-1/2}
 * (times the exponential of the loop series for lhaf) from a Householder
 * Hessenberg reduction of B = (X A)^{(Z)}, the La Budde recurrence for the
 * characteristic polynomial and a truncated power-series recurrence; this
 * equals the paper's Schur/power-trace route in exact arithmetic (App. B).
 *
 * Input conventions (all entry points).
 *   - A is row-major n x n.  Complex matrices are interleaved (re, im)
 *     doubles, i.e. C99 double _Complex / numpy complex128 layout.
 *   - Off-diagonal entries are read from the upper triangle only (i < j);
 *     the lower triangle is never read (App. C: haf(A) = haf(A + L) for
 *     lower-triangular L).  haf ignores the diagonal; lhaf reads it.
 *   - n = 0 gives 1.  Odd n: haf = 0; lhaf pads A with one isolated vertex
 *     of loop weight 1 (which leaves the single-pair-matching sum unchanged).
 *   - Supported sizes: 0 <= n <= HAF_MAX_N.
 *   - Pointers are owned by the caller.  Host-pointer entry points copy A to
 *     the device themselves and return when the result is on the host.
 *
 * Results.  The signed subset sum is accumulated in double-double
 * (compensated) arithmetic and reduced in a fixed order, so a result is
 * bit-reproducible from run to run.  Alongside the value the library
 * reports abs_sum = sum_Z |f(Z)|; the absolute error is bounded in practice
 * by a small multiple of 1e-16 * abs_sum (the accuracy contract used by the
 * tests is |error| <= 1e-10 * abs_sum).
 *
 * Errors.  Every entry point returns HAF_OK (0) or a negative HAF_E* code
 * and never throws across the ABI.  On error the outputs are left untouched,
 * except for HAF_EACCURACY (FP32-bulk mode, below), which writes the value
 * and the report so that the caller can inspect them.  haf_last_error()
 * returns a short text for the calling thread's last error.
 */
#ifndef HAFNIAN_GB300_H
#define HAFNIAN_GB300_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define HAF_MAX_N 56

/* status codes */
#define HAF_OK 0
#define HAF_EINVAL (-1)    /* bad argument (null pointer, n out of range, bad flags) */
#define HAF_ENOMEM (-2)    /* device or host allocation failed                     */
#define HAF_ECUDA (-3)     /* a CUDA runtime call failed                           */
#define HAF_ETIMEDOUT (-4) /* server poll gave up before the job finished          */
#define HAF_EBUSY (-5)     /* server refused a job (queue full)                    */
#define HAF_ENOTFOUND (-6) /* server: unknown (or already collected) ticket        */
#define HAF_ESMALL (-7)    /* caller-supplied workspace too small                  */
#define HAF_EACCURACY (-8) /* FP32-bulk result above the stated relative error      */

/* flags */
#define HAF_FLAG_LOOPS (1u << 0) /* loop hafnian                                 */
#define HAF_FLAG_REAL (1u << 1)  /* A is real float64, not complex128           */
#define HAF_FLAG_FP32 (1u << 2)  /* FP32-bulk precision mode (see below)         */

/* Accuracy.  The signed subset sum cancels: |value| is often many orders
 * of magnitude below abs_sum = sum_Z |f(Z)|, so an error that is small
 * against abs_sum can be large against the value.  Each whole-matrix call
 * therefore reports rel_err_bound = REL_TOL * abs_sum / |value|, an
 * estimate of |error| / |value| from the measured error against the
 * binary128 oracle, where REL_TOL is
 *   HAF_FP64_REL_TOL for FP64 (measured errors up to 1.2e-14 * abs_sum), or
 *   HAF_FP32_REL_TOL for the FP32-bulk mode.
 *
 * FP32-bulk precision mode.  With HAF_FLAG_FP32 the gather of B, the
 * Householder reduction, the loop moments and La Budde's recurrence run in
 * single precision (complex64 / float32) while the power series, f(Z) and
 * the double-double subset sum stay FP64 (Sec. 4 finds that the precision of
 * the eigenvalue step dominates the error; this mode trades it for speed).
 * Its error measured against FP64 over complex and real Gaussian, GBS and
 * all-ones inputs at n = 2..40 (haf and lhaf) stayed below 1.2e-5 * abs_sum;
 * HAF_FP32_REL_TOL = 3e-5 is that bound with a margin.  It is an empirical
 * bound: a summand whose loop terms cancel internally can exceed it.  A
 * whole-matrix call in this mode is gated on the value: when rel_err_bound
 * exceeds HAF_FP32_MAX_REL_ERR it returns HAF_EACCURACY (the value and the
 * report are still written; recompute without HAF_FLAG_FP32 for a result in
 * FP64).  The gate admits inputs with abs_sum / |value| <= 33: in practice
 * random Gaussian or GBS matrices up to n of about 8-10; larger inputs with
 * heavy cancellation are refused.  The device-pointer form haf_launch
 * and the part records of haf_part are not gated (their value is on the
 * device, or is only a part of the sum). */
#define HAF_FP32_MAX_N 56
#define HAF_FP64_REL_TOL 1e-13
#define HAF_FP32_REL_TOL 3e-5
#define HAF_FP32_MAX_REL_ERR 1e-3

/* Per-call report. */
typedef struct haf_info {
  double abs_sum;        /* sum over subsets Z of |f(Z)|                       */
  double value_lo[2];    /* low parts of the double-double result (re, im)     */
  int64_t subsets;       /* number of subset terms evaluated (2^{n/2} - 1)     */
  double seconds;        /* wall time of the call (host clock)                 */
  int64_t launches;      /* CUDA kernels launched by the call                  */
  double rel_err_bound;  /* estimated |error| / |value| (see Accuracy); 0 where
                            not computed (parts, the low-rank path)            */
  int32_t precision_mode; /* 0: FP64, 1: FP32-bulk                             */
  int32_t reserved;
} haf_info;

/* ------------------------------------------------------------------------
 * Single matrix, host pointers, synchronous.
 *   A   : n*n complex128 (haf_c128, lhaf_c128) or float64 (haf_f64, lhaf_f64)
 *   out : 2 doubles (re, im) for the complex forms, 1 double for the real.
 *   info: may be NULL.
 * Passage: Sec. 3.2 eq. main with the summand of Sec. 3.3 (eq. haffinal and
 * its loop-hafnian analogue).
 * ---------------------------------------------------------------------- */
int haf_c128(const double* A, int64_t n, double* out, haf_info* info);
int lhaf_c128(const double* A, int64_t n, double* out, haf_info* info);
int haf_f64(const double* A, int64_t n, double* out, haf_info* info);
int lhaf_f64(const double* A, int64_t n, double* out, haf_info* info);
/* The same with flags: HAF_FLAG_LOOPS (lhaf), HAF_FLAG_REAL (A float64,
 * out 1 double), HAF_FLAG_FP32 (precision mode above).  Unknown flags:
 * HAF_EINVAL. */
int haf_eval(const double* A, int64_t n, uint32_t flags, double* out, haf_info* info);

/* ------------------------------------------------------------------------
 * Batched: `count` independent matrices of possibly different sizes run in
 * one persistent launch (host pointers, synchronous).
 *   As[i]  : matrix i (n = ns[i]); complex128.
 *   outs   : 2*count doubles; infos: count entries or NULL.
 * Passage: eq. main applied to each matrix.
 * ---------------------------------------------------------------------- */
int haf_c128_batched(const double* const* As, const int64_t* ns, int64_t count, double* outs,
                     haf_info* infos);
int lhaf_c128_batched(const double* const* As, const int64_t* ns, int64_t count, double* outs,
                      haf_info* infos);
/* The same with flags: HAF_FLAG_LOOPS, HAF_FLAG_FP32 (complex128 input only;
 * HAF_FLAG_REAL is rejected). */
int haf_batched(const double* const* As, const int64_t* ns, int64_t count, uint32_t flags, double* outs,
                haf_info* infos);

/* ------------------------------------------------------------------------
 * Sharding one matrix over several GPUs or processes (the subset sum splits
 * into independent ranges with one final sum, Sec. 4.1).  Part p of P takes,
 * for every subset size m, the p-th of P contiguous, nearly equal slices of
 * the colex-ordered m-subsets; the slices depend only on (n, p, P), so
 * processes on different machines agree on them.
 *   haf_part        : A on the host (complex128, or float64 with HAF_FLAG_REAL;
 *                     HAF_FLAG_LOOPS for lhaf); writes the part's record
 *                     rec[5] = {re_hi, im_hi, re_lo, im_lo, abs_sum}.  Runs
 *                     on the calling thread's current CUDA device.
 *   haf_part_subsets: number of subset terms part p evaluates (host only).
 *   haf_combine     : host-only fixed-order double-double sum of `nparts`
 *                     records (recs[5*nparts]) into out[5]; the value is
 *                     (out[0] + out[2]) + i (out[1] + out[3]).
 * n = 0 and odd n follow the whole-matrix conventions (value in part 0).
 * Returns HAF_EINVAL unless 0 <= part < nparts.
 * ---------------------------------------------------------------------- */
int haf_part(const double* A, int64_t n, uint32_t flags, int64_t part, int64_t nparts, double* rec,
             haf_info* info);
int haf_part_subsets(int64_t n, int64_t part, int64_t nparts, int64_t* subsets);
int haf_combine(const double* recs, int64_t nparts, double* out);

/* ------------------------------------------------------------------------
 * Device-resident asynchronous form (for callers that own device memory and
 * streams, e.g. through PyTorch).
 *   dA        : device pointer, n*n complex128 (or float64 with HAF_FLAG_REAL)
 *   d_out     : device pointer to 5 doubles written as
 *               {re_hi, im_hi, re_lo, im_lo, abs_sum}
 *   d_work    : device workspace of at least haf_workspace_bytes(n, flags)
 *               bytes, 256-byte aligned, not shared with a concurrent call
 *   stream    : cudaStream_t (NULL = legacy default stream)
 * The call only enqueues work; it returns before the result is ready.
 * Returns HAF_ESMALL if ws_bytes is too small.  n must be even, 2..HAF_MAX_N
 * (the host entry points handle 0 and odd n).
 * ---------------------------------------------------------------------- */
size_t haf_workspace_bytes(int64_t n, uint32_t flags);
int haf_launch(const double* dA, int64_t n, uint32_t flags, double* d_out, void* d_work,
               size_t ws_bytes, void* stream);

/* ------------------------------------------------------------------------
 * Allocation-free form of haf_launch.  The paper has no counterpart: this
 * is a deployment variant for callers that may not allocate device memory
 * when they ask for a hafnian -- code running under a caching allocator or
 * memory pool that owns the device's memory, callbacks and plug-ins that may
 * not call cudaMalloc/cudaFree (both synchronise the whole device), and
 * services that must not grow their device footprint after start-up.
 *
 * It computes the same value as haf_launch (same kernels; the subset sum is
 * chunked differently, so the last bits can differ) and calls no cudaMalloc,
 * cudaFree or other allocating routine.  Its scratch lives in one static
 * device array of HAF_NOALLOC_SCRATCH_BYTES, which every GPU that loads the
 * library holds until the process exits.
 *   dA    : device pointer, n*n complex128 (float64 with HAF_FLAG_REAL)
 *   d_out : device pointer to 5 doubles {re_hi, im_hi, re_lo, im_lo, abs_sum}
 *   stream: cudaStream_t (NULL = legacy default stream); the call enqueues
 *           work and returns before the result is ready.
 * n must be even with 2 <= n <= HAF_MAX_N; anything else returns HAF_EINVAL
 * with a message.  The first call on a device looks up the array's device
 * address and sets kernel attributes; with CUDA's lazy module loading (the
 * default) it is also the call that loads the library's device code and
 * reserves the array, which takes device memory.  Make that first call at
 * start-up, before any stream capture and before a memory pool claims the
 * device's memory.  The call plans with the launch shape that haf_launch
 * uses for the same n and flags (haf_tune / haf_tune_set, else the default).  All calls share the one array: calls whose work overlaps on the
 * GPU (e.g. on two unordered streams) race and corrupt each other's results,
 * so order them on one stream or synchronise between them.
 * ---------------------------------------------------------------------- */
#define HAF_NOALLOC_SCRATCH_BYTES (1u << 20)
int haf_launch_noalloc(const double* dA, int64_t n, uint32_t flags, double* d_out, void* stream);

/* ------------------------------------------------------------------------
 * Per-subset summands (for sampling checks at large n).
 *   masks[i] : subset Z as a bitmask over the n/2 pairs (bit p <=> pair
 *              (2p, 2p+1) in Z); host array of `count` entries.
 *   terms    : 2*count doubles (host), receives f(Z) WITHOUT the sign
 *              (-1)^{n/2-|Z|}.
 *   loops    : 0 for the haf summand, 1 for the lhaf summand.
 * Passage: the summand of eq. haffinal (Sec. 3.3).
 * ---------------------------------------------------------------------- */
int haf_terms_c128(const double* A, int64_t n, int loops, const uint64_t* masks, int64_t count,
                   double* terms);
/* The same with flags (HAF_FLAG_LOOPS, HAF_FLAG_FP32; complex128 input). */
int haf_terms(const double* A, int64_t n, uint32_t flags, const uint64_t* masks, int64_t count,
              double* terms);

/* ------------------------------------------------------------------------
 * Low-rank hafnian (App. C): haf(G G^T) for G with n rows and r columns
 * (complex128, row-major n x r, owned by the caller), in time
 * ~ C(n+r-1, r-1) * r^2 instead of 2^{n/2}.  The coefficients lambda_e of
 * q(x) = prod_i sum_j g_ij x_j (eq. q) are expanded row by row on the GPU
 * and combined as sum over even e of lambda_e prod_j (e_j - 1)!!.  Only the
 * entries of G G^T above the diagonal matter (App. C: haf(A) = haf(A + L)),
 * so any G with G G^T = A + L (L lower triangular) gives haf(A).
 *   out  : 2 doubles (re, im); info (may be NULL): abs_sum is the same
 *          expansion with |g_ij| (a bound on every summand; the absolute
 *          error is a small multiple of 1e-16 n * abs_sum), subsets = number
 *          of monomials of degree n, C(n+r-1, r-1).
 * n = 0 gives 1, odd n gives 0.  HAF_EINVAL unless 0 <= n <=
 * HAF_LOWRANK_MAX_N and 1 <= r <= HAF_LOWRANK_MAX_R; HAF_ENOMEM if the two
 * degree-n coefficient arrays (48 bytes per monomial in all) do not fit the
 * free device memory.  Synchronous; uses the current device.
 * ---------------------------------------------------------------------- */
#define HAF_LOWRANK_MAX_N 128
#define HAF_LOWRANK_MAX_R 16
int haf_lowrank_c128(const double* G, int64_t n, int64_t r, double* out, haf_info* info);

/* Device-pointer form of the low-rank hafnian (App. C), like haf_launch:
 *   dG        : device pointer, G complex128 row-major n x r
 *   d_out     : device pointer to 5 doubles written as
 *               {re_hi, im_hi, re_lo, im_lo, abs_sum}
 *   d_work    : device workspace of at least haf_lowrank_workspace_bytes(n,
 *               r) bytes, 256-byte aligned, not shared with a concurrent
 *               call (it holds the two largest coefficient arrays: 48 bytes
 *               per degree-n monomial, plus small tables)
 *   stream    : cudaStream_t (NULL = legacy default stream)
 * The call only enqueues work (n + 3 kernel launches) and returns before the
 * result is ready.  n must be even, 2..HAF_LOWRANK_MAX_N (the host entry
 * point handles 0 and odd n), 1 <= r <= HAF_LOWRANK_MAX_R; HAF_EINVAL
 * otherwise or for a misaligned workspace, HAF_ESMALL if ws_bytes is too
 * small, HAF_ENOMEM if C(n+r-1, r-1) >= 2^40.  haf_lowrank_workspace_bytes
 * returns 0 for sizes that the launch rejects. */
size_t haf_lowrank_workspace_bytes(int64_t n, int64_t r);
int haf_lowrank_launch(const double* dG, int64_t n, int64_t r, double* d_out, void* d_work, size_t ws_bytes,
                       void* stream);

/* ------------------------------------------------------------------------
 * Autotuner (no counterpart in the paper).  The launch shape of a plan is
 * the number of warps per CTA (4, 8 or 16: the shared-memory slice of each
 * warp, hence the lanes per subset and the subsets per CTA, follow from it)
 * and the chunk granularity (about chunks_per_warp chunks of subsets per
 * resident warp).  haf_tune times every feasible shape (3 x 4 candidates,
 * each one warm-up plus `reps` launches of one hafnian of size n on a
 * synthetic matrix -- for large n this takes ~13 (reps+1) single-hafnian
 * times) and records the fastest for (n, flags) on the current device;
 * later haf_eval/haf_c128/haf_launch/haf_part calls with that key use it.
 * haf_tune_set records a shape without timing (e.g. one saved earlier).
 * haf_batched_tune does the same for one batch (its list of sizes and
 * flags), timing graph replays of the whole batch; later haf_batched /
 * *_c128_batched calls with the same sizes use the result.
 *   out->warps_per_block, out->chunks_per_warp : the chosen shape
 *   out->ms          : its mean time per launch (or per batch)
 *   out->ms_default  : the default shape's time (-1 if not a candidate)
 *   out->candidates  : shapes timed
 * ---------------------------------------------------------------------- */
typedef struct haf_tune_result {
  int32_t warps_per_block;
  int32_t chunks_per_warp;
  double ms;
  double ms_default;
  int32_t candidates;
} haf_tune_result;
int haf_tune(int64_t n, uint32_t flags, int32_t reps, haf_tune_result* out);
/* Host-only view of the plan a shape gives (for tests and tools): out[8] =
 * {chunks, launches (segments), warps per CTA of segments 0..2, subsets of
 * segments 0..2}.  Size classes whose tiles do not fit a warp's slice at
 * the requested warps per CTA form later segments with fewer warps.
 * `sms` is the SM count the chunk sizes are planned for. */
int haf_plan_stats(int64_t n, uint32_t flags, int32_t warps_per_block, int32_t chunks_per_warp, int32_t sms,
                   int64_t* out);
int haf_tune_set(int64_t n, uint32_t flags, int32_t warps_per_block, int32_t chunks_per_warp);
int haf_batched_tune(const double* const* As, const int64_t* ns, int64_t count, uint32_t flags, int32_t reps,
                     haf_tune_result* out);

/* ------------------------------------------------------------------------
 * Server: continuous batching of haf / lhaf requests on one GPU.
 * The paper computes one hafnian at a time (Sec. 4.1); this is the serving
 * form of the same summands.  Requests of mixed n are admitted while job
 * slots and device memory allow; each admitted job's subset chunks are
 * drained by a resident kernel together with other jobs' chunks (large-n
 * jobs are split into chunks that interleave with small ones).  A job's
 * result does not depend on what else ran with it (its chunking and its
 * reduction order are fixed by the job alone).
 *   cfg          : NULL for defaults; zero fields take their defaults.
 *   submit       : kind 0 = haf, 1 = lhaf; A is host complex128 n x n, copied
 *                  before return; returns a ticket.  HAF_EBUSY if the queue is
 *                  full, HAF_ENOMEM if the job can never fit the memory limit.
 *   poll         : waits up to timeout_us (< 0: no limit) for the ticket; out
 *                  = 2 doubles; info->seconds = latency from submit to the
 *                  result.  A ticket is collected once (then HAF_ENOTFOUND).
 *   destroy      : stops admitting and publishing work, lets the chunks
 *                  already handed to the GPU finish, then frees everything
 *                  (results not yet collected are lost).
 * The resident kernel exits once no warp has claimed a chunk for idle_us
 * and no claimed chunk is unfinished (or after 3000 x idle_us without a
 * claim, whatever is in flight), and the scheduler relaunches it when work
 * arrives; no device wait is unbounded.  create fails with HAF_EINVAL for max_jobs > 65535 or
 * ring_entries < 65536.
 * ---------------------------------------------------------------------- */
typedef struct haf_server haf_server;
typedef struct haf_server_cfg {
  int64_t max_jobs;     /* jobs admitted at once (default 256, max 65535)      */
  int64_t max_bytes;    /* device memory for admitted jobs (default 256 MiB)   */
  int64_t ring_entries; /* entries of each of the two descriptor rings (default 2^20, >= 2^16) */
  int64_t idle_us;      /* resident kernel idles out after this (default 20 ms) */
  int64_t chunk_us;     /* target warp time per work chunk (default 4 ms)      */
} haf_server_cfg;

int haf_server_create(const haf_server_cfg* cfg, haf_server** out);
int haf_server_submit(haf_server* s, int kind, const double* A, int64_t n, uint64_t* ticket);
int haf_server_poll(haf_server* s, uint64_t ticket, double* out, haf_info* info, int64_t timeout_us);
int haf_server_destroy(haf_server* s);

/* ------------------------------------------------------------------------
 * Utilities.
 * ---------------------------------------------------------------------- */
/* Measured FP64 FMA throughput of the current device, in TFLOP/s (2 flops
 * per FMA), from a dependent-chain DFMA kernel over all SMs; ms is the
 * kernel time.  Used as the roofline denominator. */
int haf_fp64_peak(double* tflops, double* ms);
const char* haf_last_error(void);
const char* haf_version(void);

#ifdef __cplusplus
}
#endif
#endif /* HAFNIAN_GB300_H */
