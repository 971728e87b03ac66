/*
 * krr.h -- C ABI of libkrr, a GB300 (sm_103a) implementation of the hot path
 * of partitioned kernel ridge regression (You, Demmel, Hsieh, Vuduc,
 * "Accurate, Fast and Scalable Kernel Ridge Regression on Parallel and
 * Distributed Systems", ICS'18): DKRR (one partition), BKRR2 with random
 * equal partitions and KKRR2 with K-means partitions.
 *
 * Conventions for every entry point
 *  - Array arguments are DEVICE pointers unless marked "host".  They are
 *    caller-owned, row-major and FP64 unless stated.  Outputs are
 *    caller-allocated.
 *  - Work is enqueued on the context's stream.  The synchronous return value
 *    reports argument and launch validation only; numerical outcomes arrive in
 *    per-solve status words valid after the stream is synchronised.
 *  - No exception crosses the ABI.  On a non-OK return krr_last_error()
 *    describes the failure.
 *  - A context is not thread-safe; use one per host thread/stream.
 */
#ifndef KRR_H
#define KRR_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct krr_ctx krr_ctx;     /* opaque: stream, HBM budget, error text */
typedef struct krr_model krr_model; /* opaque: library-owned device memory   */

typedef enum {
    KRR_OK = 0,
    KRR_ERR_ARG = 1,          /* invalid argument (sizes, null pointers, modes) */
    KRR_ERR_OOM = 2,          /* cudaMalloc failed                               */
    KRR_ERR_BUDGET = 3,       /* the context's HBM budget would be exceeded      */
    KRR_ERR_CUDA = 4,         /* a CUDA call failed                              */
    KRR_ERR_NOT_SPD = 5,      /* per solve: K + lambda m I not positive definite */
    KRR_ERR_NO_CONVERGE = 6,  /* per solve: refinement did not reach tolerance   */
    KRR_ERR_TIMEOUT = 7,      /* a bounded device-side wait expired              */
    KRR_ERR_UNSUPPORTED = 8   /* a valid request the library does not implement  */
} krr_status;

typedef enum { KRR_PART_RANDOM = 0, KRR_PART_KMEANS = 1, KRR_PART_KBALANCE = 2 } krr_part_mode;

/* Arithmetic of the kernel build, the Cholesky factor and its refinement.
 * FP64:   FP64 kernel, FP64 Cholesky, FP64 refinement (the plain path).
 * FP32:   FP32 factor of the double-float (~44-bit) kernel with FP32-class
 *         trailing updates (three TF32 tensor-core passes on hi/lo splits);
 *         conjugate-gradient refinement with double-float residuals.
 * TF32:   as FP32 but with a TF32-class factor: the panel solves store the
 *         L tiles in FP16 (the 11-bit significand of TF32) and the updates
 *         take one FP16 tensor-core pass; the preconditioner reads the FP16
 *         tiles.  A solve whose 1 + lambda m exceeds 2^24, or whose condition
 *         estimate passes the escalation threshold, is factored as FP32.
 * BF16X3: as FP32 but the trailing updates take three BF16 passes on
 *         split-BF16 operands (hi = rn(x), lo = rn(x - hi)), ~16-bit
 *         products with FP32 accumulation.                                   */
typedef enum { KRR_PREC_FP64 = 0, KRR_PREC_FP32 = 1, KRR_PREC_TF32 = 2, KRR_PREC_BF16X3 = 3 } krr_prec;

/* Table 1 kernel of the fits (Eq. 6) and predictions (Eq. 7).
 * GAUSSIAN: Phi(x, y) = exp(-||x - y||^2 / (2 sigma^2)) (the default).
 * LINEAR:   Phi(x, y) = x . y; sigma plays no part (every sigma of a fit
 *           gives the same model).  Kernel ridge regression with it is
 *           primal ridge regression (Eq. 2).  Needs KRR_PREC_FP64; the other
 *           precisions return KRR_ERR_UNSUPPORTED.                            */
typedef enum { KRR_KERNEL_GAUSSIAN = 0, KRR_KERNEL_LINEAR = 1 } krr_kernel;

/* Model choice (Eq. 3 scores):
 * PER_MODEL: one MSE per (partition, sigma, lambda) model; best model.
 * ROUTED:    each test point scored by its routed partition (the scoring
 *            step of Alg. BKRR2, KKRR2 Sec. 4.2); one MSE per grid point;
 *            best grid point.
 * AVERAGE:   DC-KRR (the averaging step of Alg. DC-KRR): predictions averaged over the
 *            partitions; one MSE per grid point.
 * ORACLE:    BKRR3 (the per-point choice of Alg. BKRR3): each test point takes the
 *            partition whose prediction is closest to its label.             */
typedef enum {
    KRR_SEL_PER_MODEL = 0,
    KRR_SEL_ROUTED = 1,
    KRR_SEL_AVERAGE = 2,
    KRR_SEL_ORACLE = 3
} krr_sel;

/* Create a context on `device` that enqueues on `cuda_stream` (a
 * cudaStream_t; NULL = legacy default stream).  hbm_budget_bytes caps the
 * device memory the library allocates (0 = no cap).  The context allocates
 * from its own stream-ordered pool, which keeps freed blocks for reuse until
 * krr_ctx_destroy (models still alive then keep theirs until freed).  One
 * context must not be used by two host threads at once; separate contexts
 * may.  Errors: KRR_ERR_ARG, KRR_ERR_CUDA. */
krr_status krr_ctx_create(krr_ctx **out, int device, void *cuda_stream, size_t hbm_budget_bytes);
/* Destroy a context (models must be freed first).  Synchronises its stream. */
krr_status krr_ctx_destroy(krr_ctx *ctx);
/* Text of the last failure on this context (valid until the next call). */
const char *krr_last_error(const krr_ctx *ctx);
/* Bytes currently allocated through the context. */
size_t krr_ctx_bytes_in_use(const krr_ctx *ctx);

/* Partition the training rows (the shuffle and even scatter of Alg. DC-KRR
 * for RANDOM; Alg. 2 plain K-means plus the KKRR2 nearest-centre rule,
 * Sec. 4.2, for KMEANS; Alg. K-balance Clustering, the BKRR partitioner, for
 * KBALANCE).
 *   X [n x d], Xt [t x d] (Xt may be NULL when t == 0).
 *   RANDOM: a seeded bijection (Feistel network over Philox4x32-10, cycle
 *     walking) shuffles the rows; the shuffled order is cut into p parts, the
 *     first n mod p one row longer.  perm[k] = row at shuffled position k.
 *     seed is used; iters, init_idx, centers, route are ignored (route, when
 *     given, is filled with 0).
 *   KMEANS: p = number of clusters; centres start at rows init_idx[0..p)
 *     (device, int64); `iters` assign+update rounds (stopping early at a
 *     fixed point is result-neutral); ties go to the lowest centre index;
 *     empty clusters keep their centre; centre sums run in one canonical
 *     order (blocks of 1024 rows, pairwise tree over blocks).  A final
 *     assignment with the final centres defines the partitions and routes
 *     the test rows.  Assignments are bit-exact with that definition (an FP64
 *     recheck decides near ties).  Workspace per assignment pass (d <= 96,
 *     p <= 256): about 76 bytes per row + 4 p bytes.
 *   KBALANCE: the K-means centres as above, then the balanced assignment of
 *     Alg. K-balance Clustering: rows in index order each take the nearest
 *     centre (squared FP64 distance in feature order, strict <, lowest index)
 *     among those holding fewer than ceil(n / p) rows; then every centre
 *     becomes the mean of its part (canonical order; an empty part keeps its
 *     centre), and the test rows are routed to the nearest such centre.
 *     Assignments are bit-exact with that sequential definition (replayed in
 *     at most p rounds).  Needs d <= 400; workspace n p 8 bytes.
 * Outputs: assign[n] (int32 partition of each row), perm[n] (int64 rows grouped
 * by partition; ascending row order inside a partition for KMEANS),
 * offsets[p+1] (int64), route[t] (int32, nullable), centers[p x d] (nullable;
 * required for KMEANS).  Errors: KRR_ERR_ARG, KRR_ERR_BUDGET, KRR_ERR_CUDA. */
krr_status krr_partition(krr_ctx *ctx, const double *X, int64_t n, int32_t d, const double *Xt, int64_t t,
                         krr_part_mode mode, int32_t p, int32_t iters, uint64_t seed, const int64_t *init_idx,
                         int32_t *assign, int32_t *route, int64_t *perm, int64_t *offsets, double *centers);

/* Fit every (partition, sigma, lambda) model: for partition j with m_j rows
 * X_j = X[perm[offsets[j] .. offsets[j+1])], solve Eq. 6 in its partitioned
 * form (K_j + lambda m_j I) alpha = y_j with the Gaussian kernel of Table 1,
 * K_ab = exp(-||x_a - x_b||^2 / (2 sigma^2)), by Cholesky factorisation
 * (Sec. 5.4) and refinement to FP64-level residuals.
 *   X [n x d], y [n], perm [offsets[p]], offsets [p+1] (device; read back to
 *   the host): offsets run from 0 to at most n, so a subset of the rows (the
 *   partitions a rank owns) can be fitted against the full X.
 *   sigmas [ns], lambdas [nl]: HOST arrays.  Grid index g = i_sigma * nl +
 *   i_lambda; solve/model index = j * (ns * nl) + g.
 *   *out receives a model owning the gathered rows and every alpha until
 *   krr_model_free.  solve_status [p*ns*nl] (device int32, nullable) receives
 *   KRR_OK, KRR_ERR_NOT_SPD or KRR_ERR_NO_CONVERGE per solve.
 *   alpha (device, nullable) receives offsets[p]*ns*nl doubles: partition j's block
 *   starts at offsets[j]*ns*nl and holds, for each g, m_j coefficients in the
 *   partition's row order.
 * A refined-precision solve (FP32, TF32, BF16X3) whose refinement does not
 * converge -- its condition estimate near the reciprocal of the factor's
 * unit roundoff, where the low-precision factor no longer preconditions --
 * is solved again on the plain FP64 path once the batch's work buffers are
 * released; it then reports KRR_OK and factor class 0
 * (krr_model_factor_class).  krr_ctx_set_fp64_fallback(ctx, 0) turns this
 * off (such solves then report KRR_ERR_NO_CONVERGE).
 * This call synchronises the stream (partition sizes are needed on the host;
 * refinement rounds poll a device flag).  Errors: KRR_ERR_ARG,
 * KRR_ERR_BUDGET, KRR_ERR_OOM, KRR_ERR_CUDA, KRR_ERR_TIMEOUT. */
krr_status krr_fit_batch(krr_ctx *ctx, const double *X, const double *y, int64_t n, int32_t d,
                         const int64_t *perm, const int64_t *offsets, int32_t p, const double *sigmas, int32_t ns,
                         const double *lambdas, int32_t nl, krr_prec prec, krr_model **out,
                         int32_t *solve_status, double *alpha);

/* Independent problems in one batched fit: partition j is its own KRR
 * problem (Eq. 6 for X_j = X[perm[offsets[j] .. offsets[j+1])]) with its own
 * sigmas[j] and lambdas[j] (HOST arrays of p values) -- the batching form that
 * packs queued requests of different sizes and hyper-parameters into the same
 * launches as uneven partitions (the paper's partitions share one grid; its
 * independent per-partition solves are what makes the packing exact).  One
 * model per partition: solve/model index j, alpha block j at offsets[j].
 * Otherwise as krr_fit_batch (same precisions, refinement, FP64 re-solve of
 * unconverged solves, status words); predict with krr_predict (route[q] = the
 * partition of test row q; yhat [1 x t]).  Each partition's result is the
 * same bits whatever else is in the batch (every solve runs on its own
 * tiles, and a converged solve stops) at a fixed panel width
 * (krr_ctx_set_panel_width).  Needs a refined precision (FP32, TF32,
 * BF16X3), the Gaussian kernel and d <= 96, else KRR_ERR_UNSUPPORTED.
 * Errors as krr_fit_batch. */
krr_status krr_fit_jobs(krr_ctx *ctx, const double *X, const double *y, int64_t n, int32_t d,
                        const int64_t *perm, const int64_t *offsets, int32_t p, const double *sigmas,
                        const double *lambdas, krr_prec prec, krr_model **out, int32_t *solve_status,
                        double *alpha);

/* Eq. 7 prediction, fused: kernel rows are built on the fly and contracted
 * with alpha; K(test, train) is never stored.
 *   Xt [t x d].  route == NULL: every model predicts every test row and
 *   yhat is [p*ns*nl x t] (model-major).  route [t] given: row q is predicted
 *   only by partition route[q]'s models and yhat is [ns*nl x t].  A partition
 *   with no rows predicts 0, and so does a row whose route lies outside
 *   [0, p) (the route is read on the device only; such a value is skipped,
 *   never followed).  Errors: KRR_ERR_ARG, KRR_ERR_CUDA. */
krr_status krr_predict(krr_ctx *ctx, const krr_model *model, const double *Xt, int64_t t, const int32_t *route,
                       double *yhat);

/* Score and choose (Eq. 3; see krr_sel).
 *   yhat as produced by krr_predict (routed layout for ROUTED, all-models
 *   layout otherwise), yt [t].  p, G = ns*nl.
 *   mse (device FP64): p*G entries for PER_MODEL, G otherwise.
 *   best (device int32, 1 entry): index of the lowest MSE, lowest index on
 *   ties.  Deterministic: fixed reduction order.  Errors: KRR_ERR_ARG,
 *   KRR_ERR_CUDA. */
krr_status krr_select(krr_ctx *ctx, const double *yhat, const double *yt, int64_t t, int32_t p, int32_t G,
                      krr_sel mode, double *mse, int32_t *best);

/* Per-solve diagnostics of a fitted model (HOST outputs, p*ns*nl entries
 * each, nullable): refinement iterations, Gershgorin condition estimate
 * (max row sum of K + lambda m I over lambda m) and final scaled residual.
 * Synchronises the stream. */
krr_status krr_model_stats(krr_ctx *ctx, const krr_model *model, int32_t *iters, double *kappa_est,
                           double *resid);

/* Factor class of every solve of a fitted model (HOST output, p*ns*nl
 * entries): 0 FP64 (plain path), 1 one FP16 tensor-core pass (TF32-class),
 * 2 three BF16 passes on split operands, 3 three TF32 passes on operands
 * split by the panel solve (FP32-class), 4 three TF32 passes split in shared
 * memory (the refactorisation after a low-precision breakdown).  No
 * counterpart in the paper; used to attribute factor time to the tensor-core
 * rate each solve ran at.  Errors: KRR_ERR_ARG. */
krr_status krr_model_factor_class(krr_ctx *ctx, const krr_model *model, int32_t *cls);

/* Release a model's device memory. */
krr_status krr_model_free(krr_ctx *ctx, krr_model *model);

/* The grouping step of krr_partition on its own (the scatter of rows to
 * their partitions, KKRR): rows grouped by partition, ascending row order
 * inside a partition.  assign [n] (device int32), perm [n] and offsets [p+1]
 * (device int64) outputs.  A value of assign outside [0, p) is skipped (its
 * row lands in no partition and offsets[p] < n).  p <= 12288.  Errors:
 * KRR_ERR_ARG, KRR_ERR_BUDGET, KRR_ERR_OOM, KRR_ERR_CUDA. */
krr_status krr_group_rows(krr_ctx *ctx, const int32_t *assign, int64_t n, int32_t p, int64_t *perm,
                          int64_t *offsets);

/* Alg. 2 (plain K-means) as separate steps, for ranks that each hold a
 * contiguous range of 1024-row blocks of the training set and exchange the
 * block sums between the two halves of the centre update (the per-round
 * exchange of the multi-process K-means; the combined centres are the same
 * bits at any number of ranks).  Same arithmetic as krr_partition(KMEANS).
 * krr_kmeans_assign: the assignment step (Alg. 2, nearest centre, FP64
 *   squared distance in feature order, strict <, lowest index; bit-exact
 *   through the FP64 recheck of near ties) of X [n x d] to the FP64 centres
 *   C [k x d]; assign [n] int32 output.  Workspace n d 4 bytes, plus for
 *   d <= 96 and k <= 256 (the tiled screen) about 76 n + 4 k bytes for the
 *   rows with several candidates and their (row, centre) pairs.
 * krr_kmeans_block_sums: first half of the centre step: for each block of
 *   1024 consecutive rows of X (X must start at a block boundary of the
 *   global row numbering), every centre's member sum in ascending row order
 *   and its member count: sums [ceil(n/1024) x k x d] FP64, counts
 *   [ceil(n/1024) x k] int64, outputs.  assign [n] must hold values in
 *   [0, k).
 * krr_kmeans_combine: second half: the block sums of all nblk blocks of the
 *   training set, in block order, combined by the pairwise tree (level by
 *   level, an odd last block carried up), one division by the member count;
 *   C [k x d] in/out, a centre with no members keeps its value.  Needs
 *   2 nblk 8 bytes <= 200 KiB of shared memory per 1..32 entries.
 * All arrays are device arrays.  Errors: KRR_ERR_ARG, KRR_ERR_UNSUPPORTED,
 * KRR_ERR_OOM, KRR_ERR_CUDA. */
krr_status krr_kmeans_assign(krr_ctx *ctx, const double *X, int64_t n, int32_t d, const double *C, int32_t k,
                             int32_t *assign);
krr_status krr_kmeans_block_sums(krr_ctx *ctx, const double *X, int64_t n, int32_t d, const int32_t *assign,
                                 int32_t k, double *sums, int64_t *counts);
krr_status krr_kmeans_combine(krr_ctx *ctx, const double *sums, const int64_t *counts, int64_t nblk, int32_t k,
                              int32_t d, double *C);

/* Group rows by partition without allocating any device memory -- the same
 * grouping krr_partition performs after its assignment (rows of partition 0
 * first, ascending row order inside a partition).  The paper has no
 * counterpart: this variant exists for callers that cannot call cudaMalloc,
 * e.g. code whose GPU memory is entirely owned by another allocator, or a
 * request loop that must not allocate because cudaMalloc/cudaFree can
 * synchronise the device and take unbounded time.
 *   cuda_stream: the stream to enqueue on (a cudaStream_t; NULL = legacy
 *   default stream).  assign [n] (device int32, every value in [0, p)),
 *   perm [n] (device int64, output), offsets [p+1] (device int64, output);
 *   all caller-owned.  assign is read on the device only, so it cannot be
 *   validated before the call returns: a value outside [0, p) is skipped
 *   (its row is placed in no partition), which leaves offsets[p] < n and
 *   perm[offsets[p] .. n) unwritten -- check offsets[p] == n after the
 *   stream has run when assign is not trusted.  No context is needed and nothing is allocated: the
 *   per-block counts live in a fixed 4 MiB device array inside the library
 *   (held on every GPU that loads it until the process exits), so
 *   ceil(n / 1024) * p must not exceed 524288 and p must not exceed 12288;
 *   larger requests return KRR_ERR_ARG before anything is enqueued.
 *   The first call on a device looks up that array's device address (once
 *   per device) and keeps it; make that first call before any stream
 *   capture.  The kept address is stale after cudaDeviceReset on that
 *   device: do not call this entry point again in such a process.  Calls share
 *   the array and keep the last call's contents (every entry read is written
 *   first); calls that overlap on the GPU race on it and must be serialised.
 * Errors: KRR_ERR_ARG, KRR_ERR_CUDA. */
krr_status krr_gather_noalloc(void *cuda_stream, const int32_t *assign, int64_t n, int32_t p, int64_t *perm,
                              int64_t *offsets);

/* ---- instrumentation and tuning (no counterpart in the paper) ----------
 * krr_ctx_set_profiling: when on, every kernel launch of the context is
 *   bracketed by CUDA events on the context's stream (adds ~2 us per launch).
 *   Turning it on or off clears the totals.
 * krr_ctx_profile: total device time (ms, host output) and launch count of
 *   one kernel class since profiling was switched on; synchronises the
 *   stream.  kind: 0 partition, 1 stage, 2 kernel build, 3 potrf, 4 trsm,
 *   5 trailing update, 6 matvec, 7 preconditioner, 8 CG vector ops,
 *   9 predict, 10 select.  Errors: KRR_ERR_ARG.
 * krr_ctx_set_panel_width: outer panel width W (tiles) of the blocked
 *   Cholesky schedule, 1..64; 0 (the default) lets the library tune it: the
 *   first fit of a context for a given (precision, largest tile count) times
 *   W in {1, 2, 4, 8} on its own matrices and keeps the fastest.
 * krr_ctx_get_panel_width: the width in force for (precision, largest tile
 *   count): the explicit one, the tuned one, or 0 if not tuned yet.
 * krr_ctx_set_target_error: forward-error target of the refinement for the
 *   refined precisions: a solve stops once its Gershgorin condition estimate
 *   times its backward error (the scaled residual) is at most `rel` (default
 *   1e-7, ten times below the 1e-6 parity bar), or at the FP64-class floor
 *   2^-46 of the scaled residual, whichever comes first.  0 always runs to the
 *   floor.  The plain FP64 path always runs to its floor 2^-50.  Errors:
 *   KRR_ERR_ARG (rel < 0 or rel > 1e-2).
 * krr_ctx_set_escalation: with KRR_PREC_TF32 (KRR_PREC_BF16X3), a solve whose
 *   Gershgorin condition estimate times 2^-11 (2^-16) exceeds `kappa_u`
 *   (default 32) has its trailing updates run in the FP32-class three-pass
 *   TF32 mode instead (the cheaper factor is then too poor a preconditioner);
 *   0 escalates every solve.  Errors: KRR_ERR_ARG (negative).
 * krr_launch_count: kernels launched by this process through libkrr. */
krr_status krr_ctx_set_profiling(krr_ctx *ctx, int on);
/* krr_ctx_wait_probe: self-check of the bounded device waits that every
 *   pipelined kernel of the library uses (no counterpart in the paper).  A
 *   one-CTA kernel starts a 4 KB bulk copy into shared memory, then waits on
 *   an mbarrier that nothing ever completes; the wait gives up after
 *   `seconds`, records KRR_ERR_TIMEOUT in the context's device error word,
 *   waits (bounded) for its own copy to land and exits, as the pipelined
 *   kernels do when a producer never delivers.  Returns KRR_ERR_TIMEOUT when
 *   all of that happened (the context stays usable; the error word is
 *   cleared), KRR_ERR_CUDA when the wait or the copy misbehaved or a CUDA
 *   call failed, KRR_ERR_ARG for seconds outside [1e-6, 10].  Synchronises
 *   the stream. */
krr_status krr_ctx_wait_probe(krr_ctx *ctx, double seconds);
krr_status krr_ctx_profile(krr_ctx *ctx, int kind, double *total_ms, long long *launches);
krr_status krr_ctx_set_panel_width(krr_ctx *ctx, int W);
krr_status krr_ctx_get_panel_width(const krr_ctx *ctx, int prec, int max_tiles, int *W);
krr_status krr_ctx_set_target_error(krr_ctx *ctx, double rel);
krr_status krr_ctx_set_escalation(krr_ctx *ctx, double kappa_u);
/* krr_ctx_set_fp64_fallback: on (the default) / off -- the FP64 re-solve of
 *   unconverged refined-precision solves described at krr_fit_batch.
 *   Errors: KRR_ERR_ARG. */
krr_status krr_ctx_set_fp64_fallback(krr_ctx *ctx, int on);

/* krr_ctx_set_kernel: the Table 1 kernel of this context's subsequent
 * krr_fit_batch calls (default GAUSSIAN); a model keeps the kernel it was
 * fitted with for krr_predict.  Errors: KRR_ERR_ARG (unknown kernel). */
krr_status krr_ctx_set_kernel(krr_ctx *ctx, krr_kernel kind);
long long krr_launch_count(void);

#ifdef __cplusplus
}
#endif
#endif /* KRR_H */
