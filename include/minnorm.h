/*
 * minnorm.h -- C ABI of the GB300 (sm_103a) randomized minimal-norm solver.
 *
 * Computes x ~ p, the minimal-Euclidean-norm solution of A p = b for a
 * full-rank complex A (m x n, m < n), with ||x - p|| <= eps ||p||, by the
 * algorithm of M. Tygert, "A fast algorithm for computing minimal-norm
 * solutions to underdetermined systems of linear equations" (arXiv:0905.4745):
 *   Step 1 (Eq. randmat)   Y = T A^*, T the l x n SRFT of Section 3
 *                           (Eqs. SRFT, SRFT2, Rokhlin_trans, big_def);
 *   Step 2 (Eq. lineq)     the pivoted Householder QR  Y P = Q R;
 *   Steps 3-4 (Eq. overdet) conjugate gradients preconditioned by R, one
 *                           A^* w and one A v pass over A per iteration;
 *   Step 5 (Eq. output)    x = A^* y.
 * Steps 2-3 enter only through R and P: since A c = b (Lemma 5.1, Eq. easy),
 * the CG of Step 4 runs on (R^{-*} P^T A A^* P R^{-1}) u = R^{-*} P^T b and
 * never forms z or c. An outer refinement loop with double-double residuals
 * (an extension of Remark 4.2's extra CG iterations) reaches eps below the
 * FP64 limit kappa * 2^-53.
 *
 * Conventions (every entry point):
 *   - "device" pointers are CUDA device (or managed) memory on the plan's
 *     device; "host" pointers are ordinary host memory. The caller owns every
 *     buffer it passes; the plan owns its own workspace (allocated by
 *     minnorm_plan_create, freed by minnorm_plan_destroy). No other entry point
 *     allocates device memory except minnorm_solve_host (see there).
 *   - complex arrays are interleaved (re, im) pairs: complex128 = 2 doubles,
 *     complex64 = 2 floats, i.e. the layout of C99 `double complex` and of
 *     torch.complex128/complex64 contiguous tensors.
 *   - A is row-major m x n with leading dimension lda >= n (row i at A + i*lda).
 *   - all work is enqueued on the plan's stream (a cudaStream_t passed as
 *     void*; NULL = the legacy default stream) and is stream-ordered; calls
 *     that return values in host memory synchronize that stream.
 *   - one plan serves one stream and one host thread at a time.
 *   - errors are returned as minnorm_status; a CUDA error inside a call is
 *     reported as MINNORM_ECUDA and leaves the plan usable only for destroy.
 */
#ifndef MINNORM_H
#define MINNORM_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct minnorm_plan_s *minnorm_plan_t;
typedef struct minnorm_batch_s *minnorm_batch_t;

typedef enum {
  MINNORM_C64 = 1,           /* A stored as complex64  */
  MINNORM_C128 = 2           /* A stored as complex128 */
} minnorm_dtype;

typedef enum {
  /* plain: sketch and CG products in complex FP64 */
  MINNORM_FP64 = 0,
  /* mixed: sketch FFT/chains and CG products in complex FP32 (from a
   * complex64 copy of A kept in the plan when A is complex128); pivoted QR,
   * R^{-1}, the CG scalars and vectors of length m, and the refinement
   * residuals stay FP64 / double-double */
  MINNORM_MIXED = 1
} minnorm_precision;

typedef enum {
  MINNORM_OK = 0,
  MINNORM_EINVAL = 1,        /* invalid argument (null pointer, m >= n, l not in (m, n], eps not in (0,1), ...) */
  MINNORM_ESTATE = 2,        /* minnorm_solve before minnorm_sketch, or a plan already failed */
  MINNORM_ENOMEM = 3,        /* device or host allocation failed */
  MINNORM_ECUDA = 4,         /* a CUDA call failed */
  MINNORM_ERANK = 5,         /* the sketch Y is numerically rank deficient (Remark 4.1): re-plan with another seed */
  MINNORM_ENOCONV = 6,       /* the refinement hit its step cap before eps; x holds the last iterate */
  MINNORM_EFLOOR = 7,        /* the refinement stagnated above eps; x holds the best iterate */
  MINNORM_ETIMEOUT = 8,      /* a bounded device-side wait expired (grid barrier); results are invalid */
  MINNORM_ENOTSUP = 9        /* a size this build does not handle (see minnorm_plan_create) */
} minnorm_status;

/* Flags for minnorm_plan_create. */
#define MINNORM_FLAG_TIMING 1u  /* record CUDA events around the phases and the hot kernels */

typedef struct {
  int32_t outer_steps;       /* refinement steps taken */
  int32_t cg_iters;          /* CG iterations summed over all steps */
  int32_t exact_passes;      /* passes over A in exact fixed-point arithmetic (x = A^* y, b - A x) */
  int32_t status;            /* this solve's minnorm_status (per column / per system in the
                                block and batch entry points) */
  double err_bound;          /* rigorous a-posteriori bound on ||x - p|| / ||x||:
                                ||R^{-*} P^T (b - A x)|| / ((1 - cert_delta) ||x||), rounding of
                                the certificate itself included; +inf when cert_delta >= 1/2 */
  double resid_rel;          /* ||b - A x|| / ||b|| from the last residual */
  double rdiag_max;          /* |R_11| */
  double rdiag_min;          /* |R_mm| */
  double sigma_min_R;        /* lower bound of sigma_min(R): 1 / ||R^{-1}||_F */
  double sigma_max_R;        /* upper bound of sigma_max(R): ||R||_F */
  double cert_delta;         /* sigma_min(A^* P R^{-1}) >= 1 - cert_delta: the a priori bounds of
                                the sketch's and the QR's rounding times ||A||_F ||R^{-1}||_F (1 when
                                they certify nothing) */
  float ms_sketch;           /* with MINNORM_FLAG_TIMING: Step 1 (sketch) of the last minnorm_sketch */
  float ms_qr;               /* with MINNORM_FLAG_TIMING: Step 2 (QR + R^{-1}) of the last minnorm_sketch */
  float ms_solve;            /* with MINNORM_FLAG_TIMING: Steps 3-5 of this solve */
  float ms_cg;               /* with MINNORM_FLAG_TIMING: this solve's CG products (Step 4) */
  float ms_refine;           /* with MINNORM_FLAG_TIMING: this solve's exact residuals (refinement, Step 5) */
  float reserved;
} minnorm_info;

/*
 * Create a plan for m x n systems (Section 4: m < l < n; l = 0 selects l = 4m,
 * the choice of Remark 5.6 and Section 7; l = n is also accepted so that tiny
 * systems with 4m >= n still run, T then being a random unitary matrix).
 * Draws one SRFT realization (Section 3) from `seed` with SplitMix64 streams
 * (d, zeta, zeta~ uniform on the unit circle; Pi, Pi~ uniform permutations;
 * theta, theta~ uniform on [0, 2 pi); l rows of F sampled without
 * replacement, as the paper's implementation does) and uploads it.
 * Allocates all device workspace for (m, n, l, dtype, precision).
 *   plan:   out, host pointer to the new handle (set to NULL on failure).
 *   m, n:   1 <= m < n; n >= 2.
 *   flags:  0 or MINNORM_FLAG_TIMING.
 *   stream: cudaStream_t as void*.
 * Errors: EINVAL (sizes, enums), ENOMEM, ECUDA, ENOTSUP (a random Givens
 * chain needing a halo longer than the kernels hold; probability ~0).
 */
minnorm_status minnorm_plan_create(minnorm_plan_t *plan, int64_t m, int64_t n, int64_t l,
                                   minnorm_dtype dtype, minnorm_precision precision,
                                   uint64_t seed, uint32_t flags, void *stream);

/*
 * Replace the plan's SRFT realization by caller-supplied parameters (host
 * arrays, read during the call): zeta_t, zeta, d: n complex128 of modulus 1;
 * pi_t, pi: n int64, permutations of 0..n-1, acting by gathering
 * ((Pi v)[j] = v[pi[j]]); theta_t, theta: n-1 doubles; s: l int64, strictly
 * increasing in [0, n). Invalidates a previous sketch.
 * Errors: EINVAL (null pointer, a value out of range), ENOTSUP (halo), ECUDA.
 */
minnorm_status minnorm_plan_set_params(minnorm_plan_t plan,
                                       const double *zeta_t, const int64_t *pi_t, const double *theta_t,
                                       const double *zeta, const int64_t *pi, const double *theta,
                                       const double *d, const int64_t *s);

/*
 * Copy the plan's SRFT realization (Section 3) into host arrays of the layout
 * minnorm_plan_set_params takes: zeta_t, zeta, d: n complex128 (2n doubles);
 * pi_t, pi: n int64; theta_t, theta: n-1 doubles; s: l int64. Any pointer may
 * be NULL to skip that array. Exporting then setting the same arrays leaves the
 * plan's transform unchanged (the oracle can also ingest them). No device
 * access. Errors: EINVAL (null plan).
 */
minnorm_status minnorm_plan_export_params(minnorm_plan_t plan, double *zeta_t, int64_t *pi_t, double *theta_t,
                                          double *zeta, int64_t *pi, double *theta, double *d, int64_t *s);

/*
 * Steps 1-2 for the matrix A (device, row-major m x n, dtype of the plan):
 * Y = T A^* (Eq. randmat), then Y P = Q R by Householder QR with column
 * pivoting (Step 2), then the plan keeps P R^{-1}. A is read, never written.
 * Errors: EINVAL (null A, lda < n), ERANK (|R_mm| <= 64 m 2^-53 |R_11|),
 * ETIMEOUT, ECUDA. Synchronizes the stream (it reads the rank test).
 */
minnorm_status minnorm_sketch(minnorm_plan_t plan, const void *A, int64_t lda);

/*
 * Steps 3-5 for the A of the last minnorm_sketch and the right-hand side b
 * (device, m complex128): writes x (device, n complex128) with
 * ||x - p|| <= eps ||p|| when it returns MINNORM_OK. A must hold the same
 * values as at minnorm_sketch.
 *   eps:  in (0, 1); the refinement stops once its a-posteriori bound is <= eps.
 *   info: host pointer, or NULL for the asynchronous form.
 * With info != NULL the call synchronizes the stream once per refinement step
 * (the stopping test is read on the host) and returns the solve's status:
 * EINVAL, ESTATE (no sketch), ENOCONV, EFLOOR (x still written), ETIMEOUT, ECUDA.
 * With info == NULL the call makes no host round trip: it enqueues the whole
 * refinement loop (at most 12 steps; the stopping test runs on the device and the
 * steps after it return at once) and the copy of x, and returns MINNORM_OK once
 * they are enqueued (argument errors are still returned at once). The solve's
 * status then sits in a device word of the plan; read it with
 * minnorm_solve_wait. Until then x, b and A must stay valid and unchanged. A
 * plan that has not yet run a synchronous solve uses its default work splits
 * (the autotuner runs only in the synchronous form).
 */
minnorm_status minnorm_solve(minnorm_plan_t plan, const void *A, int64_t lda, const void *b,
                             double eps, void *x, minnorm_info *info);

/*
 * Waits for the plan's last asynchronous minnorm_solve (synchronizes the plan's
 * stream) and returns that solve's status (OK, ENOCONV, EFLOOR, or ETIMEOUT when
 * a bounded device-side wait expired). info (host, nullable) receives its step
 * counts, bound and residual; with MINNORM_FLAG_TIMING also its times.
 * Errors: EINVAL (null plan), ESTATE (no asynchronous solve pending), ECUDA.
 */
minnorm_status minnorm_solve_wait(minnorm_plan_t plan, minnorm_info *info);

/*
 * Steps 3-5 for nrhs right-hand sides sharing the A, T and R of the last
 * minnorm_sketch (the block right-hand-side case: the sketch and the pivoted
 * QR, the costly part of a solve, are paid once for all columns).
 *   B:    device, m x nrhs complex128, column-major: column j at B + j*ldb.
 *   X:    device, n x nrhs complex128, column-major: column j at X + j*ldx.
 *   ldb >= m, ldx >= n, nrhs >= 1; eps as for minnorm_solve.
 *   infos: host array of nrhs minnorm_info, or NULL.
 * Every column gets the guarantee of minnorm_solve. Returns MINNORM_OK when
 * every column did; otherwise the status of the first column that did not
 * (ENOCONV / EFLOOR columns are still written and the later columns still
 * solved; EINVAL, ESTATE and ECUDA stop at once).
 */
minnorm_status minnorm_solve_many(minnorm_plan_t plan, const void *A, int64_t lda, const void *B, int64_t ldb,
                                  int64_t nrhs, double eps, void *X, int64_t ldx, minnorm_info *infos);

/*
 * minnorm_sketch + minnorm_solve on HOST buffers: copies A (m x n, lda) and b
 * to the device, solves, and copies x (n complex128) back. The device copy of
 * A and b is plan-owned and allocated on the first call (and again only if
 * that allocation is missing). Pinned host memory makes the copies
 * asynchronous. Errors: those of minnorm_sketch and minnorm_solve, ENOMEM.
 */
minnorm_status minnorm_solve_host(minnorm_plan_t plan, const void *A_host, int64_t lda,
                                  const void *b_host, double eps, void *x_host, minnorm_info *info);

/*
 * Batches of independent systems of uneven sizes (system i: m[i] x n[i], any
 * n[i] >= 2, m[i] < n[i], l[i] = min(4 m[i], n[i])), solved in turn on one
 * stream. System i uses the SRFT realization a plan with seed (seed + i)
 * would draw. Each system keeps its own parameter tables, sketch, R and
 * P R^{-1}; the m x n-sized scratch (the sketch's transform buffers, the
 * fixed-point and complex64 copies of A) is one pool sized for the largest
 * system and shared, so a batch holds little more than its largest plan.
 *   count: >= 1; m, n: host arrays of count sizes; dtype, precision, flags,
 *   stream as for minnorm_plan_create.
 * Errors: EINVAL (a size or enum), ENOMEM, ENOTSUP, ECUDA.
 */
minnorm_status minnorm_batch_create(minnorm_batch_t *batch, int32_t count, const int64_t *m, const int64_t *n,
                                    minnorm_dtype dtype, minnorm_precision precision, uint64_t seed,
                                    uint32_t flags, void *stream);

/*
 * Steps 1-5 for every system of the batch: A[i] (device, row-major m[i] x n[i],
 * leading dimension lda[i], or n[i] when lda is NULL), b[i] (device, m[i]
 * complex128) -> x[i] (device, n[i] complex128), each with the guarantee of
 * minnorm_solve for eps. A, lda, b, x, infos are host arrays of count entries
 * (infos may be NULL; infos[i].status is system i's status). Returns
 * MINNORM_OK when every system did; otherwise the status of the first system
 * that did not (a system ending in ERANK, ENOCONV or EFLOOR does not stop the
 * others; EINVAL, ECUDA and ETIMEOUT stop at once). Synchronizes the stream.
 */
minnorm_status minnorm_batch_solve(minnorm_batch_t batch, const void *const *A, const int64_t *lda,
                                   const void *const *b, double eps, void *const *x, minnorm_info *infos);

/* minnorm_kernel_stats for system `system` of a batch created with
 * MINNORM_FLAG_TIMING, or summed over all systems when system = -1 (each
 * system's counts cover its last Steps 1-5). Errors: EINVAL. */
minnorm_status minnorm_batch_kernel_stats(minnorm_batch_t batch, int32_t system, int32_t k, int32_t *launches,
                                          double *ms);

/* Free the batch, its plans and the shared scratch. NULL is accepted. */
minnorm_status minnorm_batch_destroy(minnorm_batch_t batch);

/* Free the plan and its workspace (synchronizes its stream). NULL is accepted. */
minnorm_status minnorm_plan_destroy(minnorm_plan_t plan);

/* Limit of the plan's bounded device-side waits (grid barriers, the QR's pivot
 * exchange, mbarrier phases): limit_ns in [1 ms, 2 s], 2 s by default. A wait
 * that runs out makes its kernel record the failure, wait (bounded) for its own
 * copies in flight, release what it holds and return; the call then reports
 * MINNORM_ETIMEOUT and the plan is left usable only for destroy. withhold = 1
 * (tests of that path) makes one CTA of the plan's next fused CG launch (mixed
 * precision, m <= 512) leave at once without arriving at the grid barrier, so
 * the wait runs out for certain. The paper has no counterpart. Errors: EINVAL. */
minnorm_status minnorm_plan_set_wait_limit(minnorm_plan_t plan, uint64_t limit_ns, int32_t withhold);

/* Static string naming a status. */
const char *minnorm_status_string(minnorm_status status);

/* ------------------------------------------------------------------------
 * Component entry points: the individual steps of the hot path, exposed so
 * that each can be checked on its own. They use the plan's workspace and its
 * stream and allocate nothing.
 * ---------------------------------------------------------------------- */

/* Copy the sketch Y = T A^* of the last minnorm_sketch (Step 1, Eq. randmat),
 * taken before the QR overwrote it, to Y_out (device, l x m complex128,
 * column-major: column i = T conj(A[i, :])). Requires a plan created with
 * MINNORM_FLAG_KEEP_SKETCH. Errors: ESTATE, EINVAL. */
#define MINNORM_FLAG_KEEP_SKETCH 2u
minnorm_status minnorm_get_sketch(minnorm_plan_t plan, void *Y_out);

/* Copy R (device, m x m complex128, column-major, upper triangular, real
 * diagonal) and the pivots (device, m int64: column k of R belongs to column
 * piv[k] of Y) of the last minnorm_sketch (Step 2). Errors: ESTATE, EINVAL. */
minnorm_status minnorm_get_factor(minnorm_plan_t plan, void *R_out, void *piv_out);

/* Copy the preconditioner P R^{-1} of the last minnorm_sketch (Step 2's
 * factors as Steps 3-4 apply them: the CG runs on the system preconditioned
 * by it) to W_out (device, m x m complex128, column-major: row piv[k] of
 * P R^{-1} is row k of R^{-1}). Computed in FP64 by back substitution, or,
 * for sketches factored by the blocked QR and m >= 256, by blocks of 32 rows
 * with the rank-32 updates on the tensor cores; either way with
 * ||R X - I||_F <= 4 m 2^-53 ||R||_F ||X||_F for X = P^T W_out, the bound the
 * certificate uses. Errors: ESTATE, EINVAL. */
minnorm_status minnorm_get_preconditioner(minnorm_plan_t plan, void *W_out);

/* One CG product pair of Step 4 in the plan's precision, on device vectors:
 * q = A^* w (w: m complex128 -> q: n complex128) and t = A q (t: m complex128).
 * In MINNORM_MIXED the products read the complex64 copy of A made by
 * minnorm_sketch and are computed in FP32; otherwise FP64. Either output
 * pointer may be NULL to skip it. With q NULL in MINNORM_MIXED and
 * 512 < m <= 4096, t comes from the CG's one-pass form (A read once, by
 * clusters of CTAs; an even lda and a 16-byte aligned A). Errors: ESTATE,
 * EINVAL, ETIMEOUT (a load of the one-pass form did not arrive within the
 * plan's wait limit; the plan is then usable only for destroy). */
minnorm_status minnorm_cg_products(minnorm_plan_t plan, const void *A, int64_t lda,
                                   const void *w, void *q, void *t);

/* The products of the block CG (Step 4 for 32 right-hand sides sharing A, as
 * minnorm_solve_many runs it in MINNORM_MIXED): Q = A^* W and T = A Q for W
 * (device, m x 32 complex128, row-major: column c of row i at i * 32 + c),
 * Q (device, n x 32 complex128, row-major) and T (device, m x 32 complex128,
 * row-major). W is rounded to complex64; Q = A^* W and T = A Q (with Q as
 * returned, complex64) are computed on the tensor cores from exact three-way
 * BF16 splits of both operands with FP32 accumulation (the six leading cross
 * products: FP32-level accuracy); the partial sums of T over column ranges
 * are added in FP64.
 * A is the complex64 copy made by minnorm_sketch (complex128 plans) or A
 * itself (complex64 plans). The plan must be MINNORM_MIXED. Synchronizes the
 * plan's stream. Errors: EINVAL, ESTATE, ETIMEOUT (a bounded wait inside the
 * tensor-core kernel expired). */
minnorm_status minnorm_block_products(minnorm_plan_t plan, const void *A, int64_t lda,
                                      const void *W, void *Q, void *T);

/* The accurate residual of the refinement: for y = y_hi + y_lo (device, m
 * complex128 each; y_lo may be NULL) computes x = A^* y into x_hi + x_lo
 * (device, n complex128 each, a double-double pair) and r = b - A x (device,
 * m complex128, rounded to FP64). Both products are accumulated exactly in
 * 128-bit fixed point: A with one exponent per row (exact for complex64
 * storage; complex128 components more than 2^9 below their row's largest are
 * rounded at 2^-62 of it), y and x with one exponent per vector and 109+
 * bits. Re-derives the plan's fixed-point copy of A from A. Errors: EINVAL. */
minnorm_status minnorm_residual_dd(minnorm_plan_t plan, const void *A, int64_t lda,
                                   const void *y_hi, const void *y_lo, const void *b,
                                   void *r, void *x_hi, void *x_lo);

/* The trailing-update products of Step 2's blocked Householder QR, on the
 * tensor cores with FP64 accuracy (exact BF16 slicing of both operands, the
 * leading levels accumulated exactly; as accurate as an FP64 dot product):
 *   W = V^H C      (when W is not NULL: W device, 32 x cols, column-major, ld 32)
 *   C = C - V Z    (when Z is not NULL, after W: Z device, 32 x cols, ldz >= 32)
 * V (device, rows x 32, ldv >= rows), C (device, rows x cols, ldc >= rows),
 * all complex128 column-major; rows <= l and cols <= m of the plan. Allocates the
 * plan's QR workspace on first use. Synchronizes the plan's stream.
 * Errors: EINVAL, ESTATE, ENOMEM, ETIMEOUT, ECUDA. */
minnorm_status minnorm_trailing_products(minnorm_plan_t plan, const void *V, int64_t ldv, void *C, int64_t ldc,
                                         int64_t rows, int64_t cols, const void *Z, int64_t ldz, void *W);

/* The schedule choices of the plan's autotuner: *x_chunks column chunks of
 * b - A x and *x_splits row splits of x = A^* y in the exact residual, and
 * *cg_l2_keep_pct, the share of L2 (percent) into which the fused CG loads the
 * tail of each sweep over A for the next, reversed sweep. A plan picks them by
 * timing the candidates on its first residual and its first inner solve (CUDA
 * events on its stream; every candidate gives the same bits) and keeps the
 * choices for later plans of the same shape in this process. Returns ESTATE
 * (with the defaults) while the plan has not yet run a residual. Errors: EINVAL. */
minnorm_status minnorm_plan_tuning(minnorm_plan_t plan, int32_t *x_chunks, int32_t *x_splits,
                                   int32_t *cg_l2_keep_pct);

/* Number of kernels this library has launched in the calling process so far
 * (host-side count of every launch it enqueues, on any plan). */
int64_t minnorm_launch_count(void);

/* Kernel timing since the last minnorm_sketch when the plan has
 * MINNORM_FLAG_TIMING: for kernel class k (0: CG product A^* w, or both
 * products in one pass over A for mixed-precision plans with 512 < m <= 4096,
 * 1: CG product A q of the two-pass form, 2: an exact residual (x = A^* y and b - A x), 3: the QR of Y (the
 * pivoted QR when l <= 2048; for taller sketches the blocked QR without
 * pivoting), 4: sketch (both chains and the FFT), 5: fused CG solves, 6: the
 * pivoted QR of the m x m triangle (taller sketches only), 7: P R^{-1}) the
 * number of timed regions (for k = 5: the CG iterations run inside them) and
 * their summed milliseconds (CUDA events on the plan's stream). Classes 0 and
 * 1 count launches enqueued: the two-pass CG enqueues its iterations in chunks,
 * and the launches after its test has fired return at once, so those counts
 * may exceed the CG iterations of minnorm_info. Errors: EINVAL (k outside
 * 0..7). */
minnorm_status minnorm_kernel_stats(minnorm_plan_t plan, int32_t k, int32_t *launches, double *ms);

/* ------------------------------------------------------------------------
 * Allocation-free entry point. The paper has no counterpart: this is the
 * pivoted QR of Step 2 offered to callers that cannot allocate device memory
 * (their memory belongs to another allocator, e.g. a framework's caching
 * allocator or a pool fixed at start-up, or they run on a latency-critical
 * path where cudaMalloc/cudaFree may synchronize the device).
 *
 * Y P = Q R for Y (device, l x m complex128, column-major, ldy == l, l >= m),
 * computed by the same kernel as minnorm_sketch's Step 2. Y is overwritten
 * (used as workspace). Writes R (device, m x m complex128, column-major, upper
 * triangular, real diagonal) and the pivots (device, m int64: column k of R
 * belongs to column piv[k] of Y). The kernel's scratch lives in one fixed
 * device array of 192 KiB inside the library, held by every GPU that loads
 * the library until the process exits; m may be at most 4096, larger m
 * returns MINNORM_ENOTSUP. Nothing is allocated: no cudaMalloc or cudaFree is
 * called. The first call on a device looks up that array's device address
 * (once per device), so make it before any stream capture. All calls share
 * the array: calls whose work may overlap on the GPU (other streams, other
 * host threads) race and must be serialized by the caller. Work is enqueued
 * on `stream` (cudaStream_t as void*); the call synchronizes it to read the
 * barrier's status. Errors: EINVAL (null pointers, sizes, Y or R_out not
 * 16-byte aligned, piv_out not 8-byte aligned), ENOTSUP (m > 4096),
 * ETIMEOUT (a bounded wait between the kernel's steps expired), ECUDA. */
minnorm_status minnorm_qr_noalloc(void *Y, int64_t ldy, int64_t l, int64_t m, void *R_out, void *piv_out,
                                  void *stream);

#ifdef __cplusplus
}
#endif

#endif
