/*
 * mpir.h -- C ABI of libmpir.so: mixed-precision iterative refinement for
 * least squares with linear equality constraints (LSE) and generalized
 * least squares (GLS) on one NVIDIA GB300 (sm_103a).
 *
 * Method: Gao, Ma, Shao, "Mixed precision iterative refinement for least
 * squares with linear equality constraints and generalized least squares
 * problems".  A generalized RQ (LSE) or QR (GLS) factorization is computed
 * once at a low precision u_f and reused to refine the solution of the
 * 3-block augmented system to FP64 accuracy (Sec. 3, Alg. 1-4).
 *
 * Conventions shared by every entry point
 * ---------------------------------------
 *  - Matrices are FP64, column-major, with a leading dimension (LAPACK
 *    convention: element (i, j) of A is A[i + j*lda]); lda >= max(1, rows).
 *  - Unless stated otherwise every pointer is a DEVICE pointer owned by the
 *    caller.  Inputs are const and never modified (unlike LAPACK xGGLSE /
 *    xGGGLM, which overwrite A, B and the right-hand sides).
 *  - Work is enqueued on the handle's stream; calls return after enqueueing
 *    unless the refinement loop needs a host decision (the classical loop
 *    reads a 4-byte convergence flag back once per iteration).  The info
 *    struct is a HOST pointer and is complete when the call returns.
 *    Internally a factorization also uses streams the handle owns (a
 *    high-priority stream for the critical path, a side stream for the
 *    aggregated compact-WY factors, one for the selector); before a call
 *    returns, all of its work is ordered before the handle's stream's
 *    subsequent work, so the caller sees one stream.
 *  - Return codes follow LAPACK's info: 0 success; -i argument i illegal
 *    (checked on the host before anything is launched); positive values
 *    are MPIR_* status codes below.
 *  - The handle owns a workspace (grown on demand with cudaMalloc unless the
 *    caller provides one with mpir_set_workspace), the factors of the last
 *    factorization, and device scratch for reductions.  One handle must not
 *    be used from two host threads at once.
 */
#ifndef MPIR_H
#define MPIR_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

/* Factorization precision u_f (Sec. 3).  The panels are FP32 for the three
 * low-precision kinds; the tensor-core trailing updates use three TF32
 * products (MPIR_FP32, FP32-accurate), one TF32 product (MPIR_TF32) or one
 * bfloat16 product (MPIR_BF16: tcgen05 kind::f16, FP32 accumulation).  For
 * MPIR_TF32 and MPIR_BF16 only the dominant factorization (the QR of A Q^T
 * for LSE, the RQ of Q^T V for GLS) runs at that precision; the first one
 * (RQ of B with Q applied to A, QR of W with Q^T applied to V) stays
 * FP32-class, and LSE factors those of (A D, B D) with a power-of-two column
 * scaling D (x = D y).  MPIR_FP64 is the fixed-precision FP64 path. */
typedef enum {
    MPIR_BF16 = 0,
    MPIR_TF32 = 1,
    MPIR_FP32 = 2,
    MPIR_FP64 = 3,
    MPIR_AUTO = 4   /* the learned selector picks the precision and the
                       refinement variant (mpir_selector_set)                 */
} mpir_prec;

/* Refinement variant. */
typedef enum {
    MPIR_CLASSICAL = 0,   /* classical IR (Alg. 2 / Alg. 4)                      */
    MPIR_GMRES = 1,       /* GMRES-IR with the block-diagonal split preconditioner
                             (Sec. 5.2, 5.3; wide shapes: eq. lse-bdpre-nlarge,
                             gls-bdpre-nlarge)                                    */
    MPIR_DIRECT = 2,      /* no refinement: null-space / Paige solve at u_f       */
    MPIR_GMRES_LEFT = 3   /* GMRES-IR with the left preconditioner M ~ F~^-1 applied
                             by the correction solver on the held factors
                             (Sec. 5.1); every shape                              */
} mpir_refine;

/* Status codes (positive return values and mpir_info.status). */
enum {
    MPIR_OK = 0,
    MPIR_SINGULAR_R = 1,      /* R (from B, or from W) has a zero diagonal       */
    MPIR_SINGULAR_T = 2,      /* T11 (LSE) / T22 (GLS) has a zero diagonal       */
    MPIR_NOT_CONVERGED = 3,   /* maxit reached without meeting the stop test     */
    MPIR_NONFINITE = 4,       /* non-finite residual or input                    */
    MPIR_UNSUPPORTED = 5,     /* size or option outside what the library handles */
    MPIR_CUDA_ERROR = 6,      /* a CUDA call failed (message: mpir_last_error)   */
    MPIR_DEVICE_TIMEOUT = 7   /* a bounded device-side wait gave up              */
};

typedef struct {
    int fact;          /* mpir_prec, default MPIR_FP32                            */
    int refine;        /* mpir_refine, default MPIR_CLASSICAL                     */
    double tol;        /* stop-test tolerance (eq. lse-stop / gls-stop); <= 0:
                          1e-15 (about 9 u: with the stop ratios below it the
                          forward error stays below 10 kappa u down to
                          kappa = 1)                                              */
    int maxit;         /* refinement steps, <= 0: 40 (Alg. 2 / Alg. 4 default)    */
    int restart;       /* GMRES restart length, <= 0: 30                          */
    int inner_maxit;   /* GMRES iterations per outer step, <= 0: 300              */
    double inner_tol;  /* GMRES relative residual target, <= 0: 1e-8 (FP32 u_f),
                          1e-4 (BF16/TF32 u_f)                                    */
    double alpha;      /* F~ scaling alpha (Sec. 5), <= 0: ||r0|| (LSE) / ||y0||
                          (GLS), floored at sqrt(u) ||A||_F ||x0|| (||V||_F ||z0||),
                          1 if both are zero                                      */
    double beta;       /* F~ scaling beta, <= 0: 1                                */
    int escalate;      /* nonzero: on failure re-factor at the next higher
                          precision up to FP64 (default 1)                         */
    int resid_dd;      /* nonzero: residuals in double-double (u_r = u^2 < u,
                          Table 2's third row): after the stop test is met the
                          refinement continues until ||dx|| <= 4 u ||x|| or the
                          corrections stop halving, so the forward error
                          reaches about u rather than kappa u.  Host-driven
                          loop; FP64 products with error-free transformations
                          (default 0)                                             */
} mpir_opts;

typedef struct {
    int status;            /* MPIR_* code of the final attempt                    */
    int iters;             /* outer refinement steps taken                        */
    int inner_iters;       /* total GMRES iterations                              */
    int fact_used;         /* mpir_prec of the factorization that produced x      */
    int refine_used;       /* mpir_refine used                                    */
    int escalated;         /* number of escalations                               */
    double stop_ratio[3];  /* ||f_i|| / (its eq. lse-stop / gls-stop bound)       */
    double time_ms[6];     /* factor, init, residual, correction, gmres, other    */
} mpir_info;

typedef struct mpir_ctx *mpir_handle;

/* Defaults as documented in mpir_opts. */
void mpir_default_opts(mpir_opts *opts);

/* Create a handle bound to device `device` (the current device if < 0) and
 * CUDA stream `stream` (a cudaStream_t, NULL = legacy default stream).
 * Returns 0 or MPIR_CUDA_ERROR.  Creation and destruction leave the caller's
 * current device as it was; every other call on a handle must be made with
 * the handle's device current (the convention of CUDA library handles). */
int mpir_create(mpir_handle *handle, int device, void *stream);
int mpir_destroy(mpir_handle handle);
/* Later calls run on `stream`; it first waits for the work already queued
 * on the handle's previous stream (and the handle's internal streams). */
int mpir_set_stream(mpir_handle handle, void *stream);

/* Caller-provided device workspace (e.g. a framework allocation).  The
 * handle then never calls cudaMalloc for the workspace.  bytes must be at
 * least what the *_workspace_size queries return; ptr 256-byte aligned.
 * Factors held from an earlier mpir_*_factor are dropped (the step-level
 * calls then return MPIR_UNSUPPORTED until the next factorization); the same
 * holds after a call that grows the handle's own workspace. */
int mpir_set_workspace(mpir_handle handle, void *ptr, size_t bytes);

/* Workspace a solve of the given shape needs (bytes). */
int mpir_lse_workspace_size(int m, int n, int p, const mpir_opts *opts, size_t *bytes);
int mpir_gls_workspace_size(int n, int m, int p, const mpir_opts *opts, size_t *bytes);

/* Last error message of this handle (static storage, never NULL).  When a
 * call returned MPIR_UNSUPPORTED because a size or launch-shape limit of a
 * kernel refused it, and nothing more specific was recorded, the message is
 * that limit's source location (file:line). */
const char *mpir_last_error(mpir_handle handle);

/* ---------------------------------------------------------------------
 * LSE:  min ||A x - b||_2  s.t.  B x = d          (eq. problem:lse, Sec. 1)
 *   A m x n (lda), B p x n (ldb), b (m), d (p), with p <= n <= m + p and,
 *   for a unique solution, rank(B) = p and rank([A; B]) = n.
 * Outputs: x (n); optionally r = b - A x (m) and the multiplier v (p) with
 * A^T r = B^T v (eq. aug-LSE); r and v may be NULL.
 * Algorithm: GRQ B = [0 R] Q, A = Z T Q at u_f, null-space start, then
 * Alg. 2 (classical), GMRES-IR with the split (Sec. 5.2) or the left
 * (Sec. 5.1) preconditioner, FP64 residuals and updates.
 * ------------------------------------------------------------------- */
int lse_solve(mpir_handle h, int m, int n, int p,
              const double *A, int lda, const double *B, int ldb,
              const double *b, const double *d,
              double *x, double *r, double *v,
              const mpir_opts *opts, mpir_info *info);

/* ---------------------------------------------------------------------
 * GLS:  min ||y||_2  s.t.  W x + V y = d          (eq. problem:gls, Sec. 1)
 *   W n x m (ldw), V n x p (ldv), d (n), with m <= n <= m + p, rank(W) = m,
 *   rank([W, V]) = n (LAPACK xGGGLM's (A, B) = (W, V)).
 * Outputs: x (m), y (p), optionally z (n) with y = V^T z, W^T z = 0.
 * Algorithm: GQR W = Q [R; 0], V = Q T Z at u_f, Paige's method, then
 * Alg. 4 (classical), GMRES-IR with the split (Sec. 5.3) or the left
 * (Sec. 5.1) preconditioner.
 * ------------------------------------------------------------------- */
int gls_solve(mpir_handle h, int n, int m, int p,
              const double *W, int ldw, const double *V, int ldv,
              const double *d, double *x, double *y, double *z,
              const mpir_opts *opts, mpir_info *info);

/* ---------------------------------------------------------------------
 * Complex LSE / GLS: the problems above over C (Sec. 1), with conjugate
 * transposes (A^H r = B^H v; y = V^H z, W^H z = 0).  Every complex array is
 * double complex in the interleaved (re, im) layout of cuDoubleComplex /
 * std::complex<double>, column-major, with leading dimensions counted in
 * complex elements; the pointers are typed double * (two doubles per
 * entry).  Dimension rules, return codes and options as lse_solve /
 * gls_solve.
 * Algorithm: the real 2 x 2 block embedding E(Z) = [Re Z, -Im Z; Im Z,
 * Re Z] (an isometry C^k -> R^2k that maps Z^H to E(Z)^T and keeps every
 * singular value) turns the problem into the real one of twice the
 * dimensions with solution [Re x; Im x]; that problem runs the real path
 * (GRQ / GQR, classical or GMRES-IR, escalation).  The handle allocates the
 * embedded copy (16 (mn + pn) + O(m + n + p) bytes for zlse_solve) when it
 * grows; the call synchronizes the handle's stream before returning.
 * ------------------------------------------------------------------- */
int zlse_solve(mpir_handle h, int m, int n, int p,
               const double *A, int lda, const double *B, int ldb,
               const double *b, const double *d,
               double *x, double *r, double *v,
               const mpir_opts *opts, mpir_info *info);
int zgls_solve(mpir_handle h, int n, int m, int p,
               const double *W, int ldw, const double *V, int ldv,
               const double *d, double *x, double *y, double *z,
               const mpir_opts *opts, mpir_info *info);

/* ---------------------------------------------------------------------
 * Batched solves of independent problems of uneven sizes.  All size, ld
 * and pointer arrays are HOST arrays of length `count`; the matrices and
 * vectors they point to are device memory.  infos (host, count entries,
 * may be NULL) receives per-problem results; the return value is the
 * largest status, or -3 (message: which problem, which argument) when a
 * problem's arguments are illegal as for lse_solve.
 * lse_solve_batched runs every problem in one persistent launch (each CTA
 * takes problems largest-first from a device queue and runs the GRQ, the
 * null-space start and classical IR on it; FP32 factors for the BF16 / TF32
 * / FP32 kinds, FP64 factors for MPIR_FP64), replayed from a CUDA graph
 * captured once per batch shape; the CTA shape is picked by timing the
 * candidates on a sample of the batch the first time a shape is seen.
 * Problems that do not converge are re-solved one by one with an FP64
 * factorization when opts->escalate is set (info.escalated = 1).
 * refine = MPIR_GMRES or MPIR_GMRES_LEFT, fact = MPIR_AUTO and resid_dd solve
 * the problems one by one with lse_solve.
 * The handle's stream is synchronized before returning.
 * ------------------------------------------------------------------- */
int lse_solve_batched(mpir_handle h, int count, const int *m, const int *n,
                      const int *p, const double *const *A, const int *lda,
                      const double *const *B, const int *ldb,
                      const double *const *b, const double *const *d,
                      double *const *x, const mpir_opts *opts,
                      mpir_info *infos);

/* Launch shapes of lse_solve_batched.  The problems of a call are split in
 * two size buckets: bucket 0 (problems whose factors and vectors need more
 * than a quarter of a CTA's shared memory) and bucket 1 (the others).  Each
 * bucket runs as 512-thread CTAs split into groups of 512, 256, 128 or 64
 * threads, one problem per group; the group size is picked by timing every
 * shape that fits on a sample of the bucket the first time the bucket's
 * signature is seen (kept per handle).  set_shape(h, g) forces group size g
 * for every bucket (where it fits; 0 restores the timing); get_shape
 * reports the shape the last call used for a bucket (group 0 and problems 0
 * for an empty bucket).  Return 0 or a negative argument index. */
int mpir_batched_set_shape(mpir_handle h, int group);
int mpir_batched_get_shape(mpir_handle h, int bucket, int *group, size_t *smem_bytes,
                           int *problems);

/* GLS analogue of lse_solve_batched (arrays of device pointers and sizes,
 * per-problem infos, worst status returned).  The problems are solved one
 * after the other with gls_solve on the handle's stream; the persistent
 * batched kernel covers LSE only. */
int gls_solve_batched(mpir_handle h, int count, const int *n, const int *m,
                      const int *p, const double *const *W, const int *ldw,
                      const double *const *V, const int *ldv,
                      const double *const *d, double *const *x,
                      double *const *y, const mpir_opts *opts,
                      mpir_info *infos);

/* Complex batches (arrays as in zlse_solve / zgls_solve, pointers typed
 * double *, leading dimensions in complex elements): every problem is
 * embedded as in zlse_solve into the handle's embedding buffer (one
 * launch), the real batched solver runs on the embedded batch, and x (and
 * y) are read back (one launch).  Status codes and infos as the real calls. */
int zlse_solve_batched(mpir_handle h, int count, const int *m, const int *n,
                       const int *p, const double *const *A, const int *lda,
                       const double *const *B, const int *ldb,
                       const double *const *b, const double *const *d,
                       double *const *x, const mpir_opts *opts, mpir_info *infos);
int zgls_solve_batched(mpir_handle h, int count, const int *n, const int *m,
                       const int *p, const double *const *W, const int *ldw,
                       const double *const *V, const int *ldv,
                       const double *const *d, double *const *x, double *const *y,
                       const mpir_opts *opts, mpir_info *infos);

/* =====================================================================
 * Step-level entry points: one per stage of the method, so that each can
 * be checked and timed on its own.  They operate on the factors held by
 * the handle (the last *_factor call).
 * ===================================================================== */

/* Stage 1-4 (LSE): scale and convert A, B, compute the GRQ at `fact`
 * precision and keep it in the handle (Lemma 4.5: RQ of B, A Q^T, QR of
 * A Q^T).  Returns MPIR_SINGULAR_R / MPIR_SINGULAR_T on a zero diagonal. */
int mpir_lse_factor(mpir_handle h, int m, int n, int p,
                    const double *A, int lda, const double *B, int ldb,
                    int fact);

/* Stage 1-4 (GLS): GQR of (W, V) (Lemma 4.6: QR of W, Q^T V, RQ of Q^T V). */
int mpir_gls_factor(mpir_handle h, int n, int m, int p,
                    const double *W, int ldw, const double *V, int ldv,
                    int fact);

/* Dense FP64 copies of the held factors' triangles in the paper's layout:
 * LSE: R (p x p, ldr) and T (m x n, ldt, zero below the diagonal);
 * GLS: R (m x m) and T (n x p, RQ-upper-trapezoidal).  Device pointers. */
int mpir_get_RT(mpir_handle h, double *R, int ldr, double *T, int ldt);

/* Apply an orthogonal factor of the held factorization to a device FP64
 * vector in place: which = 0 -> Q, 1 -> Z (the paper's names); trans = 1
 * applies the transpose.  Vector lengths: LSE Q: n, Z: m; GLS Q: n, Z: p. */
int mpir_apply_factor(mpir_handle h, int which, int trans, double *vec);

/* Stage 5 (LSE): null-space method at u_f (Sec. 2.1) -> x0 (n). */
int mpir_lse_initial(mpir_handle h, const double *b, const double *d, double *x);
/* Stage 5 (GLS): Paige's method at u_f (Sec. 2.2) -> x0 (m), y0 (p). */
int mpir_gls_initial(mpir_handle h, const double *d, double *x, double *y);

/* Stage 6 (LSE): r0 = b - A x0 in FP64, R^T v0 = (Q A^T r0)(n-p+1:n)
 * (Alg. 2 steps 3-4).  A, b as given to the factorization. */
int mpir_lse_multipliers(mpir_handle h, const double *A, int lda,
                         const double *b, const double *x, double *r,
                         double *v);
/* Stage 6 (GLS): T22^T h = (Z y)(p-n+m+1:p), z0 = Q [0; h] (Alg. 4 step 3,
 * read with Q in front, since W^T z = 0 and y = V^T z). */
int mpir_gls_multipliers(mpir_handle h, const double *y, double *z);

/* Stage 7-8: FP64 residual of the 3-block augmented system and the norms
 * of the stop test.  LSE (eq. aug-LSE, Alg. 2 step 6):
 *   f1 = b - r - A x (m), f2 = d - B x (p), f3 = -A^T r + B^T v (n).
 * norms (host array of 8, may be NULL): ||f1||, ||f2||, ||f3||, ||x||,
 * ||r||, ||v||, ||A||_F, ||B||_F.  One read of A and of B. */
int mpir_lse_residual(mpir_handle h, int m, int n, int p,
                      const double *A, int lda, const double *B, int ldb,
                      const double *b, const double *d, const double *x,
                      const double *r, const double *v,
                      double *f1, double *f2, double *f3, double *norms);
/* GLS (eq. aug-GLS, Alg. 4 step 5): f1 = -y + V^T z (p),
 * f2 = d - W x - V y (n), f3 = W^T z (m).  norms: ||f1||, ||f2||, ||f3||,
 * ||x||, ||y||, ||z||, ||W||_F, ||V||_F. */
int mpir_gls_residual(mpir_handle h, int n, int m, int p,
                      const double *W, int ldw, const double *V, int ldv,
                      const double *d, const double *x, const double *y,
                      const double *z, double *f1, double *f2, double *f3,
                      double *norms);

/* Stage 9: correction solve with the held low-precision factors.
 * LSE (Alg. 1): [I 0 A; 0 0 B; A^T B^T 0][dr; -dv; dx] = [f1; f2; f3].
 * GLS (Alg. 3, read with T22 g2 = u2 and dz = -Q h):
 *   [I V^T 0; V 0 W; 0 W^T 0][dy; -dz; dx] = [f1; f2; f3].
 * FP64 in and out; the arithmetic runs at the factor precision. */
int mpir_lse_correction(mpir_handle h, const double *f1, const double *f2,
                        const double *f3, double *dr, double *dv, double *dx);
int mpir_gls_correction(mpir_handle h, const double *f1, const double *f2,
                        const double *f3, double *dy, double *dz, double *dx);

/* GMRES-IR building blocks (Sec. 5.2 / 5.3) on the held factors: the
 * scaled augmented operator and the block-diagonal split preconditioners,
 * in FP64 arithmetic on FP64 vectors (factors read in their storage
 * precision).  which: 0 -> F~(alpha, beta) u, 1 -> M_l u, 2 -> M_r u,
 * 3 -> M_l F~ M_r u; 4 -> M u, 5 -> M F~ u with the left preconditioner
 * M ~ F~^-1 of Sec. 5.1 (eq. lse-leftpre / gls-leftpre: the correction
 * solver, Alg. 1 / Alg. 3, on the held factors; every shape).
 * LSE: vectors of length m + p + n ordered [m; p; n],
 *   F~ = [a I, 0, A; 0, 0, b B; A^T, b B^T, 0],
 *   M_l = diag(a^-1/2 I, a^-1/2 b^-1 S R^-1, a^1/2 T1^-T Q),
 *   M_r = diag(a^-1/2 I, a^-1/2 b^-1 R^-T S^T, a^1/2 Q^T T1^-1),
 *   T1 the leading n x n of T, S its trailing p x p; when n > m, T is
 *   m x n and T1 = [T; 0, I_{n-m}] (eq. lse-bdpre-nlarge).
 * GLS: vectors of length p + n + m ordered [p; n; m],
 *   F~ = [a I, V^T, 0; V, 0, b W; 0, b W^T, 0],
 *   M_l = diag(a^-1/2 I, a^1/2 T2^-1 Q^T, a^-1/2 b^-1 S^T R^-T),
 *   M_r = diag(a^-1/2 I, a^1/2 Q T2^-T, a^-1/2 b^-1 R^-1 S),
 *   T = [0, T2], S the leading m x m of T2; when n > p, T = [T^1; T^2] is
 *   n x p and T2 = [I_{n-p}, T^1; 0, T^2] (eq. gls-bdpre-nlarge).
 * A, B (W, V): the FP64 matrices that were factored.  alpha, beta > 0.
 * in, out: device arrays, distinct.  Returns 0, a negative argument index,
 * or MPIR_UNSUPPORTED (no matching factors held). */
int mpir_lse_bd_apply(mpir_handle h, const double *A, int lda, const double *B, int ldb,
                      double alpha, double beta, int which, const double *in, double *out);
int mpir_gls_bd_apply(mpir_handle h, const double *W, int ldw, const double *V, int ldv,
                      double alpha, double beta, int which, const double *in, double *out);

/* Stage 2-4 building block (xLARFB with a 128-reflector block on the
 * tensor cores): C <- (I - V X V^T) C with X = T^T (trans = 1) or T
 * (trans = 0).  V: the unit lower trapezoid of the M x K panel at V (ldv;
 * entries on and above the diagonal are ignored, the diagonal is taken as
 * 1), T: K x K upper triangular, column-major with leading dimension 128,
 * C: M x N (ldc a multiple of 4, C 16-byte aligned).  All FP32 device
 * arrays, K <= 128.  prec: MPIR_FP32 (three TF32 products, FP32-class) or
 * MPIR_TF32 (one TF32 product) or MPIR_BF16 (one bfloat16 product, FP32
 * accumulation).  Returns 0, a negative argument index, or
 * MPIR_UNSUPPORTED.  Uses the handle's workspace as scratch: factors held
 * from an earlier mpir_*_factor are dropped. */
int mpir_larfb(mpir_handle h, int prec, int M, int N, int K, const float *V, int ldv,
               const float *T, int trans, float *C, int ldc);

/* GLS residual without any allocation.  The paper has no counterpart: this
 * is an interface for callers that cannot call cudaMalloc -- framework
 * plug-ins whose host owns every device allocation through its own pool, and
 * real-time loops that must not enter the driver's allocator.
 * Same arithmetic and outputs as mpir_gls_residual (f1, f2, f3 as there;
 * norms2: a DEVICE array of 6 doubles receiving the squared norms of f1, f2,
 * f3, x, y, z, or NULL), enqueued on `stream` (a cudaStream_t), without a
 * handle.  Its scratch is a fixed file-scope device array of 4 MiB
 * (524288 doubles) that every GPU loading the library holds until the
 * process exits; shapes whose partial sums exceed it
 * (ceil(m/256)*n + ceil(n/256)*m + ceil(p/256)*n + ceil(n/256)*p + 1832
 * doubles; e.g. n = m = p = 4096 needs 264k) return MPIR_UNSUPPORTED.
 * The first call on a device looks the array's address up
 * (cudaGetSymbolAddress) with that device current.  The address is kept
 * for the life of the
 * process (concurrent first calls from several host threads are safe): a
 * cudaDeviceReset of that device, which also frees every handle's memory,
 * ends the library's use of the device in this process.  Every call shares the one array and leaves
 * its contents behind, so calls whose GPU work overlaps (two streams, two
 * host threads) race and must be serialized by the caller.  Returns 0, a
 * negative argument index, MPIR_UNSUPPORTED or MPIR_CUDA_ERROR. */
int mpir_gls_residual_noalloc(int n, int m, int p, const double *W, int ldw,
                              const double *V, int ldv, const double *d,
                              const double *x, const double *y, const double *z,
                              double *f1, double *f2, double *f3, double *norms2,
                              void *stream);

/* =====================================================================
 * Learned selector (not in the paper): picks, per problem, the
 * factorization precision {BF16, FP32, FP64} and the refinement variant
 * {classical, GMRES} (6 classes, in that order: BF16+classical,
 * BF16+GMRES, FP32+classical, FP32+GMRES, FP64+classical, FP64+GMRES).
 * ===================================================================== */

/* 16 features of a problem (device float[16]): log m, log n, log(p+1), n/m,
 * p/n, kind (0), complex flag (0), log ||A||_F, log ||B||_F, log ||b||,
 * log ||d||, log(||A||_F/||B||_F), log kappa^(A), log kappa^(B),
 * log kappa^([A; B]), log(GRQ flop estimate); kappa^ = sigma_max/sigma_min
 * of the bidiagonal of min(16, rows, columns) Golub-Kahan-Lanczos steps
 * started from s (device, length n; a wide block starts from M^T M s),
 * computed with FP32 vectors and products, each new vector reorthogonalized
 * once, stopping only at breakdown (an entry below 2^-26 of the largest),
 * the bidiagonal's extreme singular values by FP32 bisection (relative
 * error O(k u_single); kappa^ = inf below 2^-100 sigma_max).  GLS: log n,
 * log m, log(p+1), m/n, n/p, kind 1, 0, log ||W||_F, log ||V||_F, log ||d||,
 * 0, log(||W||_F/||V||_F), kappa^ of W, V, [W, V], log(flops); s has length
 * m + p (W uses s[0:m], V s[m:m+p]).  Logs are natural, of the value clamped
 * to [1e-300, 1e300].  One thread-block cluster. */
int mpir_lse_features(mpir_handle h, int m, int n, int p, const double *A, int lda,
                      const double *B, int ldb, const double *b, const double *d,
                      const double *s, float *features);
int mpir_gls_features(mpir_handle h, int n, int m, int p, const double *W, int ldw,
                      const double *V, int ldv, const double *d, const double *s,
                      float *features);

/* The MLP 16 -> 64 -> 64 -> 6 (ReLU, softmax).  params: device FP32 array
 * of mpir_mlp_param_count() floats laid out as W1[64][16], b1[64],
 * W2[64][64], b2[64], W3[6][64], b3[6] (row-major, W[o][i] maps input i to
 * output o); the kernels round the weights to bfloat16 (nearest, ties to
 * even) and accumulate in FP32.  X: device float[count][16]; prob: device
 * float[count][6]. */
int mpir_mlp_param_count(void);
int mpir_mlp_forward(mpir_handle h, const float *params, const float *X, int count, float *prob);
/* One training step on the mean cross-entropy of (X, labels) (labels: device
 * int[count] in 0..5): gradients into grad (device, param_count floats, may
 * be NULL), mean loss into *loss (device float, may be NULL), and, when
 * adam_m and adam_v (device, param_count floats each) are given and lr > 0,
 * an Adam update (beta1 0.9, beta2 0.999, eps 1e-8, bias-corrected with the
 * 1-based step count `step`) of params. */
int mpir_mlp_train_step(mpir_handle h, float *params, float *adam_m, float *adam_v, int step,
                        float lr, const float *X, const int *labels, int count, float *grad,
                        float *loss);
/* Install a trained selector in the handle (host arrays: params as above,
 * feature standardization mean[16] and scale[16]: the network sees
 * (f - mean) / scale).  Solves with opts->fact = MPIR_AUTO then compute the
 * features (start vector: splitmix64 of seed 0x5EED + j mapped to [-1, 1)),
 * run the network, and solve with the most probable class (GMRES classes
 * fall back to classical IR where the block-diagonal preconditioner does not
 * apply); escalation to FP64 stays the fallback.  The FP32 factorization
 * runs on the handle's stream while the features and the network run on a
 * stream of their own; it is kept when an FP32 class is chosen and
 * discarded otherwise.  info->fact_used / refine_used report the choice.
 * NULL params removes the selector. */
int mpir_selector_set(mpir_handle h, const float *params, const float *mean, const float *scale);

/* Library version string. */
const char *mpir_version(void);

/* Process-wide launch accounting (every kernel launch of the library is
 * counted by kind) and optional per-kind device timing: mpir_profile(1)
 * clears the records and records a CUDA event pair around every launch on
 * the launch stream; mpir_profile_read synchronizes on the last record and
 * returns, per kind, the summed event time (ms) and the number of timed
 * launches.  Kinds: 0 panel_qr, 1 larfb, 2 vec_apply, 3 trsv, 4 gemv,
 * 5 dual_gemv_fp64, 6 resid_finalize, 7 convert, 8 norm, 9 elementwise,
 * 10 larfb_tc (tcgen05 GEMM), 11 larfb_aux (V / W preparation), 12 gmres
 * (Arnoldi steps and cycle updates), 13 batched (persistent batched solves),
 * 14 selector (features and MLP kernels).
 * Launch counting is safe from any thread; the timing mode is a
 * single-threaded profiling aid, off by default. */
int mpir_profile(int enable);
int mpir_profile_read(double *ms, long long *launches, int nkinds);
long long mpir_launch_count(int kind);          /* kind < 0: all kinds */
const char *mpir_kernel_kind_name(int kind);

#ifdef __cplusplus
}
#endif

#endif /* MPIR_H */
