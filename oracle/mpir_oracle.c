/*
 * mpir_oracle.c -- plain CPU oracle for mixed-precision iterative
 * refinement of LSE and GLS problems (Gao, Ma, Shao, "Mixed precision
 * iterative refinement for least squares with linear equality constraints
 * and generalized least squares problems").
 *
 * TEST INFRASTRUCTURE ONLY.  Only tests/, the smoke check and the
 * cpu_baseline / reference leg of bench.py may load this library.  It shares
 * no code with the CUDA library: unblocked Householder, one reflector at a
 * time, FP64 (or FP32 for the u_f = single experiments), double-double
 * residuals for the truth.
 *
 * Build:  gcc -O2 -fopenmp -ffp-contract=off -fPIC -shared (oracle/build.py)
 * -ffp-contract=off keeps the error-free transformations of the
 * double-double code exact and the results identical on x86-64 and aarch64.
 */
#include <math.h>
#include <stdlib.h>
#include <string.h>
#include <omp.h>

#define IDX(i, j, ld) ((size_t)(j) * (size_t)(ld) + (size_t)(i))

/* ---------------- norms ------------------------------------------------ */

static double vnorm(int n, const double *x)
{   /* 2-norm with scaling against overflow */
    double scale = 0, ssq = 0;
    for (int i = 0; i < n; i++) { double a = fabs(x[i]); if (a > scale) scale = a; }
    if (scale == 0 || isinf(scale) || scale != scale) return scale;
    for (int i = 0; i < n; i++) { double t = x[i] / scale; ssq += t * t; }
    return scale * sqrt(ssq);
}

static double fro_norm(int rows, int cols, const double *A, int ld)
{
    double scale = 0, ssq = 0;
    for (int j = 0; j < cols; j++)
        for (int i = 0; i < rows; i++) { double a = fabs(A[IDX(i, j, ld)]); if (a > scale) scale = a; }
    if (scale == 0) return 0;
    for (int j = 0; j < cols; j++)
        for (int i = 0; i < rows; i++) { double t = A[IDX(i, j, ld)] / scale; ssq += t * t; }
    return scale * sqrt(ssq);
}

/* ---------------- double-double (Dekker / Knuth) ----------------------- */

typedef struct { double hi, lo; } dd_t;

static inline dd_t two_sum(double a, double b)
{
    double s = a + b, bb = s - a;
    dd_t r = { s, (a - (s - bb)) + (b - bb) };
    return r;
}
static inline dd_t quick_two_sum(double a, double b)
{
    double s = a + b;
    dd_t r = { s, b - (s - a) };
    return r;
}
static inline dd_t dd_add_d(dd_t a, double b)
{
    dd_t s = two_sum(a.hi, b);
    s.lo += a.lo;
    return quick_two_sum(s.hi, s.lo);
}
/* a + x*y with the product formed exactly (TwoProd through fma) */
static inline dd_t dd_add_prod(dd_t a, double x, double y)
{
    double p = x * y, e = fma(x, y, -p);
    dd_t s = two_sum(a.hi, p);
    s.lo += a.lo + e;
    return quick_two_sum(s.hi, s.lo);
}

/* acc[i] += sgn * sum_j M(i,j) x(j), i < rows, j < cols.  Rows are split
 * between threads (column-major access inside each thread). */
static void gemv_acc(int rows, int cols, const double *M, int ld,
                     const double *x, double sgn, dd_t *acc, int use_dd)
{
    #pragma omp parallel if ((size_t)rows * (size_t)cols > 65536)
    {
        int nt = omp_get_num_threads(), id = omp_get_thread_num();
        int chunk = (rows + nt - 1) / nt;
        int r0 = id * chunk, r1 = r0 + chunk < rows ? r0 + chunk : rows;
        for (int j = 0; j < cols; j++) {
            double xj = sgn * x[j];
            const double *col = &M[IDX(0, j, ld)];
            if (use_dd) for (int i = r0; i < r1; i++) acc[i] = dd_add_prod(acc[i], col[i], xj);
            else        for (int i = r0; i < r1; i++) acc[i].hi += col[i] * xj;
        }
    }
}

/* acc[j] += sgn * sum_i M(i,j) r(i), j < cols, i < rows. */
static void gemvt_acc(int rows, int cols, const double *M, int ld,
                      const double *r, double sgn, dd_t *acc, int use_dd)
{
    #pragma omp parallel for schedule(static) if ((size_t)rows * (size_t)cols > 65536)
    for (int j = 0; j < cols; j++) {
        const double *col = &M[IDX(0, j, ld)];
        dd_t a = acc[j];
        if (use_dd) for (int i = 0; i < rows; i++) a = dd_add_prod(a, col[i], sgn * r[i]);
        else        for (int i = 0; i < rows; i++) a.hi += col[i] * (sgn * r[i]);
        acc[j] = a;
    }
}

static dd_t *dd_from(int n, const double *a, double sgn)
{
    dd_t *v = (dd_t *)calloc((size_t)(n > 0 ? n : 1), sizeof(dd_t));
    if (a) for (int i = 0; i < n; i++) v[i].hi = sgn * a[i];
    return v;
}
static void dd_round(int n, const dd_t *a, double *out)
{
    for (int i = 0; i < n; i++) out[i] = a[i].hi + a[i].lo;
}

/* Residual of the 3-block LSE augmented system (eq. aug-LSE, Alg. 2 step 6):
 * f1 = b - r - A x, f2 = d - B x, f3 = -A^T r + B^T v.
 * use_dd = 1: double-double accumulation (u_r ~ 1e-32); 0: plain FP64. */
static void lse_residual(int m, int n, int p, const double *A, int lda,
                         const double *B, int ldb, const double *b,
                         const double *d, const double *x, const double *r,
                         const double *v, double *f1, double *f2, double *f3,
                         int use_dd)
{
    dd_t *a1 = dd_from(m, b, 1.0);
    for (int i = 0; i < m; i++) a1[i] = use_dd ? dd_add_d(a1[i], -r[i]) : (dd_t){ a1[i].hi - r[i], 0 };
    gemv_acc(m, n, A, lda, x, -1.0, a1, use_dd);
    dd_round(m, a1, f1);
    dd_t *a2 = dd_from(p, d, 1.0);
    gemv_acc(p, n, B, ldb, x, -1.0, a2, use_dd);
    dd_round(p, a2, f2);
    dd_t *a3 = dd_from(n, NULL, 1.0);
    gemvt_acc(m, n, A, lda, r, -1.0, a3, use_dd);
    gemvt_acc(p, n, B, ldb, v, 1.0, a3, use_dd);
    dd_round(n, a3, f3);
    free(a1); free(a2); free(a3);
}

/* Residual of the 3-block GLS augmented system (eq. aug-GLS, Alg. 4 step 5):
 * f1 = -y + V^T z, f2 = d - W x - V y, f3 = W^T z. */
static void gls_residual(int n, int m, int p, const double *W, int ldw,
                         const double *V, int ldv, const double *d,
                         const double *x, const double *y, const double *z,
                         double *f1, double *f2, double *f3, int use_dd)
{
    dd_t *a1 = dd_from(p, y, -1.0);
    gemvt_acc(n, p, V, ldv, z, 1.0, a1, use_dd);
    dd_round(p, a1, f1);
    dd_t *a2 = dd_from(n, d, 1.0);
    gemv_acc(n, m, W, ldw, x, -1.0, a2, use_dd);
    gemv_acc(n, p, V, ldv, y, -1.0, a2, use_dd);
    dd_round(n, a2, f2);
    dd_t *a3 = dd_from(m, NULL, 1.0);
    gemvt_acc(n, m, W, ldw, z, 1.0, a3, use_dd);
    dd_round(m, a3, f3);
    free(a1); free(a2); free(a3);
}

/* ---------------- templates: FP64 and FP32 instantiations -------------- */

#define REAL double
#define FN(x) x##_d
#include "hh_template.h"
#include "solve_template.h"
#undef REAL
#undef FN

#define REAL float
#define FN(x) x##_s
#include "hh_template.h"
#include "solve_template.h"
#undef REAL
#undef FN

/* ======================= exported entry points ========================= */

/* Full solves (Alg. 2 / Alg. 4).  fact_single selects u_f = u_s = FP32,
 * otherwise FP64.  Returns the status of the refinement loop. */
int or_lse_solve(int m, int n, int p, const double *A, int lda,
                 const double *B, int ldb, const double *b, const double *d,
                 double *x, double *r, double *v, int fact_single, int maxit,
                 double tol, int resid_dd, int *iters, double *ratios)
{
    if (fact_single)
        return lse_ir_s(m, n, p, A, lda, B, ldb, b, d, x, r, v, maxit, tol, resid_dd, iters, ratios);
    return lse_ir_d(m, n, p, A, lda, B, ldb, b, d, x, r, v, maxit, tol, resid_dd, iters, ratios);
}

int or_gls_solve(int n, int m, int p, const double *W, int ldw,
                 const double *V, int ldv, const double *d, double *x,
                 double *y, double *z, int fact_single, int maxit, double tol,
                 int resid_dd, int *iters, double *ratios)
{
    if (fact_single)
        return gls_ir_s(n, m, p, W, ldw, V, ldv, d, x, y, z, maxit, tol, resid_dd, iters, ratios);
    return gls_ir_d(n, m, p, W, ldw, V, ldv, d, x, y, z, maxit, tol, resid_dd, iters, ratios);
}

void or_lse_residual(int m, int n, int p, const double *A, int lda,
                     const double *B, int ldb, const double *b, const double *d,
                     const double *x, const double *r, const double *v,
                     double *f1, double *f2, double *f3, int use_dd)
{
    lse_residual(m, n, p, A, lda, B, ldb, b, d, x, r, v, f1, f2, f3, use_dd);
}

void or_gls_residual(int n, int m, int p, const double *W, int ldw,
                     const double *V, int ldv, const double *d,
                     const double *x, const double *y, const double *z,
                     double *f1, double *f2, double *f3, int use_dd)
{
    gls_residual(n, m, p, W, ldw, V, ldv, d, x, y, z, f1, f2, f3, use_dd);
}

/* Packed factors.  LSE: Bf (p x n, ld p) and Af (m x n, ld m) as left by
 * gerq2 / geqr2; GLS: Wf (n x m, ld n), Vf (n x p, ld n).  fact_single
 * computes them in FP32; they are returned widened to FP64 (exact). */
void or_lse_factor(int m, int n, int p, const double *A, int lda,
                   const double *B, int ldb, int fact_single, double *Bf,
                   double *taub, double *Af, double *taua)
{
    if (fact_single) {
        lse_fact_s F; lse_factor_s(&F, m, n, p, A, lda, B, ldb);
        for (size_t i = 0; i < (size_t)p * n; i++) Bf[i] = F.Bf[i];
        for (size_t i = 0; i < (size_t)m * n; i++) Af[i] = F.Af[i];
        for (int i = 0; i < p; i++) taub[i] = F.taub[i];
        for (int i = 0; i < (m < n ? m : n); i++) taua[i] = F.taua[i];
        lse_free_s(&F);
    } else {
        lse_fact_d F; lse_factor_d(&F, m, n, p, A, lda, B, ldb);
        memcpy(Bf, F.Bf, sizeof(double) * (size_t)p * n);
        memcpy(Af, F.Af, sizeof(double) * (size_t)m * n);
        memcpy(taub, F.taub, sizeof(double) * (size_t)p);
        memcpy(taua, F.taua, sizeof(double) * (size_t)(m < n ? m : n));
        lse_free_d(&F);
    }
}

void or_gls_factor(int n, int m, int p, const double *W, int ldw,
                   const double *V, int ldv, int fact_single, double *Wf,
                   double *tauw, double *Vf, double *tauv)
{
    int kv = n < p ? n : p;
    if (fact_single) {
        gls_fact_s F; gls_factor_s(&F, n, m, p, W, ldw, V, ldv);
        for (size_t i = 0; i < (size_t)n * m; i++) Wf[i] = F.Wf[i];
        for (size_t i = 0; i < (size_t)n * p; i++) Vf[i] = F.Vf[i];
        for (int i = 0; i < m; i++) tauw[i] = F.tauw[i];
        for (int i = 0; i < kv; i++) tauv[i] = F.tauv[i];
        gls_free_s(&F);
    } else {
        gls_fact_d F; gls_factor_d(&F, n, m, p, W, ldw, V, ldv);
        memcpy(Wf, F.Wf, sizeof(double) * (size_t)n * m);
        memcpy(Vf, F.Vf, sizeof(double) * (size_t)n * p);
        memcpy(tauw, F.tauw, sizeof(double) * (size_t)m);
        memcpy(tauv, F.tauv, sizeof(double) * (size_t)kv);
        gls_free_d(&F);
    }
}

static lse_fact_d lse_wrap(int m, int n, int p, const double *Bf,
                           const double *taub, const double *Af,
                           const double *taua)
{
    lse_fact_d F = { m, n, p, (double *)Bf, (double *)taub, (double *)Af, (double *)taua };
    return F;
}
static gls_fact_d gls_wrap(int n, int m, int p, const double *Wf,
                           const double *tauw, const double *Vf,
                           const double *tauv)
{
    gls_fact_d F = { n, m, p, (double *)Wf, (double *)tauw, (double *)Vf, (double *)tauv };
    return F;
}

/* which = 0: Q (n-vector), 1: Z (m-vector); trans = 1 applies the transpose */
void or_lse_apply(int m, int n, int p, const double *Bf, const double *taub,
                  const double *Af, const double *taua, int which, int trans,
                  double *x)
{
    lse_fact_d F = lse_wrap(m, n, p, Bf, taub, Af, taua);
    if (which == 0) lse_apply_Q_d(&F, trans, x); else lse_apply_Z_d(&F, trans, x);
}

/* which = 0: Q (n-vector), 1: Z (p-vector) */
void or_gls_apply(int n, int m, int p, const double *Wf, const double *tauw,
                  const double *Vf, const double *tauv, int which, int trans,
                  double *x)
{
    gls_fact_d F = gls_wrap(n, m, p, Wf, tauw, Vf, tauv);
    if (which == 0) gls_apply_Q_d(&F, trans, x); else gls_apply_Z_d(&F, trans, x);
}

void or_lse_nullspace(int m, int n, int p, const double *Bf, const double *taub,
                      const double *Af, const double *taua, const double *b,
                      const double *d, double *x)
{
    lse_fact_d F = lse_wrap(m, n, p, Bf, taub, Af, taua);
    lse_nullspace_d(&F, b, d, x);
}

void or_gls_paige(int n, int m, int p, const double *Wf, const double *tauw,
                  const double *Vf, const double *tauv, const double *d,
                  double *x, double *y)
{
    gls_fact_d F = gls_wrap(n, m, p, Wf, tauw, Vf, tauv);
    gls_paige_d(&F, d, x, y);
}

void or_lse_correction(int m, int n, int p, const double *Bf,
                       const double *taub, const double *Af, const double *taua,
                       const double *f1, const double *f2, const double *f3,
                       double *dr, double *dv, double *dx)
{
    lse_fact_d F = lse_wrap(m, n, p, Bf, taub, Af, taua);
    lse_correction_d(&F, f1, f2, f3, dr, dv, dx);
}

void or_gls_correction(int n, int m, int p, const double *Wf,
                       const double *tauw, const double *Vf, const double *tauv,
                       const double *f1, const double *f2, const double *f3,
                       double *dy, double *dz, double *dx)
{
    gls_fact_d F = gls_wrap(n, m, p, Wf, tauw, Vf, tauv);
    gls_correction_d(&F, f1, f2, f3, dy, dz, dx);
}

void or_lse_init_v(int m, int n, int p, const double *Bf, const double *taub,
                   const double *Af, const double *taua, const double *A,
                   int lda, const double *r, double *v)
{
    lse_fact_d F = lse_wrap(m, n, p, Bf, taub, Af, taua);
    lse_init_v_d(&F, A, lda, r, v);
}

void or_gls_init_z(int n, int m, int p, const double *Wf, const double *tauw,
                   const double *Vf, const double *tauv, const double *y,
                   double *z)
{
    gls_fact_d F = gls_wrap(n, m, p, Wf, tauw, Vf, tauv);
    gls_init_z_d(&F, y, z);
}

/* ---------------- condition estimates ---------------------------------- */

/* y = op(U) x for the upper triangle of the n x n block U (ld). */
static void tri_mul(int n, const double *U, int ld, int trans, const double *x, double *y)
{
    for (int i = 0; i < n; i++) y[i] = 0;
    for (int j = 0; j < n; j++)
        for (int i = 0; i <= j; i++) {
            if (trans) y[j] += U[IDX(i, j, ld)] * x[i];
            else       y[i] += U[IDX(i, j, ld)] * x[j];
        }
}

/* Largest singular value of an operator K given K and K^T by power
 * iteration on K^T K (iters steps, deterministic start vector). */
typedef void (*op_fn)(void *ctx, int trans, const double *x, double *y);

static double power_sigma(int n, op_fn op, void *ctx, int iters)
{
    double *x = (double *)calloc((size_t)(n > 0 ? n : 1), sizeof(double));
    double *y = (double *)calloc((size_t)(n > 0 ? n : 1), sizeof(double));
    for (int i = 0; i < n; i++) x[i] = 1.0 + 0.5 * sin(0.7 * i + 0.3);
    double s = 0, nx = vnorm(n, x);
    for (int i = 0; i < n; i++) x[i] /= nx;
    for (int it = 0; it < iters; it++) {
        op(ctx, 0, x, y);
        op(ctx, 1, y, x);
        double nrm = vnorm(n, x);
        if (nrm == 0) { s = 0; break; }
        s = sqrt(nrm);
        for (int i = 0; i < n; i++) x[i] /= nrm;
    }
    free(x); free(y);
    return s;
}

typedef struct { int n; const double *U; int ld; const double *U2; int ld2; } tri_ctx;

static void op_tri(void *c, int trans, const double *x, double *y)
{   /* K = U */
    tri_ctx *t = (tri_ctx *)c; tri_mul(t->n, t->U, t->ld, trans, x, y);
}
static void op_tri_inv(void *c, int trans, const double *x, double *y)
{   /* K = U^{-1} */
    tri_ctx *t = (tri_ctx *)c;
    memcpy(y, x, sizeof(double) * (size_t)t->n);
    if (trans) trsv_ut_d(t->n, t->U, t->ld, y); else trsv_un_d(t->n, t->U, t->ld, y);
}
static void op_ratio(void *c, int trans, const double *x, double *y)
{   /* K = U2^{-1} U  (K^T = U^T U2^{-T}) */
    tri_ctx *t = (tri_ctx *)c;
    if (!trans) { tri_mul(t->n, t->U, t->ld, 0, x, y); trsv_un_d(t->n, t->U2, t->ld2, y); }
    else {
        double *w = (double *)malloc(sizeof(double) * (size_t)t->n);
        memcpy(w, x, sizeof(double) * (size_t)t->n);
        trsv_ut_d(t->n, t->U2, t->ld2, w);
        tri_mul(t->n, t->U, t->ld, 1, w, y);
        free(w);
    }
}
static void op_ratio_inv(void *c, int trans, const double *x, double *y)
{   /* K^{-1} = U^{-1} U2  (K^{-T} = U2^T U^{-T}) */
    tri_ctx *t = (tri_ctx *)c;
    if (!trans) { tri_mul(t->n, t->U2, t->ld2, 0, x, y); trsv_un_d(t->n, t->U, t->ld, y); }
    else {
        double *w = (double *)malloc(sizeof(double) * (size_t)t->n);
        memcpy(w, x, sizeof(double) * (size_t)t->n);
        trsv_ut_d(t->n, t->U, t->ld, w);
        tri_mul(t->n, t->U2, t->ld2, 1, w, y);
        free(w);
    }
}

static void tri_sigmas(int n, const double *U, int ld, int iters, double *smax, double *smin)
{
    tri_ctx c = { n, U, ld, NULL, 0 };
    *smax = power_sigma(n, op_tri, &c, iters);
    double inv = power_sigma(n, op_tri_inv, &c, iters);
    *smin = inv > 0 ? 1.0 / inv : 0;
}

/* Condition number used for the forward-error tolerance of an LSE solution
 * (LS sensitivity of the reduced problem of the null-space method, Sec. 2.1):
 *   kN = kappa2(T11),  kappa = max(kN (1 + kN ||r|| / (sigma_max(T11) ||x||)),
 *                                  kappa2(R)).
 * Estimated from FP64 factors by power / inverse power iteration.
 * out[0] = kappa, out[1] = kappa2(T11), out[2] = kappa2(R). */
void or_lse_kappa(int m, int n, int p, const double *Bf, const double *Af,
                  const double *x, const double *r, int iters, double *out)
{
    int q = n - p;
    double tmax = 0, tmin = 0, rmax = 1, rmin = 1;
    if (q > 0) tri_sigmas(q, Af, m, iters, &tmax, &tmin);
    if (p > 0) tri_sigmas(p, &Bf[IDX(0, q, p)], p, iters, &rmax, &rmin);
    double kN = q > 0 && tmin > 0 ? tmax / tmin : 1.0;
    double kR = rmin > 0 ? rmax / rmin : INFINITY;
    double nx = vnorm(n, x), nr = vnorm(m, r);
    double k = kN;
    if (q > 0 && nx > 0 && tmax > 0) k = kN * (1.0 + kN * nr / (tmax * nx));
    out[0] = k > kR ? k : kR;
    out[1] = kN;
    out[2] = kR;
}

/* Condition number for a GLS solution with n <= p (weighted LS
 * min ||T_sq^{-1}([R;0] x - c)||, Sec. 2.2): K = S^{-1} R with
 * S = T(1:m, p-n+1:p-n+m) (upper triangular),
 *   kG = kappa2(K),  kappa = kG (1 + kG ||y|| / (sigma_max(K) ||x||)).
 * For n > p the product kappa2(R) * kappa2(T22) is returned.
 * out[0] = kappa, out[1] = kG. */
void or_gls_kappa(int n, int m, int p, const double *Wf, const double *Vf,
                  const double *x, const double *y, int iters, double *out)
{
    if (m == 0) { out[0] = out[1] = 1.0; return; }
    if (n <= p) {
        tri_ctx c = { m, Wf, n, &Vf[IDX(0, p - n, n)], n };
        double smax = power_sigma(m, op_ratio, &c, iters);
        double sinv = power_sigma(m, op_ratio_inv, &c, iters);
        double kG = smax * sinv;
        double nx = vnorm(m, x), ny = vnorm(p, y);
        out[0] = nx > 0 ? kG * (1.0 + kG * ny / (smax * nx)) : kG;
        out[1] = kG;
    } else {
        double a, b, c2, d2;
        tri_sigmas(m, Wf, n, iters, &a, &b);
        int l = n - m, o = p - n + m;
        tri_sigmas(l, &Vf[IDX(m, o, n)], n, iters, &c2, &d2);
        out[1] = (a / b) * (c2 / d2);
        out[0] = out[1];
    }
}

int or_num_threads(void) { return omp_get_max_threads(); }
