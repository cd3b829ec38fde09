/*
 * CPU oracle -- the paper's method written out step by step, instantiated
 * once per factorization precision (REAL = double for the FP64 truth,
 * REAL = float for the u_f = single experiments of Sec. 6).
 *
 * TEST INFRASTRUCTURE ONLY (see hh_template.h).
 *
 * Notation follows Sec. 2-3 of the paper.  LSE: A m x n, B p x n,
 * p <= n <= m+p.  GLS: W n x m, V n x p, m <= n <= m+p.  All matrices are
 * column-major with leading dimensions; vectors are dense arrays.
 */

/* ---------------- LSE: generalized RQ factorization (Sec. 2.1, 4.2) ---- */

typedef struct {
    int m, n, p;
    REAL *Bf; REAL *taub;     /* RQ of B:  B = [0, R] Q, ld = p           */
    REAL *Af; REAL *taua;     /* QR of A Q^T = Z T,       ld = m          */
} FN(lse_fact);

/* Entry T(i, j) of the upper trapezoidal T (zero below the diagonal). */
static inline REAL FN(lse_T)(const FN(lse_fact) *F, int i, int j)
{
    return i <= j ? F->Af[IDX(i, j, F->m)] : (REAL)0;
}

/* GRQ of (B, A): RQ of B (xGERQF), A <- A Q^T, QR of A Q^T (xGEQRF)
 * (Lemma 4.5: "an RQ factorization B=[0,R]Q and then a QR factorization
 * AQ^H = ZT").  Q = H_{p-1}...H_0 so A Q^T = A H_0 H_1 ... H_{p-1}. */
static void FN(lse_factor)(FN(lse_fact) *F, int m, int n, int p,
                           const double *A, int lda, const double *B, int ldb)
{
    F->m = m; F->n = n; F->p = p;
    F->Bf = (REAL *)malloc(sizeof(REAL) * (size_t)(p > 0 ? p : 1) * (size_t)n);
    F->Af = (REAL *)malloc(sizeof(REAL) * (size_t)m * (size_t)n);
    F->taub = (REAL *)calloc((size_t)(p > 0 ? p : 1), sizeof(REAL));
    F->taua = (REAL *)calloc((size_t)(n > 0 ? n : 1), sizeof(REAL));
    for (int j = 0; j < n; j++) {
        for (int i = 0; i < p; i++) F->Bf[IDX(i, j, p)] = (REAL)B[IDX(i, j, ldb)];
        for (int i = 0; i < m; i++) F->Af[IDX(i, j, m)] = (REAL)A[IDX(i, j, lda)];
    }
    FN(gerq2)(p, n, F->Bf, p, F->taub);
    for (int g = 0; g < p; g++) {
        int r = p - 1 - g, c = n - 1 - g;
        FN(apply_right)(m, c, F->Af, m, &F->Bf[IDX(r, 0, p)], (size_t)p, F->taub[g]);
    }
    FN(geqr2)(m, n, F->Af, m, F->taua);
}

static void FN(lse_free)(FN(lse_fact) *F)
{
    free(F->Bf); free(F->Af); free(F->taub); free(F->taua);
}

static inline void FN(lse_apply_Q)(const FN(lse_fact) *F, int trans, REAL *x)
{   /* trans = 0: x <- Q x ; trans = 1: x <- Q^T x */
    FN(rq_apply_vec)(F->p, F->n, F->p, F->Bf, F->p, F->taub, trans, x);
}
static inline void FN(lse_apply_Z)(const FN(lse_fact) *F, int trans, REAL *x)
{   /* trans = 0: x <- Z x ; trans = 1: x <- Z^T x */
    int k = F->m < F->n ? F->m : F->n;
    FN(qr_apply_vec)(F->m, k, F->Af, F->m, F->taua, trans, x);
}

/* Null-space method (Sec. 2.1): R y2 = d; T11 y1 = c1 - T12 y2 with
 * c = Z^T b; x = Q^T [y1; y2].  All at precision REAL. */
static void FN(lse_nullspace)(const FN(lse_fact) *F, const double *b,
                              const double *d, double *x)
{
    int m = F->m, n = F->n, p = F->p, q = n - p;
    REAL *c = (REAL *)malloc(sizeof(REAL) * (size_t)m);
    REAL *y = (REAL *)malloc(sizeof(REAL) * (size_t)n);
    for (int i = 0; i < m; i++) c[i] = (REAL)b[i];
    FN(lse_apply_Z)(F, 1, c);
    for (int i = 0; i < p; i++) y[q + i] = (REAL)d[i];
    FN(trsv_un)(p, &F->Bf[IDX(0, q, p)], p, y + q);
    for (int i = 0; i < q; i++) {
        REAL s = c[i];
        for (int j = 0; j < p; j++) s -= FN(lse_T)(F, i, q + j) * y[q + j];
        y[i] = s;
    }
    FN(trsv_un)(q, F->Af, m, y);
    FN(lse_apply_Q)(F, 1, y);
    for (int i = 0; i < n; i++) x[i] = (double)y[i];
    free(c); free(y);
}

/* Algorithm 1 (CorrectionSystemSolverLSE), all steps at precision REAL.
 * Solves [I 0 A; 0 0 B; A^T B^T 0][x1; -x2; x3] = [f1; f2; f3] with the
 * GRQ factors.  Outputs x1 = dr (m), x2 = dv (p), x3 = dx (n). */
static void FN(lse_correction)(const FN(lse_fact) *F, const double *f1,
                               const double *f2, const double *f3,
                               double *dr, double *dv, double *dx)
{
    int m = F->m, n = F->n, p = F->p, q = n - p;
    REAL *u = (REAL *)malloc(sizeof(REAL) * (size_t)n);
    REAL *w = (REAL *)malloc(sizeof(REAL) * (size_t)m);
    REAL *y = (REAL *)malloc(sizeof(REAL) * (size_t)n);
    REAL *qv = (REAL *)malloc(sizeof(REAL) * (size_t)m);
    REAL *t = (REAL *)malloc(sizeof(REAL) * (size_t)(p > 0 ? p : 1));
    for (int i = 0; i < n; i++) u[i] = (REAL)f3[i];
    FN(lse_apply_Q)(F, 0, u);                            /* step 1: u = Q f3   */
    for (int i = 0; i < m; i++) w[i] = (REAL)f1[i];
    FN(lse_apply_Z)(F, 1, w);                            /* step 2: w = Z^T f1 */
    for (int i = 0; i < p; i++) y[q + i] = (REAL)f2[i];
    FN(trsv_un)(p, &F->Bf[IDX(0, q, p)], p, y + q);      /* step 3: R y2 = f2  */
    for (int i = 0; i < q; i++) qv[i] = u[i];
    FN(trsv_ut)(q, F->Af, m, qv);                        /* step 4: T11^T q1 = u1 */
    for (int i = 0; i < q; i++) {                        /* step 5 */
        REAL s = w[i] - qv[i];
        for (int j = 0; j < p; j++) s -= FN(lse_T)(F, i, q + j) * y[q + j];
        y[i] = s;
    }
    FN(trsv_un)(q, F->Af, m, y);
    for (int i = q; i < m; i++) {                        /* step 6: q2 = w2 - T22 y2 */
        REAL s = w[i];
        for (int j = 0; j < p; j++) s -= FN(lse_T)(F, i, q + j) * y[q + j];
        qv[i] = s;
    }
    for (int j = 0; j < p; j++) {                        /* step 8 rhs */
        REAL s = -u[q + j];
        for (int i = 0; i < m; i++) s += FN(lse_T)(F, i, q + j) * qv[i];
        t[j] = s;
    }
    FN(trsv_ut)(p, &F->Bf[IDX(0, q, p)], p, t);          /* R^T dv = rhs      */
    FN(lse_apply_Z)(F, 0, qv);                           /* step 7: dr = Z q  */
    FN(lse_apply_Q)(F, 1, y);                            /*         dx = Q^T y */
    for (int i = 0; i < m; i++) dr[i] = (double)qv[i];
    for (int i = 0; i < n; i++) dx[i] = (double)y[i];
    for (int i = 0; i < p; i++) dv[i] = (double)t[i];
    free(u); free(w); free(y); free(qv); free(t);
}

/* Initial multiplier (Sec. 3.1, Alg. 2 step 4): r = b - A x is passed in
 * (computed in FP64); R^T v = (Q (A^T r))(n-p+1:n) with A^T r in FP64 and
 * the Q product and the solve at precision REAL. */
static void FN(lse_init_v)(const FN(lse_fact) *F, const double *A, int lda,
                           const double *r, double *v)
{
    int m = F->m, n = F->n, p = F->p, q = n - p;
    REAL *s = (REAL *)malloc(sizeof(REAL) * (size_t)n);
    for (int j = 0; j < n; j++) {
        double acc = 0;
        for (int i = 0; i < m; i++) acc += A[IDX(i, j, lda)] * r[i];
        s[j] = (REAL)acc;
    }
    FN(lse_apply_Q)(F, 0, s);
    FN(trsv_ut)(p, &F->Bf[IDX(0, q, p)], p, s + q);
    for (int i = 0; i < p; i++) v[i] = (double)s[q + i];
    free(s);
}

/* ---------------- GLS: generalized QR factorization (Sec. 2.2) -------- */

typedef struct {
    int n, m, p;
    REAL *Wf; REAL *tauw;    /* QR of W: W = Q [R; 0],  ld = n */
    REAL *Vf; REAL *tauv;    /* RQ of Q^T V = T Z,      ld = n */
} FN(gls_fact);

/* Entry T(r, j) of the n x p upper trapezoidal T (RQ sense): row r holds R
 * entries from column p-n+r on; rows r < n-k (k = min(n,p)) are full. */
static inline REAL FN(gls_T)(const FN(gls_fact) *F, int r, int j)
{
    int n = F->n, p = F->p, k = n < p ? n : p;
    if (r < n - k || j >= p - n + r) return F->Vf[IDX(r, j, n)];
    return (REAL)0;
}

/* GQR of (W, V): QR of W, V <- Q^T V, RQ of Q^T V (Lemma 4.6). */
static void FN(gls_factor)(FN(gls_fact) *F, int n, int m, int p,
                           const double *W, int ldw, const double *V, int ldv)
{
    F->n = n; F->m = m; F->p = p;
    int kv = n < p ? n : p;
    F->Wf = (REAL *)malloc(sizeof(REAL) * (size_t)n * (size_t)(m > 0 ? m : 1));
    F->Vf = (REAL *)malloc(sizeof(REAL) * (size_t)n * (size_t)p);
    F->tauw = (REAL *)calloc((size_t)(m > 0 ? m : 1), sizeof(REAL));
    F->tauv = (REAL *)calloc((size_t)(kv > 0 ? kv : 1), sizeof(REAL));
    for (int j = 0; j < m; j++)
        for (int i = 0; i < n; i++) F->Wf[IDX(i, j, n)] = (REAL)W[IDX(i, j, ldw)];
    for (int j = 0; j < p; j++)
        for (int i = 0; i < n; i++) F->Vf[IDX(i, j, n)] = (REAL)V[IDX(i, j, ldv)];
    FN(geqr2)(n, m, F->Wf, n, F->tauw);
    /* V <- Q^T V = H_{m-1} ... H_0 V: each column independently */
    #pragma omp parallel for schedule(static) if ((size_t)n * (size_t)p > 65536)
    for (int c = 0; c < p; c++)
        FN(qr_apply_vec)(n, m, F->Wf, n, F->tauw, 1, &F->Vf[IDX(0, c, n)]);
    FN(gerq2)(n, p, F->Vf, n, F->tauv);
}

static void FN(gls_free)(FN(gls_fact) *F)
{
    free(F->Wf); free(F->Vf); free(F->tauw); free(F->tauv);
}

static inline void FN(gls_apply_Q)(const FN(gls_fact) *F, int trans, REAL *x)
{
    FN(qr_apply_vec)(F->n, F->m, F->Wf, F->n, F->tauw, trans, x);
}
static inline void FN(gls_apply_Z)(const FN(gls_fact) *F, int trans, REAL *x)
{
    int k = F->n < F->p ? F->n : F->p;
    FN(rq_apply_vec)(F->n, F->p, k, F->Vf, F->n, F->tauv, trans, x);
}

/* Paige's method (Sec. 2.2): c = Q^T d; T22 s2 = c2; R x = c1 - T12 s2;
 * y = Z^T [0; s2]. */
static void FN(gls_paige)(const FN(gls_fact) *F, const double *d,
                          double *x, double *y)
{
    int n = F->n, m = F->m, p = F->p, l = n - m, o = p - n + m;
    REAL *c = (REAL *)malloc(sizeof(REAL) * (size_t)n);
    REAL *s = (REAL *)calloc((size_t)p, sizeof(REAL));
    for (int i = 0; i < n; i++) c[i] = (REAL)d[i];
    FN(gls_apply_Q)(F, 1, c);
    for (int i = 0; i < l; i++) s[o + i] = c[m + i];
    FN(trsv_un)(l, &F->Vf[IDX(m, o, n)], n, s + o);
    for (int i = 0; i < m; i++) {
        REAL t = c[i];
        for (int j = 0; j < l; j++) t -= FN(gls_T)(F, i, o + j) * s[o + j];
        c[i] = t;
    }
    FN(trsv_un)(m, F->Wf, n, c);
    FN(gls_apply_Z)(F, 1, s);
    for (int i = 0; i < m; i++) x[i] = (double)c[i];
    for (int i = 0; i < p; i++) y[i] = (double)s[i];
    free(c); free(s);
}

/* Initial z (Sec. 3.2, Alg. 4 step 3, read as z0 = Q [0; v]): T22^T v =
 * (Z y)(p-n+m+1:p); z = Q [0; v].  W^T z = 0 and y = V^T z force Q, not
 * Q^T, in front of [0; v]. */
static void FN(gls_init_z)(const FN(gls_fact) *F, const double *y, double *z)
{
    int n = F->n, m = F->m, p = F->p, l = n - m, o = p - n + m;
    REAL *s = (REAL *)malloc(sizeof(REAL) * (size_t)p);
    REAL *h = (REAL *)calloc((size_t)n, sizeof(REAL));
    for (int i = 0; i < p; i++) s[i] = (REAL)y[i];
    FN(gls_apply_Z)(F, 0, s);
    for (int i = 0; i < l; i++) h[m + i] = s[o + i];
    FN(trsv_ut)(l, &F->Vf[IDX(m, o, n)], n, h + m);
    FN(gls_apply_Q)(F, 0, h);
    for (int i = 0; i < n; i++) z[i] = (double)h[i];
    free(s); free(h);
}

/* Algorithm 3 (CorrectionSystemSolverGLS), all steps at precision REAL,
 * with two readings of the printed algorithm:
 *  - the second triangular solve is T22 g2 = u2 (eq. gls-solver), not
 *    T22^T g2 = u2 (Alg. 3 step 4);
 *  - the printed equations define h = -Q^T dz, so dz = -Q h (the printed
 *    x2 = Q h has the wrong sign: row 3 of the system reads -W^T dz = f3).
 * Outputs x1 = dy (p), x2 = dz (n), x3 = dx (m). */
static void FN(gls_correction)(const FN(gls_fact) *F, const double *f1,
                               const double *f2, const double *f3,
                               double *dy, double *dz, double *dx)
{
    int n = F->n, m = F->m, p = F->p, l = n - m, o = p - n + m;
    REAL *u = (REAL *)malloc(sizeof(REAL) * (size_t)n);
    REAL *w = (REAL *)malloc(sizeof(REAL) * (size_t)p);
    REAL *h = (REAL *)malloc(sizeof(REAL) * (size_t)n);
    REAL *g = (REAL *)malloc(sizeof(REAL) * (size_t)p);
    for (int i = 0; i < n; i++) u[i] = (REAL)f2[i];
    FN(gls_apply_Q)(F, 1, u);                              /* u = Q^T f2   */
    for (int i = 0; i < p; i++) w[i] = (REAL)f1[i];
    FN(gls_apply_Z)(F, 0, w);                              /* w = Z f1     */
    for (int i = 0; i < m; i++) h[i] = (REAL)f3[i];
    FN(trsv_ut)(m, F->Wf, n, h);                           /* R^T h1 = f3  */
    for (int i = 0; i < l; i++) g[o + i] = u[m + i];
    FN(trsv_un)(l, &F->Vf[IDX(m, o, n)], n, g + o);        /* T22 g2 = u2  */
    for (int j = 0; j < l; j++) {                          /* T22^T h2 = w2 - g2 - T12^T h1 */
        REAL s = w[o + j] - g[o + j];
        for (int i = 0; i < m; i++) s -= FN(gls_T)(F, i, o + j) * h[i];
        h[m + j] = s;
    }
    FN(trsv_ut)(l, &F->Vf[IDX(m, o, n)], n, h + m);
    for (int j = 0; j < o; j++) {                          /* g1 = w1 - T11^T h1 */
        REAL s = w[j];
        for (int i = 0; i < m; i++) s -= FN(gls_T)(F, i, j) * h[i];
        g[j] = s;
    }
    for (int i = 0; i < m; i++) {                          /* R dx = u1 - T11 g1 - T12 g2 */
        REAL s = u[i];
        for (int j = 0; j < p; j++) s -= FN(gls_T)(F, i, j) * g[j];
        u[i] = s;
    }
    FN(trsv_un)(m, F->Wf, n, u);
    FN(gls_apply_Z)(F, 1, g);                              /* dy = Z^T g   */
    FN(gls_apply_Q)(F, 0, h);                              /* dz = -Q h    */
    for (int i = 0; i < p; i++) dy[i] = (double)g[i];
    for (int i = 0; i < n; i++) dz[i] = -(double)h[i];
    for (int i = 0; i < m; i++) dx[i] = (double)u[i];
    free(u); free(w); free(h); free(g);
}

/* ---------------- classical iterative refinement (Alg. 2 / Alg. 4) ---- */

/* Algorithm 2 (MPLSE).  Factorization, initial guess and correction solves
 * at precision REAL (u_f = u_s); residuals at u_r (FP64, or double-double
 * when resid_dd != 0); updates in FP64 (u).  The initial r0 is formed in
 * FP64.  Returns 0 when the stopping criteria (eq. lse-stop) hold, 3 when
 * maxit is reached, 4 on a non-finite residual. */
static int FN(lse_ir)(int m, int n, int p, const double *A, int lda,
                      const double *B, int ldb, const double *b,
                      const double *d, double *x, double *r, double *v,
                      int maxit, double tol, int resid_dd, int *iters,
                      double *stop_ratio)
{
    FN(lse_fact) F;
    FN(lse_factor)(&F, m, n, p, A, lda, B, ldb);
    FN(lse_nullspace)(&F, b, d, x);
    double *f1 = (double *)malloc(sizeof(double) * (size_t)m);
    double *f2 = (double *)malloc(sizeof(double) * (size_t)(p > 0 ? p : 1));
    double *f3 = (double *)malloc(sizeof(double) * (size_t)n);
    double *dr = (double *)malloc(sizeof(double) * (size_t)m);
    double *dv = (double *)malloc(sizeof(double) * (size_t)(p > 0 ? p : 1));
    double *dx = (double *)malloc(sizeof(double) * (size_t)n);
    /* r0 = b - A x0 (FP64), v0 from the KKT condition */
    for (int i = 0; i < m; i++) r[i] = b[i];
    for (int j = 0; j < n; j++)
        for (int i = 0; i < m; i++) r[i] -= A[IDX(i, j, lda)] * x[j];
    FN(lse_init_v)(&F, A, lda, r, v);
    double nA = fro_norm(m, n, A, lda), nB = fro_norm(p, n, B, ldb);
    double nb = vnorm(m, b), nd = vnorm(p, d);
    int status = 3, it;
    for (it = 0; it < maxit; it++) {
        lse_residual(m, n, p, A, lda, B, ldb, b, d, x, r, v, f1, f2, f3, resid_dd);
        double s1 = vnorm(m, f1), s2 = vnorm(p, f2), s3 = vnorm(n, f3);
        if (!(s1 == s1 && s2 == s2 && s3 == s3) || isinf(s1 + s2 + s3)) { status = 4; break; }
        double d1 = nb + vnorm(m, r) + nA * vnorm(n, x);
        double d2 = nd + nB * vnorm(n, x);
        double d3 = nA * vnorm(m, r) + nB * vnorm(p, v);
        stop_ratio[0] = d1 > 0 ? s1 / d1 : 0;
        stop_ratio[1] = d2 > 0 ? s2 / d2 : 0;
        stop_ratio[2] = d3 > 0 ? s3 / d3 : 0;
        if (s1 <= tol * d1 && s2 <= tol * d2 && s3 <= tol * d3) { status = 0; break; }
        FN(lse_correction)(&F, f1, f2, f3, dr, dv, dx);
        for (int i = 0; i < m; i++) r[i] += dr[i];
        for (int i = 0; i < n; i++) x[i] += dx[i];
        for (int i = 0; i < p; i++) v[i] += dv[i];
    }
    *iters = it;
    free(f1); free(f2); free(f3); free(dr); free(dv); free(dx);
    FN(lse_free)(&F);
    return status;
}

/* Algorithm 4 (MPGLS), same precision split as FN(lse_ir); stopping
 * criteria eq. gls-stop. */
static int FN(gls_ir)(int n, int m, int p, const double *W, int ldw,
                      const double *V, int ldv, const double *d, double *x,
                      double *y, double *z, int maxit, double tol,
                      int resid_dd, int *iters, double *stop_ratio)
{
    FN(gls_fact) F;
    FN(gls_factor)(&F, n, m, p, W, ldw, V, ldv);
    FN(gls_paige)(&F, d, x, y);
    FN(gls_init_z)(&F, y, z);
    double *f1 = (double *)malloc(sizeof(double) * (size_t)p);
    double *f2 = (double *)malloc(sizeof(double) * (size_t)n);
    double *f3 = (double *)malloc(sizeof(double) * (size_t)(m > 0 ? m : 1));
    double *dy = (double *)malloc(sizeof(double) * (size_t)p);
    double *dz = (double *)malloc(sizeof(double) * (size_t)n);
    double *dx = (double *)malloc(sizeof(double) * (size_t)(m > 0 ? m : 1));
    double nW = fro_norm(n, m, W, ldw), nV = fro_norm(n, p, V, ldv), nd = vnorm(n, d);
    int status = 3, it;
    for (it = 0; it < maxit; it++) {
        gls_residual(n, m, p, W, ldw, V, ldv, d, x, y, z, f1, f2, f3, resid_dd);
        double s1 = vnorm(p, f1), s2 = vnorm(n, f2), s3 = vnorm(m, f3);
        if (!(s1 == s1 && s2 == s2 && s3 == s3) || isinf(s1 + s2 + s3)) { status = 4; break; }
        double d1 = vnorm(p, y) + nV * vnorm(n, z);
        double d2 = nd + nW * vnorm(m, x) + nV * vnorm(p, y);
        double d3 = nW * vnorm(n, z);
        stop_ratio[0] = d1 > 0 ? s1 / d1 : 0;
        stop_ratio[1] = d2 > 0 ? s2 / d2 : 0;
        stop_ratio[2] = d3 > 0 ? s3 / d3 : 0;
        if (s1 <= tol * d1 && s2 <= tol * d2 && s3 <= tol * d3) { status = 0; break; }
        FN(gls_correction)(&F, f1, f2, f3, dy, dz, dx);
        for (int i = 0; i < p; i++) y[i] += dy[i];
        for (int i = 0; i < n; i++) z[i] += dz[i];
        for (int i = 0; i < m; i++) x[i] += dx[i];
    }
    *iters = it;
    free(f1); free(f2); free(f3); free(dy); free(dz); free(dx);
    FN(gls_free)(&F);
    return status;
}
