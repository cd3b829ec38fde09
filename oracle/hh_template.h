/*
 * CPU oracle -- Householder building blocks, instantiated once per real type.
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product library links or calls
 * this code; only tests/, the smoke check and the cpu_baseline leg of the
 * benchmark do.
 *
 * The file is included by mpir_oracle.c with
 *     REAL  = double | float   (arithmetic and storage type)
 *     FN(x) = x##_d  | x##_s   (name suffix)
 * so the factorization can be run entirely at the factorization precision u_f
 * of the paper's four-precision framework (Sec. 3).  Everything here is the
 * plain unblocked textbook form: one reflector at a time, no blocking, no
 * compact-WY, matrices column-major with a leading dimension.
 */

/* Elementary reflector H = I - tau * v * v^T with v(0) = 1 that maps
 * [alpha; x] to [beta; 0] (Sec. 4.2 uses Householder transformations for
 * xGEQRF/xGERQF).  Sign convention beta = -sign(alpha)*||[alpha;x]||.
 * On return alpha holds beta and x holds v(1:).  If x == 0, tau = 0. */
static void FN(larfg)(int len, REAL *alpha, REAL *x, size_t incx, REAL *tau)
{
    *tau = 0;
    if (len <= 1) return;
    REAL scale = 0;
    for (int i = 0; i < len - 1; i++) {
        REAL a = (REAL)fabs((double)x[i * incx]);
        if (a > scale) scale = a;
    }
    if (scale == 0) return;
    REAL ssq = 0;
    for (int i = 0; i < len - 1; i++) {
        REAL t = x[i * incx] / scale;
        ssq += t * t;
    }
    REAL xnorm = scale * (REAL)sqrt((double)ssq);
    REAL a = *alpha;
    REAL beta = (REAL)hypot((double)a, (double)xnorm);
    if (a >= 0) beta = -beta;
    *tau = (beta - a) / beta;
    REAL inv = (REAL)1 / (a - beta);
    for (int i = 0; i < len - 1; i++) x[i * incx] *= inv;
    *alpha = beta;
}

/* QR by Householder (xGEQRF, unblocked): A (m x n) = Z * T with
 * Z = H_0 H_1 ... H_{k-1}, k = min(m, n).  H_j acts on rows j..m-1 and its
 * vector is [1; A(j+1:m, j)].  T is left in the upper trapezoid of A. */
static void FN(geqr2)(int m, int n, REAL *A, int lda, REAL *tau)
{
    int k = m < n ? m : n;
    for (int j = 0; j < k; j++) {
        FN(larfg)(m - j, &A[IDX(j, j, lda)], &A[IDX(j + 1, j, lda)], 1, &tau[j]);
        REAL t = tau[j];
        if (t == 0) continue;
        const REAL *v = &A[IDX(j, j, lda)];          /* v(0) is implicit 1 */
        #pragma omp parallel for schedule(static) if ((size_t)(m - j) * (size_t)(n - j) > 65536)
        for (int c = j + 1; c < n; c++) {
            REAL *col = &A[IDX(j, c, lda)];
            REAL w = col[0];
            for (int i = 1; i < m - j; i++) w += v[i] * col[i];
            w *= t;
            col[0] -= w;
            for (int i = 1; i < m - j; i++) col[i] -= w * v[i];
        }
    }
}

/* X(0:nr, 0:c+1) <- X * (I - tau v v^T) where v(c) = 1 and v(0:c) is read
 * with stride vinc from vrow.  Rows are split between threads; every thread
 * does its own rows completely, so the result does not depend on the number
 * of threads. */
static void FN(apply_right)(int nr, int c, REAL *X, int ldx,
                            const REAL *vrow, size_t vinc, REAL tau)
{
    if (tau == 0 || nr <= 0) return;
    #pragma omp parallel if ((size_t)nr * (size_t)(c + 1) > 65536)
    {
        int nt = omp_get_num_threads(), id = omp_get_thread_num();
        int chunk = (nr + nt - 1) / nt;
        int r0 = id * chunk, r1 = r0 + chunk < nr ? r0 + chunk : nr;
        if (r1 > r0) {
            REAL *w = (REAL *)malloc(sizeof(REAL) * (size_t)(r1 - r0));
            for (int i = r0; i < r1; i++) w[i - r0] = X[IDX(i, c, ldx)];
            for (int j = 0; j < c; j++) {
                REAL vj = vrow[j * vinc];
                const REAL *col = &X[IDX(0, j, ldx)];
                for (int i = r0; i < r1; i++) w[i - r0] += col[i] * vj;
            }
            for (int i = r0; i < r1; i++) w[i - r0] *= tau;
            for (int i = r0; i < r1; i++) X[IDX(i, c, ldx)] -= w[i - r0];
            for (int j = 0; j < c; j++) {
                REAL vj = vrow[j * vinc];
                REAL *col = &X[IDX(0, j, ldx)];
                for (int i = r0; i < r1; i++) col[i] -= w[i - r0] * vj;
            }
            free(w);
        }
    }
}

/* RQ by Householder (xGERQF, unblocked): A (M x N) = T * Qr.  Reflector g
 * (g = 0..k-1, k = min(M,N)) is generated from row r = M-1-g with pivot
 * column c = N-1-g; it annihilates A(r, 0:c) and is applied from the right
 * to rows 0..r-1.  Hence A H_0 H_1 ... H_{k-1} = T and
 * Qr = H_{k-1} ... H_1 H_0.  The vector of H_g is [A(r, 0:c), 1]. */
static void FN(gerq2)(int M, int N, REAL *A, int lda, REAL *tau)
{
    int k = M < N ? M : N;
    for (int g = 0; g < k; g++) {
        int r = M - 1 - g, c = N - 1 - g;
        FN(larfg)(c + 1, &A[IDX(r, c, lda)], &A[IDX(r, 0, lda)], (size_t)lda, &tau[g]);
        FN(apply_right)(r, c, A, lda, &A[IDX(r, 0, lda)], (size_t)lda, tau[g]);
    }
}

/* ---- reflector sets applied to one vector ------------------------------ */

/* QR-type set from geqr2 on an (m x ?) matrix with k reflectors.
 * trans = 1: x <- Zq^T x = H_{k-1} ... H_0 x   (H_0 first)
 * trans = 0: x <- Zq   x = H_0 ... H_{k-1} x   (H_{k-1} first)           */
static void FN(qr_apply_vec)(int m, int k, const REAL *F, int ldf,
                             const REAL *tau, int trans, REAL *x)
{
    for (int s = 0; s < k; s++) {
        int j = trans ? s : k - 1 - s;
        if (tau[j] == 0) continue;
        const REAL *v = &F[IDX(j, j, ldf)];
        REAL w = x[j];
        for (int i = 1; i < m - j; i++) w += v[i] * x[j + i];
        w *= tau[j];
        x[j] -= w;
        for (int i = 1; i < m - j; i++) x[j + i] -= w * v[i];
    }
}

/* RQ-type set from gerq2 on an (M x N) matrix, k = min(M, N) reflectors,
 * Qr = H_{k-1} ... H_0 acting on vectors of length N.
 * trans = 0: x <- Qr   x   (H_0 first)
 * trans = 1: x <- Qr^T x   (H_{k-1} first)                              */
static void FN(rq_apply_vec)(int M, int N, int k, const REAL *F, int ldf,
                             const REAL *tau, int trans, REAL *x)
{
    for (int s = 0; s < k; s++) {
        int g = trans ? k - 1 - s : s;
        if (tau[g] == 0) continue;
        int r = M - 1 - g, c = N - 1 - g;
        REAL w = x[c];
        for (int j = 0; j < c; j++) w += F[IDX(r, j, ldf)] * x[j];
        w *= tau[g];
        x[c] -= w;
        for (int j = 0; j < c; j++) x[j] -= w * F[IDX(r, j, ldf)];
    }
}

/* ---- triangular solves on an n x n block whose (0,0) entry is T0 ------- */

/* upper, no transpose: T x = b (back substitution) */
static void FN(trsv_un)(int n, const REAL *T0, int ldt, REAL *x)
{
    for (int i = n - 1; i >= 0; i--) {
        REAL s = x[i];
        for (int j = i + 1; j < n; j++) s -= T0[IDX(i, j, ldt)] * x[j];
        x[i] = s / T0[IDX(i, i, ldt)];
    }
}

/* upper, transpose: T^T x = b (forward substitution) */
static void FN(trsv_ut)(int n, const REAL *T0, int ldt, REAL *x)
{
    for (int i = 0; i < n; i++) {
        REAL s = x[i];
        for (int j = 0; j < i; j++) s -= T0[IDX(j, i, ldt)] * x[j];
        x[i] = s / T0[IDX(i, i, ldt)];
    }
}
