// batched.cu -- many independent small LSE problems in one persistent launch.
//
// Each CTA takes problems from a device work queue (largest first) and runs
// the whole method on one problem at a time: scaling and down-conversion,
// the GRQ factorization (Lemma 4.5) as blocked Householder QR in shared
// memory (32-column panels, compact-WY trailing updates), the null-space
// start (Sec. 2.1), the multipliers, and classical IR (Alg. 2) with FP64
// residuals read from the FP64 inputs and corrections by Alg. 1 on the
// factors.  Coordinates are the reversed ones of the single-problem solver:
//   B~ = P_n B^T P_p = Q~ [R~; 0],   At = A P_n Q~ P_n = Z T,
// so R = P_p R~^T P_p, Q = P_n Q~^T P_n, and every step below names the
// step of Alg. 1 / Alg. 2 it implements.
//
// TF is the factorization type: float (FP32 factors, FP32 correction solves
// with a power-of-two normalized right-hand side, FP64 residuals) or double
// (the fixed-precision FP64 comparator).  A problem whose factors do not fit
// the shared-memory budget keeps them in a per-CTA global scratch instead
// (same code through generic pointers).
#include <cstdio>
#include <cstring>
#include <algorithm>
#include <vector>

#include "batched.h"
#include "common.cuh"
#include "kernels.h"
#include "mpir.h"

namespace mpir {

constexpr int BNB = 32;    // panel width = compact-WY block size

// ------------------------------------------------------------ reductions --
template <int NT, typename T>
__device__ __forceinline__ T bsum(T v, T *red)
{
    v = warp_sum(v);
    __syncthreads();
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
    __syncthreads();
    T s = T(0);
#pragma unroll
    for (int k = 0; k < NT / 32; k++) s += red[k];
    return s;
}

template <int NT>
__device__ __forceinline__ double bmax(double v, double *red)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, o));
    __syncthreads();
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
    __syncthreads();
    double s = 0.0;
#pragma unroll
    for (int k = 0; k < NT / 32; k++) s = fmax(s, red[k]);
    return s;
}

__device__ __forceinline__ double pow2_of(double amax)
{   // 2^-e with amax * 2^-e in [0.5, 1); 1 for 0 / non-finite
    if (!(amax > 0.0) || !isfinite(amax)) return 1.0;
    return ldexp(1.0, -(ilogb(amax) + 1));
}

// ------------------------------------------------- blocked Householder QR --
// A (M x N, ld) = Z T, Z = H_0 ... H_{K-1}; reflector vectors below the
// diagonal, tau[K]; Tb: ceil(K/32) compact-WY factors (32 x 32, column-major)
// with H_j0 ... H_j0+nb-1 = I - V Tb V^T.  G: 1024 scratch.  (Zero
// diagonals are checked by the caller on the part it solves with.)
template <int NT, typename T>
__device__ void cta_geqrf(T *A, int ld, int M, int N, T *tau, T *Tb, T *G, T *red)
{
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    constexpr int NW = NT / 32;
    const int K = min(M, N);
    for (int j0 = 0; j0 < K; j0 += BNB) {
        const int nb = min(BNB, K - j0);
        // ---- panel: unblocked Householder on columns j0 .. j0+nb-1
        for (int k = j0; k < j0 + nb; k++) {
            T *ak = A + (size_t)k * ld;
            const T alpha = ak[k];
            T sq = T(0);
            for (int i = k + 1 + tid; i < M; i += NT) sq = fma(ak[i], ak[i], sq);
            sq = bsum<NT>(sq, red);
            const T xnorm = sqrt(sq);
            T t = T(0), beta = alpha, scal = T(1);
            if (xnorm != T(0)) {
                beta = -copysign(sqrt(alpha * alpha + sq), alpha);
                t = (beta - alpha) / beta;
                scal = T(1) / (alpha - beta);
                for (int i = k + 1 + tid; i < M; i += NT) ak[i] *= scal;
            }
            __syncthreads();
            if (tid == 0) {
                tau[k] = t;
                ak[k] = beta;
            }
            for (int j = k + 1 + warp; j < j0 + nb; j += NW) {
                T *aj = A + (size_t)j * ld;
                T dot = lane == 0 ? aj[k] : T(0);
                for (int i = k + 1 + lane; i < M; i += 32) dot = fma(ak[i], aj[i], dot);
                dot = warp_sum(dot) * t;
                if (lane == 0) aj[k] -= dot;
                for (int i = k + 1 + lane; i < M; i += 32) aj[i] = fma(-dot, ak[i], aj[i]);
            }
            __syncthreads();
        }
        // ---- compact-WY factor of the panel: G(a, c) = v_a^T v_c (a < c)
        T *Tk = Tb + (size_t)(j0 / BNB) * 1024;
        for (int pr = warp; pr < nb * nb; pr += NW) {
            const int a = pr % nb, c = pr / nb;
            if (a >= c) continue;
            const T *va = A + (size_t)(j0 + a) * ld, *vc = A + (size_t)(j0 + c) * ld;
            T dot = lane == 0 ? va[j0 + c] : T(0);
            for (int i = j0 + c + 1 + lane; i < M; i += 32) dot = fma(va[i], vc[i], dot);
            dot = warp_sum(dot);
            if (lane == 0) G[a + 32 * c] = dot;
        }
        __syncthreads();
        // Tk(:, c) = [-tau_c Tk(0:c, 0:c) G(0:c, c); tau_c; 0]
        if (warp == 0) {
            for (int c = 0; c < BNB; c++) {
                T s = T(0);
                if (c < nb && lane < c)
                    for (int b = lane; b < c; b++) s = fma(Tk[lane + 32 * b], G[b + 32 * c], s);
                __syncwarp();
                T val = T(0);
                if (c < nb) val = lane < c ? -tau[j0 + c] * s : (lane == c ? tau[j0 + c] : T(0));
                Tk[lane + 32 * c] = val;
                __syncwarp();
            }
        }
        __syncthreads();
        // ---- trailing update C <- (I - V Tk^T V^T) C, C = A(j0:M, j0+nb:N)
        const int cb = j0 + nb, Nc = N - cb;
        if (Nc > 0) {
            int S = 1;
            while (S < 8 && 2 * S * Nc <= NT) S *= 2;
            const int s = tid % S, per = NT / S;
            for (int jj0 = 0; jj0 < Nc; jj0 += per) {
                const int jj = jj0 + tid / S;
                const bool act = jj < Nc;
                T *cj = A + (size_t)(cb + (act ? jj : 0)) * ld;
                T w[BNB];
#pragma unroll
                for (int c = 0; c < BNB; c++) w[c] = T(0);
                if (act) {
                    // rows inside the unit-triangular top of V
                    for (int i = j0 + s; i < min(M, j0 + nb); i += S) {
                        const T x = cj[i];
                        const int r = i - j0;
#pragma unroll
                        for (int c = 0; c < BNB; c++) {
                            const T v = c < r ? A[i + (size_t)(j0 + c) * ld] : (c == r ? T(1) : T(0));
                            w[c] = fma(v, x, w[c]);
                        }
                    }
                    for (int i = j0 + nb + s; i < M; i += S) {
                        const T x = cj[i];
#pragma unroll
                        for (int c = 0; c < BNB; c++)
                            if (c < nb) w[c] = fma(A[i + (size_t)(j0 + c) * ld], x, w[c]);
                    }
                }
                for (int o = 1; o < S; o <<= 1) {
#pragma unroll
                    for (int c = 0; c < BNB; c++) w[c] += __shfl_xor_sync(0xffffffffu, w[c], o);
                }
                // w' = Tk^T w
                T wp[BNB];
#pragma unroll
                for (int a = 0; a < BNB; a++) {
                    T acc = T(0);
#pragma unroll
                    for (int c = 0; c <= a; c++) acc = fma(Tk[c + 32 * a], w[c], acc);
                    wp[a] = acc;
                }
                if (act) {
                    for (int i = j0 + s; i < min(M, j0 + nb); i += S) {
                        const int r = i - j0;
                        T d = T(0);
#pragma unroll
                        for (int c = 0; c < BNB; c++) {
                            const T v = c < r ? A[i + (size_t)(j0 + c) * ld] : (c == r ? T(1) : T(0));
                            d = fma(v, wp[c], d);
                        }
                        cj[i] -= d;
                    }
                    for (int i = j0 + nb + s; i < M; i += S) {
                        T d = T(0);
#pragma unroll
                        for (int c = 0; c < BNB; c++)
                            if (c < nb) d = fma(A[i + (size_t)(j0 + c) * ld], wp[c], d);
                        cj[i] -= d;
                    }
                }
            }
        }
        __syncthreads();
    }
}

// At (M x N, lda) <- At H'_0 ... H'_{K-1}, H'_k = P_N H_k P_N, H_k the
// reflectors of the N x K QR factor in Vb (ldv) with compact-WY factors Tb:
// the product At P_N Q~ P_N of the GRQ (Lemma 4.5, A Q^T).
template <int NT, typename T>
__device__ void cta_apply_right_rev(T *At, int lda, int M, int N, const T *Vb, int ldv, int K, const T *Tb)
{
    const int tid = threadIdx.x;
    for (int j0 = 0; j0 < K; j0 += BNB) {
        const int nb = min(BNB, K - j0);
        const T *Tk = Tb + (size_t)(j0 / BNB) * 1024;
        for (int i = tid; i < M; i += NT) {
            T y[BNB];
#pragma unroll
            for (int c = 0; c < BNB; c++) y[c] = T(0);
            // v'_c(j) = v_c(N-1-j): unit at j = N-1-(j0+c), zero for larger j
            for (int r = j0; r < N; r++) {          // r = N-1-j, the reflector row
                const T a = At[i + (size_t)(N - 1 - r) * lda];
                const int rr = r - j0;
#pragma unroll
                for (int c = 0; c < BNB; c++) {
                    if (c >= nb) continue;
                    const T v = c < rr ? Vb[r + (size_t)(j0 + c) * ldv] : (c == rr ? T(1) : T(0));
                    y[c] = fma(a, v, y[c]);
                }
            }
            // y' = y Tk
            T yp[BNB];
#pragma unroll
            for (int a = 0; a < BNB; a++) {
                T acc = T(0);
#pragma unroll
                for (int c = 0; c <= a; c++) acc = fma(y[c], Tk[c + 32 * a], acc);
                yp[a] = acc;
            }
            for (int r = j0; r < N; r++) {
                const int rr = r - j0;
                T d = T(0);
#pragma unroll
                for (int c = 0; c < BNB; c++) {
                    if (c >= nb) continue;
                    const T v = c < rr ? Vb[r + (size_t)(j0 + c) * ldv] : (c == rr ? T(1) : T(0));
                    d = fma(yp[c], v, d);
                }
                At[i + (size_t)(N - 1 - r) * lda] -= d;
            }
        }
        __syncthreads();
    }
}

// x (M) <- Z^T x (trans = 1) or Z x (trans = 0) for the reflector set of a
// cta_geqrf factorization (V in A, ld, K reflectors, Tb).
template <int NT, typename T>
__device__ void cta_apply_vec(const T *V, int ld, int M, int K, const T *Tb, int trans, T *x, T *wbuf)
{
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    constexpr int NW = NT / 32;
    const int nblk = ceil_div(K, BNB);
    for (int t = 0; t < nblk; t++) {
        const int b = trans ? t : nblk - 1 - t;
        const int j0 = b * BNB, nb = min(BNB, K - j0);
        const T *Tk = Tb + (size_t)b * 1024;
        for (int c = warp; c < nb; c += NW) {
            const T *vc = V + (size_t)(j0 + c) * ld;
            const int jc = j0 + c;
            T dot = lane == 0 ? x[jc] : T(0);
            for (int i = jc + 1 + lane; i < M; i += 32) dot = fma(vc[i], x[i], dot);
            dot = warp_sum(dot);
            if (lane == 0) wbuf[c] = dot;
        }
        __syncthreads();
        if (warp == 0) {
            T acc = T(0);
            if (lane < nb) {
                if (trans) {       // (Tk^T w)(a) = sum_{c <= a} Tk(c, a) w(c)
                    for (int c = 0; c <= lane; c++) acc = fma(Tk[c + 32 * lane], wbuf[c], acc);
                } else {           // (Tk w)(a) = sum_{c >= a} Tk(a, c) w(c)
                    for (int c = lane; c < nb; c++) acc = fma(Tk[lane + 32 * c], wbuf[c], acc);
                }
            }
            __syncwarp();
            wbuf[32 + lane] = acc;
        }
        __syncthreads();
        for (int i = j0 + tid; i < M; i += NT) {
            const int r = i - j0;
            T d = T(0);
            for (int c = 0; c < nb; c++) {
                const T v = c < r ? V[i + (size_t)(j0 + c) * ld] : (c == r ? T(1) : T(0));
                d = fma(v, wbuf[32 + c], d);
            }
            x[i] -= d;
        }
        __syncthreads();
    }
}

// Solve U x = b (trans = 0) or U^T x = b (trans = 1) in place, U the n x n
// upper triangle at (ld).  Zero pivot -> *st |= stbit.
template <int NT, typename T>
__device__ void cta_trsv(const T *U, int ld, int n, int trans, T *x, int *st, int stbit)
{
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int nblk = ceil_div(n, 32);
    for (int t = 0; t < nblk; t++) {
        const int blk = trans ? t : nblk - 1 - t;
        const int r0 = blk * 32, bs = min(32, n - r0);
        if (warp == 0) {
            T rhs = lane < bs ? x[r0 + lane] : T(0);
            T xv = T(0);
            if (!trans) {
                for (int c = bs - 1; c >= 0; c--) {
                    const T dcc = U[(r0 + c) + (size_t)(r0 + c) * ld];
                    T xc = __shfl_sync(0xffffffffu, rhs, c);
                    if (dcc == T(0) && lane == 0) atomicOr(st, stbit);
                    xc = xc / dcc;
                    if (lane == c) xv = xc;
                    if (lane < c) rhs = fma(-U[(r0 + lane) + (size_t)(r0 + c) * ld], xc, rhs);
                }
            } else {
                for (int c = 0; c < bs; c++) {
                    const T dcc = U[(r0 + c) + (size_t)(r0 + c) * ld];
                    T xc = __shfl_sync(0xffffffffu, rhs, c);
                    if (dcc == T(0) && lane == 0) atomicOr(st, stbit);
                    xc = xc / dcc;
                    if (lane == c) xv = xc;
                    if (lane > c && lane < bs) rhs = fma(-U[(r0 + c) + (size_t)(r0 + lane) * ld], xc, rhs);
                }
            }
            if (lane < bs) x[r0 + lane] = xv;
        }
        __syncthreads();
        if (!trans) {
            for (int i = tid; i < r0; i += NT) {
                T d = T(0);
                for (int c = 0; c < bs; c++) d = fma(U[i + (size_t)(r0 + c) * ld], x[r0 + c], d);
                x[i] -= d;
            }
        } else {
            for (int i = r0 + bs + tid; i < n; i += NT) {
                const T *ucol = U + (size_t)i * ld + r0;
                T d = T(0);
                for (int c = 0; c < bs; c++) d = fma(ucol[c], x[r0 + c], d);
                x[i] -= d;
            }
        }
        __syncthreads();
    }
}

// y (rows) += alpha * M x  (M rows x cols, ld); upper: M(i, j) = 0 for i > j
template <int NT, typename T>
__device__ void cta_gemv_n(const T *M, int ld, int rows, int cols, T alpha, const T *x, T *y, bool upper)
{
    for (int i = threadIdx.x; i < rows; i += NT) {
        T d = T(0);
        for (int j = upper ? i : 0; j < cols; j++) d = fma(M[i + (size_t)j * ld], x[j], d);
        y[i] = fma(alpha, d, y[i]);
    }
    __syncthreads();
}

// y (cols) += alpha * M^T x ; upper as above (column j uses rows i <= j)
template <int NT, typename T>
__device__ void cta_gemv_t(const T *M, int ld, int rows, int cols, T alpha, const T *x, T *y, bool upper)
{
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    for (int j = warp; j < cols; j += NT / 32) {
        const int ih = upper ? min(rows, j + 1) : rows;
        T d = T(0);
        for (int i = lane; i < ih; i += 32) d = fma(M[i + (size_t)j * ld], x[i], d);
        d = warp_sum(d);
        if (lane == 0) y[j] = fma(alpha, d, y[j]);
    }
    __syncthreads();
}

// ------------------------------------------------------ shared-memory plan --
struct BPlan {
    int ldB, ldA;                     // leading dimensions of Bt (n rows) and At (m rows)
    size_t vec_d;                     // doubles: x r v f1 f2 f3
    size_t vec_t;                     // TF words: 7 work vectors + tau + W/G scratch
    size_t fac_small;                 // TF words: TB + TA
    size_t fac_big;                   // TF words: Bt + At
};

__host__ __device__ inline int odd_ld(int r) { return (r | 1); }

__host__ __device__ inline BPlan bplan(int m, int n, int p)
{
    BPlan P;
    const int mx = max(max(m, n), max(p, 1));
    const int kA = min(m, n);
    P.ldB = odd_ld(max(n, 1));
    P.ldA = odd_ld(max(m, 1));
    P.vec_d = (size_t)2 * (m + n + p) + 64;
    P.vec_t = (size_t)7 * mx + p + kA + 64 + 1024;
    P.fac_small = (size_t)1024 * (ceil_div(p, BNB) + ceil_div(kA, BNB));
    P.fac_big = (size_t)P.ldB * p + (size_t)P.ldA * n;
    return P;
}

template <typename TF>
__host__ __device__ inline size_t bsmem_need(const BPlan &P, bool big_in_smem)
{
    size_t t = P.vec_t + P.fac_small + (big_in_smem ? P.fac_big : 0);
    return P.vec_d * 8 + ((t * sizeof(TF) + 15) & ~(size_t)15) + 64;
}

// ------------------------------------------------------------ one problem --
template <int NT, typename TF>
__device__ void solve_one(const BInst &I, BResult *res, unsigned char *smem, size_t smem_bytes, TF *gscr,
                          const BParams &prm)
{
    const int tid = threadIdx.x;
    const int m = I.m, n = I.n, p = I.p, q = n - p, kA = min(m, n);
    const int lda = I.lda, ldb = I.ldb;
    const double *A = I.A, *B = I.B, *b = I.b, *d = I.d;
    __shared__ double redd[NT / 32];
    __shared__ TF redt[NT / 32];
    __shared__ int st;
    const BPlan P = bplan(m, n, p);
    const bool big_smem = bsmem_need<TF>(P, true) <= smem_bytes;
    // carve
    double *X = reinterpret_cast<double *>(smem);
    double *R = X + n, *Vm = R + m, *F1 = Vm + p, *F2 = F1 + m, *F3 = F2 + p;
    TF *tb0 = reinterpret_cast<TF *>(smem + P.vec_d * 8);
    const int mx = max(max(m, n), max(p, 1));
    TF *tu = tb0, *tw = tu + mx, *ty = tw + mx, *tq = ty + mx, *tbv = tq + mx, *tt = tbv + mx, *tt2 = tt + mx;
    TF *tauB = tt2 + mx, *tauA = tauB + p, *wbuf = tauA + kA, *G = wbuf + 64;
    TF *TB = G + 1024, *TA = TB + (size_t)1024 * ceil_div(p, BNB);
    TF *big = TA + (size_t)1024 * ceil_div(kA, BNB);
    if (!big_smem) big = gscr;
    TF *Bt = big, *At = big + (size_t)P.ldB * p;
    if (tid == 0) st = 0;
    // ---- scaling (Sec. 6.1): powers of two, norms for the stop test
    double amA = 0.0, ssA = 0.0, amB = 0.0, ssB = 0.0;
    for (int e = tid; e < m * n; e += NT) {
        const double a = A[(size_t)(e % m) + (size_t)(e / m) * lda];
        amA = fmax(amA, fabs(a));
        ssA = fma(a, a, ssA);
    }
    for (int e = tid; e < p * n; e += NT) {
        const double a = B[(size_t)(e % p) + (size_t)(e / p) * ldb];
        amB = fmax(amB, fabs(a));
        ssB = fma(a, a, ssB);
    }
    amA = bmax<NT>(amA, redd);
    amB = bmax<NT>(amB, redd);
    ssA = bsum<NT>(ssA, redd);
    ssB = bsum<NT>(ssB, redd);
    const double fA = sqrt(ssA), fB = sqrt(ssB);
    if (!isfinite(ssA) || !isfinite(ssB)) {
        if (tid == 0) { res->status = MPIR_NONFINITE; res->iters = 0; }
        __syncthreads();
        return;
    }
    const double sA = prm.scale ? pow2_of(amA) : 1.0, sB = prm.scale ? pow2_of(amB) : 1.0;
    // B~ = P_n B^T P_p (n x p), At = A (m x n), both scaled
    for (int e = tid; e < p * n; e += NT) {
        const int r = e % p, c = e / p;
        Bt[(n - 1 - c) + (size_t)(p - 1 - r) * P.ldB] = (TF)(sB * B[r + (size_t)c * ldb]);
    }
    for (int e = tid; e < m * n; e += NT) {
        const int r = e % m, c = e / m;
        At[r + (size_t)c * P.ldA] = (TF)(sA * A[r + (size_t)c * lda]);
    }
    __syncthreads();
    // ---- GRQ (Lemma 4.5): QR of B~, At P_n Q~ P_n, QR of that
    cta_geqrf<NT, TF>(Bt, P.ldB, n, p, tauB, TB, G, redt);
    if (p > 0) cta_apply_right_rev<NT, TF>(At, P.ldA, m, n, Bt, P.ldB, p, TB);
    cta_geqrf<NT, TF>(At, P.ldA, m, n, tauA, TA, G, redt);
    __syncthreads();
    // zero diagonals: R~ (bit 1), T11 (bit 2)
    for (int i = tid; i < p; i += NT) if (Bt[i + (size_t)i * P.ldB] == TF(0)) atomicOr(&st, 1);
    for (int i = tid; i < q; i += NT) if (At[i + (size_t)i * P.ldA] == TF(0)) atomicOr(&st, 2);
    __syncthreads();
    if (st) {
        if (tid == 0) { res->status = (st & 1) ? MPIR_SINGULAR_R : MPIR_SINGULAR_T; res->iters = 0; }
        __syncthreads();
        return;
    }
    // ---- null-space start (Sec. 2.1), right-hand side normalized by g
    double mxr = 0.0;
    for (int i = tid; i < m; i += NT) mxr = fmax(mxr, fabs(sA * b[i]));
    for (int i = tid; i < p; i += NT) mxr = fmax(mxr, fabs(sB * d[i]));
    mxr = bmax<NT>(mxr, redd);
    double g = sizeof(TF) == 4 ? pow2_of(mxr) : 1.0;
    for (int i = tid; i < m; i += NT) tw[i] = (TF)(g * sA * b[i]);
    for (int i = tid; i < p; i += NT) tbv[i] = (TF)(g * sB * d[p - 1 - i]);
    __syncthreads();
    cta_apply_vec<NT, TF>(At, P.ldA, m, kA, TA, 1, tw, wbuf);              // c = Z^T (sA b)
    cta_trsv<NT, TF>(Bt, P.ldB, p, 1, tbv, &st, 1);                         // R~^T y~2 = P_p sB d
    for (int i = tid; i < p; i += NT) ty[q + i] = tbv[p - 1 - i];
    for (int i = tid; i < q; i += NT) ty[i] = tw[i];
    __syncthreads();
    if (p > 0 && q > 0) cta_gemv_n<NT, TF>(At + (size_t)q * P.ldA, P.ldA, q, p, TF(-1), ty + q, ty, false);
    cta_trsv<NT, TF>(At, P.ldA, q, 0, ty, &st, 2);                          // T11 y1 = c1 - T12 y2
    for (int i = tid; i < n; i += NT) tt[i] = ty[n - 1 - i];
    __syncthreads();
    cta_apply_vec<NT, TF>(Bt, P.ldB, n, p, TB, 0, tt, wbuf);                // x = Q^T y
    for (int i = tid; i < n; i += NT) X[i] = (double)tt[n - 1 - i] / g;
    __syncthreads();
    int it = 0, status = MPIR_OK;
    double ratio[3] = {0, 0, 0};
    if (prm.refine != MPIR_DIRECT) {
        // ---- multipliers (Alg. 2 steps 3-4): r0 = b - A x, R^T v0 = (Q A^T r0)(q+1:n)
        for (int i = tid; i < m; i += NT) {
            double acc = 0.0;
            for (int j = 0; j < n; j++) acc = fma(A[i + (size_t)j * lda], X[j], acc);
            R[i] = b[i] - acc;
        }
        __syncthreads();
        if (p > 0) {
            const int lane = tid & 31, warp = tid >> 5;
            for (int j = warp; j < n; j += NT / 32) {
                double acc = 0.0;
                for (int i = lane; i < m; i += 32) acc = fma(A[i + (size_t)j * lda], R[i], acc);
                acc = warp_sum(acc);
                if (lane == 0) F3[j] = acc;
            }
            __syncthreads();
            double mf = 0.0;
            for (int i = tid; i < n; i += NT) mf = fmax(mf, fabs(sA * F3[i]));
            mf = bmax<NT>(mf, redd);
            const double g3 = sizeof(TF) == 4 ? pow2_of(mf) : 1.0;
            for (int i = tid; i < n; i += NT) tu[i] = (TF)(g3 * sA * F3[n - 1 - i]);
            __syncthreads();
            cta_apply_vec<NT, TF>(Bt, P.ldB, n, p, TB, 1, tu, wbuf);
            cta_trsv<NT, TF>(Bt, P.ldB, p, 0, tu, &st, 1);
            for (int i = tid; i < p; i += NT) Vm[i] = (double)tu[p - 1 - i] * (sB / sA) / g3;
            __syncthreads();
        }
        double nb2 = 0.0, nd2 = 0.0;
        for (int i = tid; i < m; i += NT) nb2 = fma(b[i], b[i], nb2);
        for (int i = tid; i < p; i += NT) nd2 = fma(d[i], d[i], nd2);
        const double nbv = sqrt(bsum<NT>(nb2, redd)), ndv = sqrt(bsum<NT>(nd2, redd));
        double best = INFINITY;
        int since = 0;
        status = MPIR_NOT_CONVERGED;
        for (it = 0; it < prm.maxit; it++) {
            // ---- FP64 residual (Alg. 2 step 6) and norms
            const int lane = tid & 31, warp = tid >> 5;
            double s1 = 0.0, s2 = 0.0, sx = 0.0, sr = 0.0, sv = 0.0;
            for (int i = tid; i < m; i += NT) {
                double acc = 0.0;
                for (int j = 0; j < n; j++) acc = fma(A[i + (size_t)j * lda], X[j], acc);
                const double f = b[i] - R[i] - acc;
                F1[i] = f;
                s1 = fma(f, f, s1);
                sr = fma(R[i], R[i], sr);
            }
            for (int i = tid; i < p; i += NT) {
                double acc = 0.0;
                for (int j = 0; j < n; j++) acc = fma(B[i + (size_t)j * ldb], X[j], acc);
                const double f = d[i] - acc;
                F2[i] = f;
                s2 = fma(f, f, s2);
                sv = fma(Vm[i], Vm[i], sv);
            }
            for (int i = tid; i < n; i += NT) sx = fma(X[i], X[i], sx);
            double s3 = 0.0;
            for (int j = warp; j < n; j += NT / 32) {
                double acc = 0.0;
                for (int i = lane; i < m; i += 32) acc = fma(-A[i + (size_t)j * lda], R[i], acc);
                for (int i = lane; i < p; i += 32) acc = fma(B[i + (size_t)j * ldb], Vm[i], acc);
                acc = warp_sum(acc);
                if (lane == 0) { F3[j] = acc; s3 = fma(acc, acc, s3); }
            }
            const double n1 = sqrt(bsum<NT>(s1, redd)), n2 = sqrt(bsum<NT>(s2, redd));
            const double n3 = sqrt(bsum<NT>(s3, redd)), nx = sqrt(bsum<NT>(sx, redd));
            const double nr = sqrt(bsum<NT>(sr, redd)), nv = sqrt(bsum<NT>(sv, redd));
            // ---- stop test (eq. lse-stop) and stagnation
            const double den[3] = {nbv + nr + fA * nx, ndv + fB * nx, fA * nr + fB * nv};
            const double nrm[3] = {n1, n2, n3};
            bool ok = true, fin = true;
            for (int k = 0; k < 3; k++) {
                ratio[k] = den[k] > 0 ? nrm[k] / den[k] : (nrm[k] > 0 ? INFINITY : 0.0);
                if (!(nrm[k] <= prm.tol * den[k])) ok = false;
                if (!isfinite(nrm[k])) fin = false;
            }
            if (!fin) { status = MPIR_NONFINITE; break; }
            if (ok) { status = MPIR_OK; break; }
            const double eta = fmax(ratio[0], fmax(ratio[1], ratio[2]));
            if (eta < 0.5 * best) { best = eta; since = 0; }
            else if (++since >= 3) { status = best <= 1e-14 ? MPIR_OK : MPIR_NOT_CONVERGED; break; }
            // ---- correction (Alg. 1) on the scaled system, rhs normalized by gamma
            const double gam = sizeof(TF) == 4 ? pow2_of(fmax(n1, fmax(n2 * sB / sA, n3 * sA))) : 1.0;
            const double c1 = gam, c2 = gam * sB / sA, c3 = gam * sA;
            for (int i = tid; i < n; i += NT) tu[i] = (TF)(c3 * F3[n - 1 - i]);
            for (int i = tid; i < m; i += NT) tw[i] = (TF)(c1 * F1[i]);
            for (int i = tid; i < p; i += NT) tbv[i] = (TF)(c2 * F2[p - 1 - i]);
            __syncthreads();
            cta_apply_vec<NT, TF>(Bt, P.ldB, n, p, TB, 1, tu, wbuf);          // step 1: u~ = Q~^T P_n f3
            cta_apply_vec<NT, TF>(At, P.ldA, m, kA, TA, 1, tw, wbuf);         // step 2: w = Z^T f1
            if (p > 0) {                                                        // step 3: R y2 = f2
                cta_trsv<NT, TF>(Bt, P.ldB, p, 1, tbv, &st, 1);
                for (int i = tid; i < p; i += NT) ty[q + i] = tbv[p - 1 - i];
                __syncthreads();
            }
            if (q > 0) {
                for (int i = tid; i < q; i += NT) tq[i] = tu[p + q - 1 - i];
                __syncthreads();
                cta_trsv<NT, TF>(At, P.ldA, q, 1, tq, &st, 2);                 // step 4: T11^T q1 = u1
                for (int i = tid; i < q; i += NT) ty[i] = tw[i] - tq[i];
                __syncthreads();
                if (p > 0) cta_gemv_n<NT, TF>(At + (size_t)q * P.ldA, P.ldA, q, p, TF(-1), ty + q, ty, false);
                cta_trsv<NT, TF>(At, P.ldA, q, 0, ty, &st, 2);                 // step 5: T11 y1 = w1 - q1 - T12 y2
            }
            if (m - q > 0) {                                                    // step 6: q2 = w2 - T22 y2
                for (int i = tid; i < m - q; i += NT) tq[q + i] = tw[q + i];
                __syncthreads();
                if (p > 0)
                    cta_gemv_n<NT, TF>(At + q + (size_t)q * P.ldA, P.ldA, m - q, p, TF(-1), ty + q, tq + q, true);
            }
            if (p > 0) {                                                        // step 8: R^T dv = T12^T q1 + T22^T q2 - u2
                for (int i = tid; i < p; i += NT) tt[i] = TF(0);
                __syncthreads();
                if (q > 0) cta_gemv_t<NT, TF>(At + (size_t)q * P.ldA, P.ldA, q, p, TF(1), tq, tt, false);
                if (m - q > 0)
                    cta_gemv_t<NT, TF>(At + q + (size_t)q * P.ldA, P.ldA, m - q, p, TF(1), tq + q, tt, true);
                for (int i = tid; i < p; i += NT) tbv[i] = tt[p - 1 - i] - tu[i];
                __syncthreads();
                cta_trsv<NT, TF>(Bt, P.ldB, p, 0, tbv, &st, 1);
                for (int i = tid; i < p; i += NT) Vm[i] += (double)tbv[p - 1 - i] * (sB / sA) / gam;
            }
            for (int i = tid; i < n; i += NT) tt2[i] = ty[n - 1 - i];
            __syncthreads();
            cta_apply_vec<NT, TF>(At, P.ldA, m, kA, TA, 0, tq, wbuf);         // step 7: dr = Z q
            cta_apply_vec<NT, TF>(Bt, P.ldB, n, p, TB, 0, tt2, wbuf);         //         dx = Q^T y
            for (int i = tid; i < m; i += NT) R[i] += (double)tq[i] / gam;
            for (int i = tid; i < n; i += NT) X[i] += (double)tt2[n - 1 - i] * sA / gam;
            __syncthreads();
        }
    }
    // ---- result
    for (int i = tid; i < n; i += NT) I.x[i] = X[i];
    __syncthreads();
    if (tid == 0) {
        res->status = st ? ((st & 1) ? MPIR_SINGULAR_R : MPIR_SINGULAR_T) : status;
        res->iters = it;
        for (int k = 0; k < 3; k++) res->ratio[k] = ratio[k];
    }
    __syncthreads();
}

// ------------------------------------------------------- persistent kernel --
template <int NT, int MINB, typename TF>
__global__ void __launch_bounds__(NT, MINB)
k_lse_batched(const BInst *__restrict__ tab, const int *__restrict__ order, int count, int *__restrict__ next,
              BResult *__restrict__ res, TF *__restrict__ gscr, size_t gstride, size_t smem_bytes, BParams prm)
{
    extern __shared__ __align__(16) unsigned char smem[];
    __shared__ int s_k;
    TF *my = gscr + (size_t)blockIdx.x * gstride;
    for (;;) {
        if (threadIdx.x == 0) s_k = atomicAdd(next, 1);
        __syncthreads();
        const int k = s_k;
        __syncthreads();
        if (k >= count) break;
        const int idx = order[k];
        solve_one<NT, TF>(tab[idx], res + idx, smem, smem_bytes, my, prm);
    }
}

// ------------------------------------------------------------------ host --
template <int NT, int MINB, typename TF>
static int launch_cfg(const BInst *tab, const int *order, int count, int *next, BResult *res, TF *gscr,
                      size_t gstride, size_t smem, int grid, const BParams &prm, cudaStream_t s)
{
    auto kern = k_lse_batched<NT, MINB, TF>;
    if (cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess) {
        cudaGetLastError();
        return MPIR_UNSUPPORTED;
    }
    cudaMemsetAsync(next, 0, sizeof(int), s);
    prof_count(K_BATCHED);
    kern<<<grid, NT, smem, s>>>(tab, order, count, next, res, gscr, gstride, smem, prm);
    return cudaGetLastError() == cudaSuccess ? 0 : MPIR_CUDA_ERROR;
}

template <int NT, int MINB, typename TF>
static int occupancy_of(size_t smem)
{
    auto kern = k_lse_batched<NT, MINB, TF>;
    if (cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess) {
        cudaGetLastError();
        return 0;
    }
    int per = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, kern, NT, smem) != cudaSuccess) {
        cudaGetLastError();
        return 0;
    }
    return per;
}

int batched_ctas_per_sm(const BConfig &cfg, bool fp64)
{
    if (fp64) {
        if (cfg.threads == 512) return occupancy_of<512, 1, double>(cfg.smem);
        if (cfg.minb == 2) return occupancy_of<256, 2, double>(cfg.smem);
        return occupancy_of<256, 1, double>(cfg.smem);
    }
    if (cfg.threads == 512) return occupancy_of<512, 1, float>(cfg.smem);
    if (cfg.minb == 2) return occupancy_of<256, 2, float>(cfg.smem);
    return occupancy_of<256, 1, float>(cfg.smem);
}

int batched_launch(const BConfig &cfg, bool fp64, const BInst *tab, const int *order, int count, int *next,
                   BResult *res, void *gscr, size_t gstride_words, int grid, const BParams &prm, cudaStream_t s)
{
    if (fp64) {
        double *g = (double *)gscr;
        if (cfg.threads == 512)
            return launch_cfg<512, 1, double>(tab, order, count, next, res, g, gstride_words, cfg.smem, grid, prm, s);
        if (cfg.minb == 2)
            return launch_cfg<256, 2, double>(tab, order, count, next, res, g, gstride_words, cfg.smem, grid, prm, s);
        return launch_cfg<256, 1, double>(tab, order, count, next, res, g, gstride_words, cfg.smem, grid, prm, s);
    }
    float *g = (float *)gscr;
    if (cfg.threads == 512)
        return launch_cfg<512, 1, float>(tab, order, count, next, res, g, gstride_words, cfg.smem, grid, prm, s);
    if (cfg.minb == 2)
        return launch_cfg<256, 2, float>(tab, order, count, next, res, g, gstride_words, cfg.smem, grid, prm, s);
    return launch_cfg<256, 1, float>(tab, order, count, next, res, g, gstride_words, cfg.smem, grid, prm, s);
}

size_t batched_big_words(int m, int n, int p)
{
    const BPlan P = bplan(m, n, p);
    return P.fac_big;
}

size_t batched_smem_min(int m, int n, int p, bool fp64)
{
    const BPlan P = bplan(m, n, p);
    return fp64 ? bsmem_need<double>(P, false) : bsmem_need<float>(P, false);
}

size_t batched_smem_full(int m, int n, int p, bool fp64)
{
    const BPlan P = bplan(m, n, p);
    return fp64 ? bsmem_need<double>(P, true) : bsmem_need<float>(P, true);
}

double batched_work(int m, int n, int p)
{
    // GRQ flops (QR of n x p, apply to m x n from the right, QR of m x n)
    const double kA = std::min(m, n);
    double f = 2.0 * n * p * p - 2.0 * p * p * p / 3.0;
    f += 4.0 * (double)m * n * p;
    f += 2.0 * m * n * kA - 2.0 * kA * kA * kA / 3.0;
    return f + 8.0 * ((double)m * n + (double)p * n);
}

} // namespace mpir
