// batched_kernel.cuh -- device code of the batched LSE / GLS solver: many
// independent small problems in one persistent launch.
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
#pragma once
#include <algorithm>

#include "batched.h"
#include "common.cuh"
#include "kernels.h"
#include "mpir.h"

namespace mpir {

constexpr int BNB = 32;    // panel width = compact-WY block size
constexpr int BWC = 256;   // trailing-update columns per pass (W scratch 32 x BWC)

// Threads of one problem ("group"): GT consecutive threads of the CTA, with
// their own named barrier (id 1 + group index; at most 16 groups).
template <int GT>
__device__ __forceinline__ void gsync()
{
    asm volatile("bar.sync %0, %1;" ::"r"(1 + (int)(threadIdx.x / GT)), "n"(GT) : "memory");
}

// ------------------------------------------------------------ reductions --
template <int GT, typename T>
__device__ __forceinline__ T bsum(T v, T *red)
{
    v = warp_sum(v);
    gsync<GT>();
    if (((threadIdx.x & (GT - 1)) & 31) == 0) red[(threadIdx.x & (GT - 1)) >> 5] = v;
    gsync<GT>();
    const int lane = (threadIdx.x & (GT - 1)) & 31;
    T s = lane < GT / 32 ? red[lane] : T(0);
    return warp_sum(s);
}

template <int GT>
__device__ __forceinline__ double bmax(double v, double *red)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, o));
    gsync<GT>();
    if (((threadIdx.x & (GT - 1)) & 31) == 0) red[(threadIdx.x & (GT - 1)) >> 5] = v;
    gsync<GT>();
    double s = 0.0;
#pragma unroll
    for (int k = 0; k < GT / 32; k++) s = fmax(s, red[k]);
    return s;
}

__device__ __forceinline__ double pow2_of(double amax)
{   // 2^-e with amax * 2^-e in [0.5, 1); 1 for 0 / non-finite
    if (!(amax > 0.0) || !isfinite(amax)) return 1.0;
    return ldexp(1.0, -(ilogb(amax) + 1));
}

// row[jj * ld] -= v . Wb(:, jj) for jj = j0, j0 + step, ... < Nc, eight
// columns at a time with their loads issued before the stores (the row may
// live in global memory).
template <typename T>
__device__ __forceinline__ void sub_vw(T *row, int ld, const T (&v)[BNB], const T *Wb, int j0, int step, int Nc)
{
    int jj = j0;
    for (; jj + 7 * step < Nc; jj += 8 * step) {
        T c8[8];
#pragma unroll
        for (int u = 0; u < 8; u++) c8[u] = row[(size_t)(jj + u * step) * ld];
#pragma unroll
        for (int u = 0; u < 8; u++) {
            const T *wj = Wb + 32 * (jj + u * step);
            T d = T(0);
#pragma unroll
            for (int c = 0; c < BNB; c++) d = fma(v[c], wj[c], d);
            row[(size_t)(jj + u * step) * ld] = c8[u] - d;
        }
    }
    for (; jj < Nc; jj += step) {
        const T *wj = Wb + 32 * jj;
        T d = T(0);
#pragma unroll
        for (int c = 0; c < BNB; c++) d = fma(v[c], wj[c], d);
        row[(size_t)jj * ld] -= d;
    }
}

// ------------------------------------------------- blocked Householder QR --
// A (M x N, ld) = Z T, Z = H_0 ... H_{K-1}; reflector vectors below the
// diagonal, tau[K]; Tb: ceil(K/32) compact-WY factors (32 x 32, column-major)
// with H_j0 ... H_j0+nb-1 = I - V Tb V^T.  G: 1024 scratch; Wb: 32 x (N-32)
// scratch (32 x min(N-32, BWC): the trailing update runs over column chunks).
// K = min(M, N), or kmax when kmax >= 0 is smaller: the columns
// beyond K then only receive the reflectors (Q^T applied to them).  (Zero
// diagonals are checked by the caller on the part it solves with.)
//
// Panel step k (one CTA barrier per column): every thread forms the larfg
// scalars of column k from alpha = A(k,k) and the held ||A(k+1:M, k)||^2;
// warps update the remaining panel columns with the still unscaled column k
// (v = scal * A(k+1:M, k)), and the warp that updates column k+1 also
// leaves its new sub-diagonal norm; after the barrier column k is scaled in
// place while the next step runs on the columns to its right.
template <int GT, typename T>
__device__ void cta_geqrf(T *A, int ld, int M, int N, T *tau, T *Tb, T *G, T *Wb, T *stage, int kmax = -1)
{
    const int tid = (threadIdx.x & (GT - 1)), lane = tid & 31, warp = tid >> 5;
    constexpr int NW = GT / 32;
    __shared__ T cn2_g[512 / GT][2];
    T *cn2 = cn2_g[threadIdx.x / GT];
    const int K = kmax >= 0 ? min(kmax, min(M, N)) : min(M, N);
    for (int j0 = 0; j0 < K; j0 += BNB) {
        const int nb = min(BNB, K - j0);
        // panel access: element (i, j0 + c) at P[(i - roff) + c * pld]; with a
        // stage (factors in global memory) the panel is copied to shared memory
        T *P;
        int pld, roff;
        if (stage) {
            P = stage;
            pld = M - j0;
            roff = j0;
            for (int e = tid; e < pld * nb; e += GT) {
                const int r = e % pld, c = e / pld;
                P[e] = A[(j0 + r) + (size_t)(j0 + c) * ld];
            }
            gsync<GT>();
        } else {
            P = A + (size_t)j0 * ld;
            pld = ld;
            roff = 0;
        }
        if (warp == 0) {
            T sq = T(0);
            for (int i = j0 + 1 + lane; i < M; i += 32) sq = fma(P[i - roff], P[i - roff], sq);
            sq = warp_sum(sq);
            if (lane == 0) cn2[j0 & 1] = sq;
        }
        gsync<GT>();
        // ---- panel
        for (int k = j0; k < j0 + nb; k++) {
            T *ak = P + (size_t)(k - j0) * pld;
            const T alpha = ak[k - roff];
            const T sq = cn2[k & 1];
            T t = T(0), beta = alpha, scal = T(1);
            if (sq != T(0)) {
                beta = -copysign(sqrt(alpha * alpha + sq), alpha);
                t = (beta - alpha) / beta;
                scal = T(1) / (alpha - beta);
            }
            for (int j = k + 1 + warp; j < j0 + nb; j += NW) {
                T *aj = P + (size_t)(j - j0) * pld;
                T dot = T(0);
                for (int i = k + 1 + lane; i < M; i += 32) dot = fma(ak[i - roff], aj[i - roff], dot);
                dot = warp_sum(dot);
                const T td = t * fma(scal, dot, aj[k - roff]);
                const T tds = td * scal;
                T nsq = T(0);
                int i = k + 1 + lane;
                for (; i + 96 < M; i += 128) {     // four rows per lane in flight
                    T c4[4], v4[4];
#pragma unroll
                    for (int u = 0; u < 4; u++) { c4[u] = aj[i + 32 * u - roff]; v4[u] = ak[i + 32 * u - roff]; }
#pragma unroll
                    for (int u = 0; u < 4; u++) {
                        const T w = fma(-tds, v4[u], c4[u]);
                        aj[i + 32 * u - roff] = w;
                        if (i + 32 * u > k + 1) nsq = fma(w, w, nsq);
                    }
                }
                for (; i < M; i += 32) {
                    const T w = fma(-tds, ak[i - roff], aj[i - roff]);
                    aj[i - roff] = w;
                    if (i > k + 1) nsq = fma(w, w, nsq);
                }
                if (j == k + 1) {
                    nsq = warp_sum(nsq);
                    if (lane == 0) cn2[(k + 1) & 1] = nsq;
                }
                if (lane == 0) aj[k - roff] -= td;
            }
            gsync<GT>();
            if (t != T(0))
                for (int i = k + 1 + tid; i < M; i += GT) ak[i - roff] *= scal;
            if (tid == 0) {
                tau[k] = t;
                ak[k - roff] = beta;
            }
        }
        gsync<GT>();
        // ---- compact-WY factor of the panel: G(a, c) = v_a^T v_c (a < c)
        T *Tk = Tb + (size_t)(j0 / BNB) * 1024;
        for (int pr = warp; pr < nb * nb; pr += NW) {
            const int a = pr % nb, c = pr / nb;
            if (a >= c) continue;
            const T *va = P + (size_t)a * pld - roff, *vc = P + (size_t)c * pld - roff;
            T dot = lane == 0 ? va[j0 + c] : T(0);
            for (int i = j0 + c + 1 + lane; i < M; i += 32) dot = fma(va[i], vc[i], dot);
            dot = warp_sum(dot);
            if (lane == 0) G[a + 32 * c] = dot;
        }
        gsync<GT>();
        // Tk(a, c) = -tau_c sum_{a <= b < c} Tk(a, b) G(b, c), Tk(c, c) = tau_c:
        // lane a builds row a in registers
        if (warp == 0) {
            T tr[BNB];
#pragma unroll
            for (int c = 0; c < BNB; c++) {
                T sacc = T(0);
#pragma unroll
                for (int b = 0; b < c; b++)
                    if (b >= lane) sacc = fma(tr[b], G[b + 32 * c], sacc);
                const T tc = c < nb ? tau[j0 + c] : T(0);
                tr[c] = c < nb ? (lane < c ? -tc * sacc : (lane == c ? tc : T(0))) : T(0);
            }
#pragma unroll
            for (int c = 0; c < BNB; c++) Tk[lane + 32 * c] = tr[c];
        }
        gsync<GT>();
        // ---- trailing update C <- (I - V Tk^T V^T) C, C = A(j0:M, cb:N), in
        // chunks of BWC columns
        const int cb0 = j0 + nb;
        const T *Vp = P - roff;      // Vp[i + c * pld] = V(i, c) below the diagonal
        for (int cb = cb0; cb < N; cb += BWC) {
            const int Nc = min(BWC, N - cb);
            // W = V^T C (warp per column, lanes over rows; lane c keeps W(c, j))
            for (int jj = warp; jj < Nc; jj += NW) {
                const T *cj = A + (size_t)(cb + jj) * ld;
                T w[BNB];
#pragma unroll
                for (int c = 0; c < BNB; c++) w[c] = T(0);
                for (int i = j0 + lane; i < M; i += 32) {
                    const T x = cj[i];
                    const int r = i - j0;
#pragma unroll
                    for (int c = 0; c < BNB; c++) {
                        const T v = c < nb ? (c < r ? Vp[i + (size_t)c * pld] : (c == r ? T(1) : T(0))) : T(0);
                        w[c] = fma(v, x, w[c]);
                    }
                }
                const T wc = warp_transpose_reduce<T, BNB>(w);
                // W' = Tk^T W: W'(a) = sum_{c <= a} Tk(c, a) W(c)
                T acc = T(0);
#pragma unroll
                for (int c = 0; c < BNB; c++) {
                    const T wcc = __shfl_sync(0xffffffffu, wc, c);
                    if (c <= lane) acc = fma(Tk[c + 32 * lane], wcc, acc);
                }
                Wb[lane + 32 * jj] = acc;
            }
            gsync<GT>();
            // C -= V W' (rows over threads; column groups when rows are few)
            const int R = M - j0;
            const int grp = max(1, min(8, GT / max(R, 1)));
            const int gi = tid / R, ri = tid % R;
            if (gi < grp) {
                const int i = j0 + ri;
                T v[BNB];
#pragma unroll
                for (int c = 0; c < BNB; c++)
                    v[c] = c < nb ? (c < ri ? Vp[i + (size_t)c * pld] : (c == ri ? T(1) : T(0))) : T(0);
                sub_vw<T>(A + i + (size_t)cb * ld, ld, v, Wb, gi, grp, Nc);
            }
            for (int i0 = j0 + GT; i0 < M; i0 += GT) {    // rows beyond one per thread
                const int i = i0 + tid;
                if (i < M) {
                    const int r = i - j0;
                    T v[BNB];
#pragma unroll
                    for (int c = 0; c < BNB; c++)
                        v[c] = c < nb ? (c < r ? Vp[i + (size_t)c * pld] : (c == r ? T(1) : T(0))) : T(0);
                    sub_vw<T>(A + i + (size_t)cb * ld, ld, v, Wb, 0, 1, Nc);
                }
            }
            gsync<GT>();
        }
        if (stage) {
            gsync<GT>();
            for (int e = tid; e < pld * nb; e += GT) {
                const int r = e % pld, c = e / pld;
                A[(j0 + r) + (size_t)(j0 + c) * ld] = P[e];
            }
        }
        gsync<GT>();
    }
}

// At (M x N, lda) <- At H'_0 ... H'_{K-1}, H'_k = P_N H_k P_N, H_k the
// reflectors of the N x K QR factor in Vb (ldv) with compact-WY factors Tb
// (32 x 32 per panel): the product At P_N Q~ P_N of the GRQ (Lemma 4.5,
// A Q^T).  Rows are independent (one thread per row); reflectors go in
// blocks of 8 with the 8 x 8 diagonal blocks of Tb as their factors (the
// factor of a contiguous run of reflectors is that diagonal block), so a
// small K wastes little.
template <int GT, typename T>
__device__ void cta_apply_right_rev(T *At, int lda, int M, int N, const T *Vb, int ldv, int K, const T *Tb)
{
    constexpr int RB = 8;
    for (int i = (threadIdx.x & (GT - 1)); i < M; i += GT) {
        T *row = At + i;
        for (int k0 = 0; k0 < K; k0 += RB) {
            const int nb = min(RB, K - k0);
            const T *Tk = Tb + (size_t)(k0 / 32) * 1024 + (k0 % 32) * 33;   // Tb(k0%32, k0%32) of the panel
            // y(c) = sum_r row(N-1-r) v_{k0+c}(r), r >= k0 + c (unit at r = k0 + c)
            T y[RB];
#pragma unroll
            for (int c = 0; c < RB; c++) y[c] = T(0);
            for (int r = k0; r < N; r += 4) {
                T a4[4];
#pragma unroll
                for (int u = 0; u < 4; u++) a4[u] = r + u < N ? row[(size_t)(N - 1 - r - u) * lda] : T(0);
#pragma unroll
                for (int u = 0; u < 4; u++) {
                    const int rr = r + u - k0;
#pragma unroll
                    for (int c = 0; c < RB; c++) {
                        if (c >= nb) continue;
                        const T v = c < rr ? (r + u < N ? Vb[r + u + (size_t)(k0 + c) * ldv] : T(0))
                                           : (c == rr ? T(1) : T(0));
                        y[c] = fma(a4[u], v, y[c]);
                    }
                }
            }
            // y' = y Tk (Tk upper, 8 x 8 with leading dimension 32)
            T yp[RB];
#pragma unroll
            for (int a = 0; a < RB; a++) {
                T acc = T(0);
#pragma unroll
                for (int c = 0; c <= a; c++) acc = fma(y[c], Tk[c + 32 * a], acc);
                yp[a] = a < nb ? acc : T(0);
            }
            for (int r = k0; r < N; r += 4) {
                T a4[4];
#pragma unroll
                for (int u = 0; u < 4; u++) a4[u] = r + u < N ? row[(size_t)(N - 1 - r - u) * lda] : T(0);
#pragma unroll
                for (int u = 0; u < 4; u++) {
                    const int rr = r + u - k0;
                    T d = T(0);
#pragma unroll
                    for (int c = 0; c < RB; c++) {
                        if (c >= nb) continue;
                        const T v = c < rr ? (r + u < N ? Vb[r + u + (size_t)(k0 + c) * ldv] : T(0))
                                           : (c == rr ? T(1) : T(0));
                        d = fma(yp[c], v, d);
                    }
                    if (r + u < N) row[(size_t)(N - 1 - r - u) * lda] = a4[u] - d;
                }
            }
        }
    }
    gsync<GT>();
}

// x (M) <- Z^T x (trans = 1) or Z x (trans = 0) for the reflector set of a
// cta_geqrf factorization (V in A, ld, K reflectors, Tb).
template <int GT, typename T>
__device__ void cta_apply_vec(const T *V, int ld, int M, int K, const T *Tb, int trans, T *x, T *wbuf)
{
    const int tid = (threadIdx.x & (GT - 1)), lane = tid & 31, warp = tid >> 5;
    constexpr int NW = GT / 32;
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
        gsync<GT>();
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
        gsync<GT>();
        for (int i = j0 + tid; i < M; i += GT) {
            const int r = i - j0;
            T d = T(0);
            for (int c = 0; c < nb; c++) {
                const T v = c < r ? V[i + (size_t)(j0 + c) * ld] : (c == r ? T(1) : T(0));
                d = fma(v, wbuf[32 + c], d);
            }
            x[i] -= d;
        }
        gsync<GT>();
    }
}

// Solve U x = b (trans = 0) or U^T x = b (trans = 1) in place, U the n x n
// upper triangle at (ld).  Zero pivot -> *st |= stbit.
template <int GT, typename T>
__device__ void cta_trsv(const T *U, int ld, int n, int trans, T *x, int *st, int stbit)
{
    const int tid = (threadIdx.x & (GT - 1)), lane = tid & 31, warp = tid >> 5;
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
        gsync<GT>();
        if (!trans) {
            for (int i = tid; i < r0; i += GT) {
                T d = T(0);
                for (int c = 0; c < bs; c++) d = fma(U[i + (size_t)(r0 + c) * ld], x[r0 + c], d);
                x[i] -= d;
            }
        } else {
            for (int i = r0 + bs + tid; i < n; i += GT) {
                const T *ucol = U + (size_t)i * ld + r0;
                T d = T(0);
                for (int c = 0; c < bs; c++) d = fma(ucol[c], x[r0 + c], d);
                x[i] -= d;
            }
        }
        gsync<GT>();
    }
}

// y (rows) += alpha * M x  (M rows x cols, ld); upper: M(i, j) = 0 for i > j
template <int GT, typename T>
__device__ void cta_gemv_n(const T *M, int ld, int rows, int cols, T alpha, const T *x, T *y, bool upper)
{
    for (int i = (threadIdx.x & (GT - 1)); i < rows; i += GT) {
        T d = T(0);
        for (int j = upper ? i : 0; j < cols; j++) d = fma(M[i + (size_t)j * ld], x[j], d);
        y[i] = fma(alpha, d, y[i]);
    }
    gsync<GT>();
}

// y (cols) += alpha * M^T x ; upper as above (column j uses rows i <= j)
template <int GT, typename T>
__device__ void cta_gemv_t(const T *M, int ld, int rows, int cols, T alpha, const T *x, T *y, bool upper)
{
    const int lane = (threadIdx.x & (GT - 1)) & 31, warp = (threadIdx.x & (GT - 1)) >> 5;
    for (int j = warp; j < cols; j += GT / 32) {
        const int ih = upper ? min(rows, j + 1) : rows;
        T d = T(0);
        for (int i = lane; i < ih; i += 32) d = fma(M[i + (size_t)j * ld], x[i], d);
        d = warp_sum(d);
        if (lane == 0) y[j] = fma(alpha, d, y[j]);
    }
    gsync<GT>();
}

// ------------------------------------------------------ shared-memory plan --
struct BPlan {
    int ldB, ldA;                     // leading dimensions of Bt (n rows) and At (m rows)
    size_t vec_d;                     // doubles: x r v f1 f2 f3
    size_t vec_t;                     // TF words: 7 work vectors + tau + W/G scratch
    size_t fac_small;                 // TF words: TB + TA
    size_t fac_big;                   // TF words: Bt + At
    size_t stage;                     // TF words: panel stage when the factors are in global memory
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
    P.vec_t = (size_t)7 * mx + p + kA + 64 + 1024 + (size_t)32 * min(BWC, max(max(n, p), 1));
    P.fac_small = (size_t)1024 * (ceil_div(p, BNB) + ceil_div(kA, BNB));
    P.fac_big = (size_t)P.ldB * p + (size_t)P.ldA * n;
    P.stage = (size_t)BNB * max(max(m, n), 1);
    return P;
}

// mode 2: everything in shared memory; 1: factors in global scratch with
// the current panel staged in shared memory; 0: factors in global scratch.
template <typename TF>
__host__ __device__ inline size_t bsmem_need(const BPlan &P, int mode)
{
    size_t t = P.vec_t + P.fac_small + (mode == 2 ? P.fac_big : (mode == 1 ? P.stage : 0));
    return P.vec_d * 8 + ((t * sizeof(TF) + 15) & ~(size_t)15) + 64;
}

// GLS (n x m W, n x p V): [Wf Cf] n x (m + p) (ldB = odd_ld(n)) with Q^T V
// in its last p columns, then Ct = P_p C^T P_n (p x n, ldA = odd_ld(p)).
__host__ __device__ inline BPlan gplan(int m, int n, int p)
{
    BPlan P;
    const int mx = max(max(m, n), max(p, 1));
    const int kC = min(n, p);
    P.ldB = odd_ld(max(n, 1));
    P.ldA = odd_ld(max(p, 1));
    P.vec_d = (size_t)2 * (m + n + p) + 64;
    P.vec_t = (size_t)7 * mx + m + kC + 64 + 1024 + (size_t)32 * min(BWC, max(m + p, max(n, 1)));
    // the panels' compact-WY factors travel with the big factors (shared
    // memory, or the global scratch)
    P.fac_small = 0;
    P.fac_big = (size_t)P.ldB * (m + p) + (size_t)P.ldA * n + (size_t)1024 * (ceil_div(m, BNB) + ceil_div(kC, BNB));
    P.stage = (size_t)BNB * max(max(n, p), 1);
    return P;
}

// ------------------------------------------------------------ one problem --
template <int GT, typename TF>
__device__ void solve_one(const BInst &I, BResult *res, unsigned char *smem, size_t smem_bytes, TF *gscr,
                          const BParams &prm)
{
    const int tid = (threadIdx.x & (GT - 1));
    const int m = I.m, n = I.n, p = I.p, q = n - p, kA = min(m, n);
    const int lda = I.lda, ldb = I.ldb;
    const double *A = I.A, *B = I.B, *b = I.b, *d = I.d;
    __shared__ double redd_g[512 / GT][GT / 32];
    __shared__ int st_g[512 / GT];
    double *redd = redd_g[threadIdx.x / GT];
    int &st = st_g[threadIdx.x / GT];
    const BPlan P = bplan(m, n, p);
    const bool big_smem = bsmem_need<TF>(P, 2) <= smem_bytes;
    const bool use_stage = !big_smem && bsmem_need<TF>(P, 1) <= smem_bytes;
    // carve
    double *X = reinterpret_cast<double *>(smem);
    double *R = X + n, *Vm = R + m, *F1 = Vm + p, *F2 = F1 + m, *F3 = F2 + p;
    TF *tb0 = reinterpret_cast<TF *>(smem + P.vec_d * 8);
    const int mx = max(max(m, n), max(p, 1));
    TF *tu = tb0, *tw = tu + mx, *ty = tw + mx, *tq = ty + mx, *tbv = tq + mx, *tt = tbv + mx, *tt2 = tt + mx;
    TF *tauB = tt2 + mx, *tauA = tauB + p, *wbuf = tauA + kA, *G = wbuf + 64;
    TF *Wb = G + 1024;
    TF *TB = Wb + (size_t)32 * min(BWC, max(max(n, p), 1)), *TA = TB + (size_t)1024 * ceil_div(p, BNB);
    TF *big = TA + (size_t)1024 * ceil_div(kA, BNB);
    TF *stage = nullptr;
    if (!big_smem) {
        if (use_stage) stage = big;
        big = gscr;
    }
    TF *Bt = big, *At = big + (size_t)P.ldB * p;
    if (tid == 0) st = 0;
    // ---- scaling (Sec. 6.1): powers of two, norms for the stop test
    double amA = 0.0, ssA = 0.0, amB = 0.0, ssB = 0.0;
    for (int e = tid; e < m * n; e += GT) {
        const double a = A[(size_t)(e % m) + (size_t)(e / m) * lda];
        amA = fmax(amA, fabs(a));
        ssA = fma(a, a, ssA);
    }
    for (int e = tid; e < p * n; e += GT) {
        const double a = B[(size_t)(e % p) + (size_t)(e / p) * ldb];
        amB = fmax(amB, fabs(a));
        ssB = fma(a, a, ssB);
    }
    amA = bmax<GT>(amA, redd);
    amB = bmax<GT>(amB, redd);
    ssA = bsum<GT>(ssA, redd);
    ssB = bsum<GT>(ssB, redd);
    const double fA = sqrt(ssA), fB = sqrt(ssB);
    if (!isfinite(ssA) || !isfinite(ssB)) {
        if (tid == 0) { res->status = MPIR_NONFINITE; res->iters = 0; }
        gsync<GT>();
        return;
    }
    const double sA = prm.scale ? pow2_of(amA) : 1.0, sB = prm.scale ? pow2_of(amB) : 1.0;
    // B~ = P_n B^T P_p (n x p), At = A (m x n), both scaled
    for (int e = tid; e < p * n; e += GT) {
        const int r = e % p, c = e / p;
        Bt[(n - 1 - c) + (size_t)(p - 1 - r) * P.ldB] = (TF)(sB * B[r + (size_t)c * ldb]);
    }
    for (int e = tid; e < m * n; e += GT) {
        const int r = e % m, c = e / m;
        At[r + (size_t)c * P.ldA] = (TF)(sA * A[r + (size_t)c * lda]);
    }
    gsync<GT>();
    // ---- GRQ (Lemma 4.5): QR of B~, At P_n Q~ P_n, QR of that
    cta_geqrf<GT, TF>(Bt, P.ldB, n, p, tauB, TB, G, Wb, stage);
    if (p > 0) cta_apply_right_rev<GT, TF>(At, P.ldA, m, n, Bt, P.ldB, p, TB);
    cta_geqrf<GT, TF>(At, P.ldA, m, n, tauA, TA, G, Wb, stage);
    gsync<GT>();
    // zero diagonals: R~ (bit 1), T11 (bit 2)
    for (int i = tid; i < p; i += GT) if (Bt[i + (size_t)i * P.ldB] == TF(0)) atomicOr(&st, 1);
    for (int i = tid; i < q; i += GT) if (At[i + (size_t)i * P.ldA] == TF(0)) atomicOr(&st, 2);
    gsync<GT>();
    if (st) {
        if (tid == 0) { res->status = (st & 1) ? MPIR_SINGULAR_R : MPIR_SINGULAR_T; res->iters = 0; }
        gsync<GT>();
        return;
    }
    // ---- null-space start (Sec. 2.1), right-hand side normalized by g
    double mxr = 0.0;
    for (int i = tid; i < m; i += GT) mxr = fmax(mxr, fabs(sA * b[i]));
    for (int i = tid; i < p; i += GT) mxr = fmax(mxr, fabs(sB * d[i]));
    mxr = bmax<GT>(mxr, redd);
    double g = sizeof(TF) == 4 ? pow2_of(mxr) : 1.0;
    for (int i = tid; i < m; i += GT) tw[i] = (TF)(g * sA * b[i]);
    for (int i = tid; i < p; i += GT) tbv[i] = (TF)(g * sB * d[p - 1 - i]);
    gsync<GT>();
    cta_apply_vec<GT, TF>(At, P.ldA, m, kA, TA, 1, tw, wbuf);              // c = Z^T (sA b)
    cta_trsv<GT, TF>(Bt, P.ldB, p, 1, tbv, &st, 1);                         // R~^T y~2 = P_p sB d
    for (int i = tid; i < p; i += GT) ty[q + i] = tbv[p - 1 - i];
    for (int i = tid; i < q; i += GT) ty[i] = tw[i];
    gsync<GT>();
    if (p > 0 && q > 0) cta_gemv_n<GT, TF>(At + (size_t)q * P.ldA, P.ldA, q, p, TF(-1), ty + q, ty, false);
    cta_trsv<GT, TF>(At, P.ldA, q, 0, ty, &st, 2);                          // T11 y1 = c1 - T12 y2
    for (int i = tid; i < n; i += GT) tt[i] = ty[n - 1 - i];
    gsync<GT>();
    cta_apply_vec<GT, TF>(Bt, P.ldB, n, p, TB, 0, tt, wbuf);                // x = Q^T y
    for (int i = tid; i < n; i += GT) X[i] = (double)tt[n - 1 - i] / g;
    gsync<GT>();
    int it = 0, status = MPIR_OK;
    double ratio[3] = {0, 0, 0};
    if (prm.refine != MPIR_DIRECT) {
        // ---- multipliers (Alg. 2 steps 3-4): r0 = b - A x, R^T v0 = (Q A^T r0)(q+1:n)
        for (int i = tid; i < m; i += GT) {
            double acc = 0.0;
            for (int j = 0; j < n; j++) acc = fma(A[i + (size_t)j * lda], X[j], acc);
            R[i] = b[i] - acc;
        }
        gsync<GT>();
        if (p > 0) {
            const int lane = tid & 31, warp = tid >> 5;
            for (int j = warp; j < n; j += GT / 32) {
                double acc = 0.0;
                for (int i = lane; i < m; i += 32) acc = fma(A[i + (size_t)j * lda], R[i], acc);
                acc = warp_sum(acc);
                if (lane == 0) F3[j] = acc;
            }
            gsync<GT>();
            double mf = 0.0;
            for (int i = tid; i < n; i += GT) mf = fmax(mf, fabs(sA * F3[i]));
            mf = bmax<GT>(mf, redd);
            const double g3 = sizeof(TF) == 4 ? pow2_of(mf) : 1.0;
            for (int i = tid; i < n; i += GT) tu[i] = (TF)(g3 * sA * F3[n - 1 - i]);
            gsync<GT>();
            cta_apply_vec<GT, TF>(Bt, P.ldB, n, p, TB, 1, tu, wbuf);
            cta_trsv<GT, TF>(Bt, P.ldB, p, 0, tu, &st, 1);
            for (int i = tid; i < p; i += GT) Vm[i] = (double)tu[p - 1 - i] * (sB / sA) / g3;
            gsync<GT>();
        }
        double nb2 = 0.0, nd2 = 0.0;
        for (int i = tid; i < m; i += GT) nb2 = fma(b[i], b[i], nb2);
        for (int i = tid; i < p; i += GT) nd2 = fma(d[i], d[i], nd2);
        const double nbv = sqrt(bsum<GT>(nb2, redd)), ndv = sqrt(bsum<GT>(nd2, redd));
        double best = INFINITY;
        int since = 0;
        status = MPIR_NOT_CONVERGED;
        for (it = 0; it < prm.maxit; it++) {
            // ---- FP64 residual (Alg. 2 step 6) and norms
            const int lane = tid & 31, warp = tid >> 5;
            double s1 = 0.0, s2 = 0.0, sx = 0.0, sr = 0.0, sv = 0.0;
            for (int i = tid; i < m; i += GT) {
                double acc = 0.0;
                for (int j = 0; j < n; j++) acc = fma(A[i + (size_t)j * lda], X[j], acc);
                const double f = b[i] - R[i] - acc;
                F1[i] = f;
                s1 = fma(f, f, s1);
                sr = fma(R[i], R[i], sr);
            }
            for (int i = tid; i < p; i += GT) {
                double acc = 0.0;
                for (int j = 0; j < n; j++) acc = fma(B[i + (size_t)j * ldb], X[j], acc);
                const double f = d[i] - acc;
                F2[i] = f;
                s2 = fma(f, f, s2);
                sv = fma(Vm[i], Vm[i], sv);
            }
            for (int i = tid; i < n; i += GT) sx = fma(X[i], X[i], sx);
            double s3 = 0.0;
            for (int j = warp; j < n; j += GT / 32) {
                double acc = 0.0;
                for (int i = lane; i < m; i += 32) acc = fma(-A[i + (size_t)j * lda], R[i], acc);
                for (int i = lane; i < p; i += 32) acc = fma(B[i + (size_t)j * ldb], Vm[i], acc);
                acc = warp_sum(acc);
                if (lane == 0) { F3[j] = acc; s3 = fma(acc, acc, s3); }
            }
            const double n1 = sqrt(bsum<GT>(s1, redd)), n2 = sqrt(bsum<GT>(s2, redd));
            const double n3 = sqrt(bsum<GT>(s3, redd)), nx = sqrt(bsum<GT>(sx, redd));
            const double nr = sqrt(bsum<GT>(sr, redd)), nv = sqrt(bsum<GT>(sv, redd));
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
            for (int i = tid; i < n; i += GT) tu[i] = (TF)(c3 * F3[n - 1 - i]);
            for (int i = tid; i < m; i += GT) tw[i] = (TF)(c1 * F1[i]);
            for (int i = tid; i < p; i += GT) tbv[i] = (TF)(c2 * F2[p - 1 - i]);
            gsync<GT>();
            cta_apply_vec<GT, TF>(Bt, P.ldB, n, p, TB, 1, tu, wbuf);          // step 1: u~ = Q~^T P_n f3
            cta_apply_vec<GT, TF>(At, P.ldA, m, kA, TA, 1, tw, wbuf);         // step 2: w = Z^T f1
            if (p > 0) {                                                        // step 3: R y2 = f2
                cta_trsv<GT, TF>(Bt, P.ldB, p, 1, tbv, &st, 1);
                for (int i = tid; i < p; i += GT) ty[q + i] = tbv[p - 1 - i];
                gsync<GT>();
            }
            if (q > 0) {
                for (int i = tid; i < q; i += GT) tq[i] = tu[p + q - 1 - i];
                gsync<GT>();
                cta_trsv<GT, TF>(At, P.ldA, q, 1, tq, &st, 2);                 // step 4: T11^T q1 = u1
                for (int i = tid; i < q; i += GT) ty[i] = tw[i] - tq[i];
                gsync<GT>();
                if (p > 0) cta_gemv_n<GT, TF>(At + (size_t)q * P.ldA, P.ldA, q, p, TF(-1), ty + q, ty, false);
                cta_trsv<GT, TF>(At, P.ldA, q, 0, ty, &st, 2);                 // step 5: T11 y1 = w1 - q1 - T12 y2
            }
            if (m - q > 0) {                                                    // step 6: q2 = w2 - T22 y2
                for (int i = tid; i < m - q; i += GT) tq[q + i] = tw[q + i];
                gsync<GT>();
                if (p > 0)
                    cta_gemv_n<GT, TF>(At + q + (size_t)q * P.ldA, P.ldA, m - q, p, TF(-1), ty + q, tq + q, true);
            }
            if (p > 0) {                                                        // step 8: R^T dv = T12^T q1 + T22^T q2 - u2
                for (int i = tid; i < p; i += GT) tt[i] = TF(0);
                gsync<GT>();
                if (q > 0) cta_gemv_t<GT, TF>(At + (size_t)q * P.ldA, P.ldA, q, p, TF(1), tq, tt, false);
                if (m - q > 0)
                    cta_gemv_t<GT, TF>(At + q + (size_t)q * P.ldA, P.ldA, m - q, p, TF(1), tq + q, tt, true);
                for (int i = tid; i < p; i += GT) tbv[i] = tt[p - 1 - i] - tu[i];
                gsync<GT>();
                cta_trsv<GT, TF>(Bt, P.ldB, p, 0, tbv, &st, 1);
                for (int i = tid; i < p; i += GT) Vm[i] += (double)tbv[p - 1 - i] * (sB / sA) / gam;
            }
            for (int i = tid; i < n; i += GT) tt2[i] = ty[n - 1 - i];
            gsync<GT>();
            cta_apply_vec<GT, TF>(At, P.ldA, m, kA, TA, 0, tq, wbuf);         // step 7: dr = Z q
            cta_apply_vec<GT, TF>(Bt, P.ldB, n, p, TB, 0, tt2, wbuf);         //         dx = Q^T y
            for (int i = tid; i < m; i += GT) R[i] += (double)tq[i] / gam;
            for (int i = tid; i < n; i += GT) X[i] += (double)tt2[n - 1 - i] * sA / gam;
            gsync<GT>();
        }
    }
    // ---- result
    for (int i = tid; i < n; i += GT) I.x[i] = X[i];
    gsync<GT>();
    if (tid == 0) {
        res->status = st ? ((st & 1) ? MPIR_SINGULAR_R : MPIR_SINGULAR_T) : status;
        res->iters = it;
        for (int k = 0; k < 3; k++) res->ratio[k] = ratio[k];
    }
    gsync<GT>();
}

// ------------------------------------------------------- one GLS problem --
// GLS in the xGGGLM convention (W n x m, V n x p, d -> x, y), the method of
// the single-problem solver in its reversed coordinates (Lemma 4.6, Sec. 2.2,
// Alg. 3 / Alg. 4):  [W V] = Q [R T~; 0 ...] through the first m columns
// (QR of W with Q^T V formed by the same trailing updates), C~ = P_p C^T P_n
// = Z~ T~ (p x n), T~_L = T~(0:L, 0:L) the solved triangle (L = n - m),
// Paige's start, z0 = Q [0; h], classical IR with FP64 residuals.
template <int GT, typename TF>
__device__ void solve_one_gls(const BInst &I, BResult *res, unsigned char *smem, size_t smem_bytes, TF *gscr,
                              const BParams &prm)
{
    const int tid = (threadIdx.x & (GT - 1));
    const int m = I.m, n = I.n, p = I.p, L = n - m, o = p - n + m, kC = min(n, p);
    const int ldw = I.lda, ldv = I.ldb;
    const double *W = I.A, *V = I.B, *d = I.d;
    __shared__ double redd_g[512 / GT][GT / 32];
    __shared__ int st_g[512 / GT];
    double *redd = redd_g[threadIdx.x / GT];
    int &st = st_g[threadIdx.x / GT];
    const BPlan P = gplan(m, n, p);
    const bool big_smem = bsmem_need<TF>(P, 2) <= smem_bytes;
    const bool use_stage = !big_smem && bsmem_need<TF>(P, 1) <= smem_bytes;
    double *X = reinterpret_cast<double *>(smem);
    double *Y = X + m, *Z = Y + p, *F1 = Z + n, *F2 = F1 + p, *F3 = F2 + n;
    TF *tb0 = reinterpret_cast<TF *>(smem + P.vec_d * 8);
    const int mx = max(max(m, n), max(p, 1));
    TF *tu = tb0, *tw = tu + mx, *th = tw + mx, *tg = th + mx, *tt = tg + mx, *tt2 = tt + mx;
    TF *tauW = tt2 + 2 * mx, *tauC = tauW + m, *wbuf = tauC + kC, *G = wbuf + 64;
    TF *Wb = G + 1024;
    TF *big = Wb + (size_t)32 * min(BWC, max(m + p, max(n, 1)));
    TF *stage = nullptr;
    if (!big_smem) {
        if (use_stage) stage = big;
        big = gscr;
    }
    TF *Wf = big, *Ct = big + (size_t)P.ldB * (m + p);
    TF *TW = Ct + (size_t)P.ldA * n, *TC = TW + (size_t)1024 * ceil_div(m, BNB);
    const int ldW = P.ldB, ldC = P.ldA;
    if (tid == 0) st = 0;
    // ---- scaling (Sec. 6.1) and the norms of the stop test
    double amW = 0.0, ssW = 0.0, amV = 0.0, ssV = 0.0, sd = 0.0;
    for (int e = tid; e < n * m; e += GT) {
        const double a = W[(size_t)(e % n) + (size_t)(e / n) * ldw];
        amW = fmax(amW, fabs(a));
        ssW = fma(a, a, ssW);
    }
    for (int e = tid; e < n * p; e += GT) {
        const double a = V[(size_t)(e % n) + (size_t)(e / n) * ldv];
        amV = fmax(amV, fabs(a));
        ssV = fma(a, a, ssV);
    }
    for (int i = tid; i < n; i += GT) sd = fma(d[i], d[i], sd);
    amW = bmax<GT>(amW, redd);
    amV = bmax<GT>(amV, redd);
    ssW = bsum<GT>(ssW, redd);
    ssV = bsum<GT>(ssV, redd);
    const double ndv = sqrt(bsum<GT>(sd, redd));
    const double fW = sqrt(ssW), fV = sqrt(ssV);
    if (!isfinite(ssW) || !isfinite(ssV)) {
        if (tid == 0) { res->status = MPIR_NONFINITE; res->iters = 0; }
        gsync<GT>();
        return;
    }
    const double sW = prm.scale ? pow2_of(amW) : 1.0, sV = prm.scale ? pow2_of(amV) : 1.0;
    for (int e = tid; e < n * m; e += GT) {
        const int r = e % n, c = e / n;
        Wf[r + (size_t)c * ldW] = (TF)(sW * W[r + (size_t)c * ldw]);
    }
    for (int e = tid; e < n * p; e += GT) {
        const int r = e % n, c = e / n;
        Wf[r + (size_t)(m + c) * ldW] = (TF)(sV * V[r + (size_t)c * ldv]);
    }
    gsync<GT>();
    // ---- GQR (Lemma 4.6): QR of W with C = Q^T V, then the QR of C~
    cta_geqrf<GT, TF>(Wf, ldW, n, m + p, tauW, TW, G, Wb, stage, m);
    for (int e = tid; e < p * n; e += GT) {              // Ct(i, j) = C(n-1-j, p-1-i)
        const int i = e % p, j = e / p;
        Ct[i + (size_t)j * ldC] = Wf[(n - 1 - j) + (size_t)(m + p - 1 - i) * ldW];
    }
    gsync<GT>();
    cta_geqrf<GT, TF>(Ct, ldC, p, n, tauC, TC, G, Wb, stage);
    gsync<GT>();
    // zero diagonals: R (bit 1), T~_L (bit 2)
    for (int i = tid; i < m; i += GT) if (Wf[i + (size_t)i * ldW] == TF(0)) atomicOr(&st, 1);
    for (int i = tid; i < L; i += GT) if (Ct[i + (size_t)i * ldC] == TF(0)) atomicOr(&st, 2);
    gsync<GT>();
    if (st) {
        if (tid == 0) { res->status = (st & 1) ? MPIR_SINGULAR_R : MPIR_SINGULAR_T; res->iters = 0; }
        gsync<GT>();
        return;
    }
    // ---- Paige's method (Sec. 2.2): c = Q^T (g d)
    double mxr = 0.0;
    for (int i = tid; i < n; i += GT) mxr = fmax(mxr, fabs(d[i]));
    mxr = bmax<GT>(mxr, redd);
    const double g = sizeof(TF) == 4 ? pow2_of(mxr) : 1.0;
    for (int i = tid; i < n; i += GT) tu[i] = (TF)(g * d[i]);
    gsync<GT>();
    cta_apply_vec<GT, TF>(Wf, ldW, n, m, TW, 1, tu, wbuf);
    // T22 s2 = c2  <=>  T~_L^T s~2 = P_L c2   (tg[0:L]; tg[L:p] = 0)
    for (int i = tid; i < p; i += GT) tg[i] = i < L ? tu[m + L - 1 - i] : TF(0);
    for (int i = tid; i < m; i += GT) tt[i] = TF(0);
    gsync<GT>();
    cta_trsv<GT, TF>(Ct, ldC, L, 1, tg, &st, 2);
    // R x = c1 - T12 s2,  P_m (T12 s2) = T~_12^T s~2
    if (L > 0) cta_gemv_t<GT, TF>(Ct + (size_t)L * ldC, ldC, L, m, TF(1), tg, tt, false);
    for (int i = tid; i < m; i += GT) tt2[i] = tu[i] - tt[m - 1 - i];
    gsync<GT>();
    cta_trsv<GT, TF>(Wf, ldW, m, 0, tt2, &st, 1);
    for (int i = tid; i < m; i += GT) X[i] = (double)tt2[i] * sW / g;
    gsync<GT>();
    // y = Z^T [0; s2] = P_p Z~ [s~2; 0]
    cta_apply_vec<GT, TF>(Ct, ldC, p, kC, TC, 0, tg, wbuf);
    for (int i = tid; i < p; i += GT) Y[i] = (double)tg[p - 1 - i] * sV / g;
    for (int i = tid; i < n; i += GT) Z[i] = 0.0;
    gsync<GT>();
    int it = 0, status = MPIR_OK;
    double ratio[3] = {0, 0, 0};
    if (prm.refine != MPIR_DIRECT) {
        // ---- multipliers (Alg. 4 step 3, z0 = Q [0; h]): w~ = Z~^T (P_p g y / sV)
        double my = 0.0;
        for (int i = tid; i < p; i += GT) my = fmax(my, fabs(Y[i] / sV));
        my = bmax<GT>(my, redd);
        const double gy = sizeof(TF) == 4 ? pow2_of(my) : 1.0;
        for (int i = tid; i < p; i += GT) tw[i] = (TF)(gy * Y[p - 1 - i] / sV);
        gsync<GT>();
        cta_apply_vec<GT, TF>(Ct, ldC, p, kC, TC, 1, tw, wbuf);
        for (int i = tid; i < L; i += GT) th[i] = tw[i];
        for (int i = tid; i < n; i += GT) tt[i] = TF(0);
        gsync<GT>();
        cta_trsv<GT, TF>(Ct, ldC, L, 0, th, &st, 2);                          // T~_L h~2 = w~[0:L]
        for (int i = tid; i < L; i += GT) tt[m + i] = th[L - 1 - i];
        gsync<GT>();
        cta_apply_vec<GT, TF>(Wf, ldW, n, m, TW, 0, tt, wbuf);               // z' = Q [0; P_L h~2]
        for (int i = tid; i < n; i += GT) Z[i] = (double)tt[i] * sV * sV / gy;
        gsync<GT>();
        double best = INFINITY;
        int since = 0;
        status = MPIR_NOT_CONVERGED;
        for (it = 0; it < prm.maxit; it++) {
            // ---- FP64 residual (Alg. 4 step 5): f1 = -y + V^T z, f2 = d - W x - V y, f3 = W^T z
            const int lane = tid & 31, warp = tid >> 5;
            double s1 = 0.0, s2 = 0.0, s3 = 0.0, sx = 0.0, sy = 0.0, sz = 0.0;
            for (int i = tid; i < n; i += GT) {
                double acc = d[i];
                for (int j = 0; j < m; j++) acc = fma(-W[i + (size_t)j * ldw], X[j], acc);
                for (int j = 0; j < p; j++) acc = fma(-V[i + (size_t)j * ldv], Y[j], acc);
                F2[i] = acc;
                s2 = fma(acc, acc, s2);
                sz = fma(Z[i], Z[i], sz);
            }
            for (int j = warp; j < p; j += GT / 32) {
                double acc = 0.0;
                for (int i = lane; i < n; i += 32) acc = fma(V[i + (size_t)j * ldv], Z[i], acc);
                acc = warp_sum(acc);
                if (lane == 0) { const double f = acc - Y[j]; F1[j] = f; s1 = fma(f, f, s1); }
            }
            for (int j = warp; j < m; j += GT / 32) {
                double acc = 0.0;
                for (int i = lane; i < n; i += 32) acc = fma(W[i + (size_t)j * ldw], Z[i], acc);
                acc = warp_sum(acc);
                if (lane == 0) { F3[j] = acc; s3 = fma(acc, acc, s3); }
            }
            for (int i = tid; i < m; i += GT) sx = fma(X[i], X[i], sx);
            for (int i = tid; i < p; i += GT) sy = fma(Y[i], Y[i], sy);
            const double n1 = sqrt(bsum<GT>(s1, redd)), n2 = sqrt(bsum<GT>(s2, redd));
            const double n3 = sqrt(bsum<GT>(s3, redd)), nx = sqrt(bsum<GT>(sx, redd));
            const double ny = sqrt(bsum<GT>(sy, redd)), nz = sqrt(bsum<GT>(sz, redd));
            // ---- stop test (eq. gls-stop) and stagnation
            const double den[3] = {ny + fV * nz, ndv + fW * nx + fV * ny, fW * nz};
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
            // ---- correction (Alg. 3, read with T22 g2 = u2 and dz = -Q h)
            const double gam = sizeof(TF) == 4 ? pow2_of(fmax(n1, fmax(n2 * sV, n3 * sW / sV))) : 1.0;
            const double c1 = gam, c2 = gam * sV, c3 = gam * sW / sV;
            for (int i = tid; i < n; i += GT) tu[i] = (TF)(c2 * F2[i]);
            for (int i = tid; i < p; i += GT) tw[i] = (TF)(c1 * F1[p - 1 - i]);
            for (int i = tid; i < m; i += GT) th[i] = (TF)(c3 * F3[i]);
            gsync<GT>();
            cta_apply_vec<GT, TF>(Wf, ldW, n, m, TW, 1, tu, wbuf);          // step 1: u = Q^T f2
            cta_apply_vec<GT, TF>(Ct, ldC, p, kC, TC, 1, tw, wbuf);         // step 2: w~ = Z~^T P_p f1
            cta_trsv<GT, TF>(Wf, ldW, m, 1, th, &st, 1);                     // step 3: R^T h1 = f3
            for (int i = tid; i < m; i += GT) tt[i] = th[m - 1 - i];         // h~1 = P_m h1
            for (int i = tid; i < L; i += GT) tg[i] = tu[m + L - 1 - i];     // step 4: T~_L^T g~2 = P_L u2
            for (int i = tid; i < L; i += GT) tt2[i] = TF(0);
            gsync<GT>();
            cta_trsv<GT, TF>(Ct, ldC, L, 1, tg, &st, 2);
            // step 5: T~_L h~2 = w~2 - g~2 - T~_12 h~1   (th[m:m+L])
            if (L > 0) cta_gemv_n<GT, TF>(Ct + (size_t)L * ldC, ldC, L, m, TF(1), tt, tt2, false);
            for (int i = tid; i < L; i += GT) th[m + i] = tw[i] - tg[i] - tt2[i];
            gsync<GT>();
            cta_trsv<GT, TF>(Ct, ldC, L, 0, th + m, &st, 2);
            // step 6: g~1 = w~1 - T~_22 h~1   (tg[L:p])
            if (o > 0) {
                for (int i = tid; i < o; i += GT) tg[L + i] = tw[L + i];
                gsync<GT>();
                cta_gemv_n<GT, TF>(Ct + L + (size_t)L * ldC, ldC, o, m, TF(-1), tt, tg + L, true);
            }
            // step 8: R dx = u1 - P_m (T~_22^T g~1 + T~_12^T g~2)
            for (int i = tid; i < m; i += GT) tt2[i] = TF(0);
            gsync<GT>();
            if (L > 0) cta_gemv_t<GT, TF>(Ct + (size_t)L * ldC, ldC, L, m, TF(1), tg, tt2, false);
            if (o > 0) cta_gemv_t<GT, TF>(Ct + L + (size_t)L * ldC, ldC, o, m, TF(1), tg + L, tt2, true);
            for (int i = tid; i < m; i += GT) tt[i] = tu[i] - tt2[m - 1 - i];
            gsync<GT>();
            cta_trsv<GT, TF>(Wf, ldW, m, 0, tt, &st, 1);
            for (int i = tid; i < m; i += GT) X[i] += (double)tt[i] * sW / sV / gam;
            gsync<GT>();
            // step 7: dy = P_p Z~ g~ ;  dz = -Q [h1; P_L h~2]
            cta_apply_vec<GT, TF>(Ct, ldC, p, kC, TC, 0, tg, wbuf);
            for (int i = tid; i < L; i += GT) tt2[i] = th[m + L - 1 - i];
            gsync<GT>();
            for (int i = tid; i < L; i += GT) th[m + i] = tt2[i];
            for (int i = tid; i < p; i += GT) Y[i] += (double)tg[p - 1 - i] / gam;
            gsync<GT>();
            cta_apply_vec<GT, TF>(Wf, ldW, n, m, TW, 0, th, wbuf);
            for (int i = tid; i < n; i += GT) Z[i] -= (double)th[i] * sV / gam;
            gsync<GT>();
        }
    }
    // ---- result
    for (int i = tid; i < m; i += GT) I.x[i] = X[i];
    for (int i = tid; i < p; i += GT) I.y[i] = Y[i];
    gsync<GT>();
    if (tid == 0) {
        res->status = st ? ((st & 1) ? MPIR_SINGULAR_R : MPIR_SINGULAR_T) : status;
        res->iters = it;
        for (int k = 0; k < 3; k++) res->ratio[k] = ratio[k];
    }
    gsync<GT>();
}

// ------------------------------------------------------- persistent kernel --
// NT threads per CTA in NT / GT groups; each group takes problems from the
// queue on its own (largest first) and solves them with its share of the
// dynamic shared memory (gsmem bytes) and of the global scratch.
template <int NT, int GT, typename TF>
__global__ void __launch_bounds__(NT, 1)
k_lse_batched(const BInst *__restrict__ tab, const int *__restrict__ order, int count, int *__restrict__ next,
              BResult *__restrict__ res, TF *__restrict__ gscr, size_t gstride, size_t gsmem, BParams prm)
{
    extern __shared__ __align__(16) unsigned char smem[];
    __shared__ int s_k[NT / GT];
    const int gid = threadIdx.x / GT, gtid = threadIdx.x & (GT - 1);
    unsigned char *mysm = smem + (size_t)gid * gsmem;
    TF *my = gscr + ((size_t)blockIdx.x * (NT / GT) + gid) * gstride;
    for (;;) {
        if (gtid == 0) s_k[gid] = atomicAdd(next, 1);
        gsync<GT>();
        const int k = s_k[gid];
        gsync<GT>();
        if (k >= count) break;
        const int idx = order[k];
        if (tab[idx].kind == BKIND_GLS)
            solve_one_gls<GT, TF>(tab[idx], res + idx, mysm, gsmem, my, prm);
        else
            solve_one<GT, TF>(tab[idx], res + idx, mysm, gsmem, my, prm);
    }
}

// ------------------------------------------------------------------ host --
// The dynamic shared-memory limit of a kernel instantiation is raised once
// per device to the device's opt-in maximum less the kernel's static shared
// memory (a launch with less uses less),
// so host threads launching the same instantiation with different sizes
// never lower it under one another.
template <int GT, typename TF>
static bool batched_smem_limit(size_t smem)
{
    auto kern = k_lse_batched<512, GT, TF>;
    static PerDeviceOnce once;
    once([&] {
        int dev = 0, optin = 0;
        cudaGetDevice(&dev);
        if (cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev) != cudaSuccess) optin = 0;
        cudaFuncAttributes st{};
        if (cudaFuncGetAttributes(&st, kern) != cudaSuccess) { cudaGetLastError(); return; }
        // the opt-in maximum covers static and dynamic shared memory together
        const int dyn = optin - (int)st.sharedSizeBytes;
        if (dyn <= 0 || cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, dyn) != cudaSuccess)
            cudaGetLastError();
    });
    cudaFuncAttributes fa{};
    if (cudaFuncGetAttributes(&fa, kern) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return smem <= (size_t)fa.maxDynamicSharedSizeBytes;
}

template <int GT, typename TF>
static int launch_cfg(const BInst *tab, const int *order, int count, int *next, BResult *res, TF *gscr,
                      size_t gstride, size_t smem, int grid, const BParams &prm, cudaStream_t s)
{
    constexpr int NT = 512;
    auto kern = k_lse_batched<NT, GT, TF>;
    if (!batched_smem_limit<GT, TF>(smem)) return MPIR_UNSUPPORTED;
    const size_t gsmem = (smem / (NT / GT)) & ~(size_t)15;
    cudaMemsetAsync(next, 0, sizeof(int), s);
    prof_count(K_BATCHED);
    kern<<<grid, NT, smem, s>>>(tab, order, count, next, res, gscr, gstride, gsmem, prm);
    return cudaGetLastError() == cudaSuccess ? 0 : MPIR_CUDA_ERROR;
}

template <int GT, typename TF>
static int occupancy_of(size_t smem)
{
    auto kern = k_lse_batched<512, GT, TF>;
    if (!batched_smem_limit<GT, TF>(smem)) return 0;
    int per = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, kern, 512, smem) != cudaSuccess) {
        cudaGetLastError();
        return 0;
    }
    return per;
}

} // namespace mpir
