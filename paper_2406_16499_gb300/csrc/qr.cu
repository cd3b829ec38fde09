// qr.cu -- blocked Householder QR on GB300: cluster panel kernel + fused
// trailing update.  The generalized factorizations of the paper (GRQ for
// LSE, GQR for GLS, Lemma 4.5 / 4.6) are built from this one QR: an RQ
// factorization of C is a QR factorization of the reversed transpose of C
// (the host driver forms that copy), so every reflector is a column of a
// column-major matrix and every access below is coalesced.
#include "common.cuh"
#include "kernels.h"
#include "mpir.h"

namespace mpir {

constexpr int PANEL_NT = 512;
constexpr int PANEL_RPT = 2;                      // rows held per thread
constexpr int PANEL_ROWS_PER_CTA = PANEL_NT * PANEL_RPT;
constexpr int PANEL_MAX_CLUSTER = 16;

// ---------------------------------------------------------------------------
// Panel factorization (xGEQR2 of an L x nb panel, L = M - j0).
//
// The panel lives in registers of a thread-block cluster of `cs` CTAs
// (rows split in contiguous chunks; thread t of a CTA holds rows t + q*512).
// Column kk needs one reduction over the rows below the pivot j = j0 + kk:
//     acc[c] = sum_{i > j} a(i, kk) a(i, c)     for all c < nb,
// slot kk being the squared norm of the sub-pivot part.  With the pivot row
// a(j, :) broadcast this gives, with v = [1; scale * a(j+1:, kk)],
//     v^T a(:, c) = a(j, c) + scale * acc[c]           (c > kk, update)
//     v_c^T v_kk  = a(j, c) + scale * acc[c]           (c < kk, Gram entry)
// so the reflector, the update of the remaining columns and the strictly
// upper part of V^T V all come from that single reduction.  The reduction is
// a warp transpose-reduce, a shared-memory sum over warps and a DSMEM sum
// over the cluster (one cluster barrier per column, double-buffered).
// After the loop the compact-WY factor follows from
//     Tw^{-1} = triu(V^T V, 1) + diag(1 / tau)
// by one back substitution per column (lane k solves column k).
// ---------------------------------------------------------------------------
template <typename T, int NB>
__global__ void __launch_bounds__(PANEL_NT, 1)
k_panel_qr(T *__restrict__ A, int lda, int M, int j0, int ncols, int chunk,
           T *__restrict__ tau, T *__restrict__ Tw)
{
    constexpr int NW = PANEL_NT / 32;
    constexpr int RPT = PANEL_RPT;
    cg::cluster_group cluster = cg::this_cluster();
    const int cs = (int)cluster.num_blocks();
    const int crank = (int)cluster.block_rank();
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int L = M - j0;
    const int kpanel = min(ncols, L);

    __shared__ T red_s[NW][32];
    __shared__ T xbuf[2][32];
    __shared__ T prow[2][NB];
    __shared__ T coef_s[NB];
    __shared__ T sc_s[2];
    __shared__ T G_s[NB][NB + 1];
    __shared__ T tau_s[NB];
    __shared__ T T_s[NB][NB + 1];

    const int row_base = crank * chunk;
    const int row_end = min(row_base + chunk, L);
    int rr[RPT];
    T a[RPT][NB];
#pragma unroll
    for (int q = 0; q < RPT; q++) {
        int r = row_base + tid + q * PANEL_NT;
        rr[q] = r < row_end ? r : -1;
    }
#pragma unroll
    for (int c = 0; c < NB; c++) {
        const T *col = A + idx2(j0, j0 + c, lda);
#pragma unroll
        for (int q = 0; q < RPT; q++)
            a[q][c] = (rr[q] >= 0 && c < ncols) ? col[rr[q]] : T(0);
    }

#pragma unroll
    for (int kk = 0; kk < NB; kk++) {
        if (kk < kpanel) {
            const int par = kk & 1;
            // the reduction runs in halves of H columns to bound the number
            // of live accumulators (registers hold the panel itself)
            constexpr int H = NB > 16 ? 16 : NB;
#pragma unroll
            for (int h0 = 0; h0 < NB; h0 += H) {
                T acc[H];
#pragma unroll
                for (int c = 0; c < H; c++) acc[c] = T(0);
#pragma unroll
                for (int q = 0; q < RPT; q++) {
                    const T ak = rr[q] > kk ? a[q][kk] : T(0);   // rows below the pivot
#pragma unroll
                    for (int c = 0; c < H; c++) acc[c] = fma(ak, a[q][h0 + c], acc[c]);
                }
                T wsum = warp_transpose_reduce<T, H>(acc);
                if (lane < H) red_s[warp][h0 + lane] = wsum;
            }
#pragma unroll
            for (int q = 0; q < RPT; q++) {
                if (rr[q] == kk) {
#pragma unroll
                    for (int c = 0; c < NB; c++) prow[par][c] = a[q][c];
                }
            }
            __syncthreads();
            T tot = T(0), pj = T(0);
            if (warp == 0 && lane < NB) {
#pragma unroll
                for (int w = 0; w < NW; w++) tot += red_s[w][lane];
                xbuf[par][lane] = tot;
            }
            if (cs > 1) cluster.sync();
            if (warp == 0) {
                if (lane < NB) {
                    if (cs > 1) {
                        T t = T(0);
                        for (int r = 0; r < cs; r++) t += *cluster.map_shared_rank(&xbuf[par][lane], r);
                        tot = t;
                        pj = *cluster.map_shared_rank(&prow[par][lane], 0);
                    } else {
                        pj = prow[par][lane];
                    }
                }
                const T alpha = __shfl_sync(0xffffffffu, pj, kk);
                const T sp = __shfl_sync(0xffffffffu, tot, kk);
                T beta, tv, scale;
                if (sp == T(0)) {
                    tv = T(0); beta = alpha; scale = T(1);
                } else {
                    const T nrm = sqrt(alpha * alpha + sp);
                    beta = alpha >= T(0) ? -nrm : nrm;
                    tv = (beta - alpha) / beta;
                    scale = T(1) / (alpha - beta);
                }
                const T dot = pj + scale * tot;
                if (lane < NB) {
                    coef_s[lane] = lane > kk ? tv * dot : T(0);
                    if (lane < kk) G_s[lane][kk] = dot;
                }
                if (lane == 0) { sc_s[0] = scale; sc_s[1] = beta; tau_s[kk] = tv; }
            }
            __syncthreads();
            const T scale = sc_s[0], beta = sc_s[1];
            // columns c <= kk are untouched (their coefficient is zero), so
            // only c > kk is visited; coefficients are broadcast smem reads
            // branch-free: f = v_i (scale * a(i,kk) below the pivot, 1 on the
            // pivot row, 0 above), a(i, c) -= coef_c * f for c > kk
#pragma unroll
            for (int q = 0; q < RPT; q++) {
                const bool below = rr[q] > kk, piv = rr[q] == kk;
                const T sk = a[q][kk] * scale;
                const T f = below ? sk : (piv ? T(1) : T(0));
#pragma unroll
                for (int c = kk + 1; c < NB; c++) a[q][c] = fma(-coef_s[c], f, a[q][c]);
                a[q][kk] = below ? sk : (piv ? beta : a[q][kk]);
            }
        }
    }

    // write the factored panel back.  The base pointer is laundered so that
    // the compiler does not keep the 64 load addresses alive across the loop.
    T *Aw = A;
    asm volatile("" : "+l"(Aw));
#pragma unroll
    for (int c = 0; c < NB; c++) {
        if (c < ncols) {
            T *col = Aw + idx2(j0, j0 + c, lda);
#pragma unroll
            for (int q = 0; q < RPT; q++)
                if (rr[q] >= 0) col[rr[q]] = a[q][c];
        }
    }

    if (crank == 0 && warp == 0) {
        if (lane < kpanel) tau[j0 + lane] = tau_s[lane];
        // Tw = (triu(G, 1) + diag(1/tau))^{-1}, column `lane` by back substitution.
        const int k = lane;
        if (k < NB) {
            for (int i = NB - 1; i >= 0; i--) {
                T val = T(0);
                if (k < kpanel && i <= k) {
                    if (i == k) {
                        val = tau_s[k];
                    } else {
                        T s = T(0);
                        for (int c = i + 1; c <= k; c++) s = fma(G_s[i][c], T_s[c][k], s);
                        val = -tau_s[i] * s;
                    }
                }
                T_s[i][k] = val;
            }
            for (int i = 0; i < NB; i++) Tw[i + (size_t)k * NB] = T_s[i][k];
        }
    }
    if (cs > 1) cluster.sync();   // keep shared memory alive for remote readers
}

// ---------------------------------------------------------------------------
// Trailing update / block reflector application (xLARFB, SIMT):
//   C <- (I - V X V^T) C,  X = Tw^T (trans = 1, applies H_{k-1}..H_0) or
//   X = Tw (trans = 0, applies H_0..H_{k-1}).
// V: L x kb unit lower trapezoid (entries above the diagonal ignored).
// One CTA per 32-column slab of C: W = V^T C_slab (K = L), W <- X W,
// C_slab -= V W.  C is read twice and written once.
// ---------------------------------------------------------------------------
template <typename T, int NB>
__global__ void __launch_bounds__(256)
k_larfb_left(const T *__restrict__ V, int ldv, const T *__restrict__ Tw, int kb, int L,
             T *__restrict__ C, int ldc, int Nc, int trans)
{
    constexpr int CT = 32, RB = 64;
    constexpr int WROWS = NB * CT / 256;         // W entries per thread (NB rows)
    constexpr int UROWS = RB * CT / 256;         // update entries per thread
    __shared__ T Vs[RB][NB + 1];
    __shared__ T Cs[RB][CT + 1];
    __shared__ T Ws[NB][CT + 1];
    __shared__ T Xs[NB][NB + 1];

    const int tid = threadIdx.x;
    const int c0 = blockIdx.x * CT;
    const int col = tid % CT;
    const int rsub = tid / CT;                    // 0..7
    T acc[WROWS];
#pragma unroll
    for (int s = 0; s < WROWS; s++) acc[s] = T(0);

    for (int r0 = 0; r0 < L; r0 += RB) {
        for (int e = tid; e < RB * NB; e += 256) {
            int r = e % RB, c = e / RB, gr = r0 + r;
            T v = T(0);
            if (gr < L && c < kb) v = gr > c ? V[idx2(gr, c, ldv)] : (gr == c ? T(1) : T(0));
            Vs[r][c] = v;
        }
        for (int e = tid; e < RB * CT; e += 256) {
            int r = e % RB, c = e / RB, gr = r0 + r;
            Cs[r][c] = (gr < L && c0 + c < Nc) ? C[idx2(gr, c0 + c, ldc)] : T(0);
        }
        __syncthreads();
#pragma unroll 8
        for (int r = 0; r < RB; r++) {
            const T cv = Cs[r][col];
#pragma unroll
            for (int s = 0; s < WROWS; s++) acc[s] = fma(Vs[r][rsub + 8 * s], cv, acc[s]);
        }
        __syncthreads();
    }
#pragma unroll
    for (int s = 0; s < WROWS; s++) Ws[rsub + 8 * s][col] = acc[s];
    for (int e = tid; e < NB * NB; e += 256) {
        int i = e % NB, k = e / NB;
        T t = Tw[i + (size_t)k * NB];            // Tw(i, k)
        if (trans) Xs[k][i] = t; else Xs[i][k] = t;
    }
    __syncthreads();
    // W <- X W (X triangular, small)
    T nw[WROWS];
#pragma unroll
    for (int s = 0; s < WROWS; s++) {
        const int i = rsub + 8 * s;
        T t = T(0);
        for (int k = 0; k < NB; k++) t = fma(Xs[i][k], Ws[k][col], t);
        nw[s] = t;
    }
    __syncthreads();
#pragma unroll
    for (int s = 0; s < WROWS; s++) Ws[rsub + 8 * s][col] = nw[s];
    __syncthreads();

    for (int r0 = 0; r0 < L; r0 += RB) {
        for (int e = tid; e < RB * NB; e += 256) {
            int r = e % RB, c = e / RB, gr = r0 + r;
            T v = T(0);
            if (gr < L && c < kb) v = gr > c ? V[idx2(gr, c, ldv)] : (gr == c ? T(1) : T(0));
            Vs[r][c] = v;
        }
        __syncthreads();
#pragma unroll
        for (int s = 0; s < UROWS; s++) {
            const int r = rsub + 8 * s, gr = r0 + r;
            if (gr < L && c0 + col < Nc) {
                T t = T(0);
#pragma unroll 8
                for (int k = 0; k < NB; k++) t = fma(Vs[r][k], Ws[k][col], t);
                C[idx2(gr, c0 + col, ldc)] -= t;
            }
        }
        __syncthreads();
    }
}

// ------------------------------------------------------------------ host --

template <typename T>
static int launch_panel(T *A, int lda, int M, int j0, int ncols, T *tau, T *Tw, cudaStream_t s)
{
    constexpr int NB = panel_nb<T>();
    const int L = M - j0;
    int cs = ceil_div(L, PANEL_ROWS_PER_CTA);
    if (cs < 1) cs = 1;
    if (cs > PANEL_MAX_CLUSTER) return MPIR_UNSUPPORTED;
    const int chunk = ceil_div(L, cs);
    auto kern = k_panel_qr<T, NB>;
    static bool attr_done = false;
    if (!attr_done) {
        cudaFuncSetAttribute(kern, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
        attr_done = true;
    }
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(cs, 1, 1);
    cfg.blockDim = dim3(PANEL_NT, 1, 1);
    cfg.dynamicSmemBytes = 0;
    cfg.stream = s;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = cs;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    ProfScope ps(K_PANEL, s);
    cudaError_t e = cudaLaunchKernelEx(&cfg, kern, A, lda, M, j0, ncols, chunk, tau, Tw);
    return e == cudaSuccess ? 0 : MPIR_CUDA_ERROR;
}

template <typename T>
static int launch_larfb(const T *V, int ldv, const T *Tw, int kb, int L, T *C, int ldc, int Nc,
                        int trans, GemmPrec, cudaStream_t s)
{
    constexpr int NB = panel_nb<T>();
    if (Nc <= 0 || L <= 0 || kb <= 0) return 0;
    ProfScope ps(K_LARFB, s);
    k_larfb_left<T, NB><<<ceil_div(Nc, 32), 256, 0, s>>>(V, ldv, Tw, kb, L, C, ldc, Nc, trans);
    return cudaGetLastError() == cudaSuccess ? 0 : MPIR_CUDA_ERROR;
}

template <typename T>
int geqrf(T *A, int lda, int M, int N, T *tau, T *Tw, GemmPrec prec, cudaStream_t s)
{
    constexpr int NB = panel_nb<T>();
    const int k = M < N ? M : N;
    for (int j0 = 0; j0 < k; j0 += NB) {
        const int ncols = N - j0 < NB ? N - j0 : NB;
        const int L = M - j0;
        T *Twb = Tw + (size_t)(j0 / NB) * NB * NB;
        int rc = launch_panel<T>(A, lda, M, j0, ncols, tau, Twb, s);
        if (rc) return rc;
        const int kb = ncols < L ? ncols : L;
        const int Nc = N - j0 - ncols;
        if (Nc > 0) {
            rc = launch_larfb<T>(A + idx2(j0, j0, lda), lda, Twb, kb, L, A + idx2(j0, j0 + ncols, lda),
                                 lda, Nc, 1, prec, s);
            if (rc) return rc;
        }
    }
    return 0;
}

template <typename T>
int apply_reflectors_left(const T *V, int ldv, int M, int K, const T *Tw, int trans, T *C, int ldc,
                          int Nc, GemmPrec prec, cudaStream_t s)
{
    constexpr int NB = panel_nb<T>();
    const int nblk = ceil_div(K, NB);
    for (int t = 0; t < nblk; t++) {
        const int b = trans ? t : nblk - 1 - t;
        const int j0 = b * NB;
        const int kb = K - j0 < NB ? K - j0 : NB;
        int rc = launch_larfb<T>(V + idx2(j0, j0, ldv), ldv, Tw + (size_t)b * NB * NB, kb, M - j0,
                                 C + j0, ldc, Nc, trans, prec, s);
        if (rc) return rc;
    }
    return 0;
}

template int geqrf<float>(float *, int, int, int, float *, float *, GemmPrec, cudaStream_t);
template int geqrf<double>(double *, int, int, int, double *, double *, GemmPrec, cudaStream_t);
template int apply_reflectors_left<float>(const float *, int, int, int, const float *, int, float *,
                                          int, int, GemmPrec, cudaStream_t);
template int apply_reflectors_left<double>(const double *, int, int, int, const double *, int,
                                           double *, int, int, GemmPrec, cudaStream_t);

} // namespace mpir
