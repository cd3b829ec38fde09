// resid.cu -- FP64 residual of the 3-block augmented systems (eq. aug-LSE,
// eq. aug-GLS; Alg. 2 step 6, Alg. 4 step 5) and the norms of the stopping
// criteria (eq. lse-stop, eq. gls-stop).  The paper computes the residual at
// u_r = double; both A x and A^T r (resp. W x, W^T z, V y, V^T z) come from a
// single read of each matrix.  Partial sums are combined in a fixed order, so
// the result is bitwise reproducible.
#include "common.cuh"
#include "kernels.h"

namespace mpir {

constexpr int RB = 256;   // rows per tile
constexpr int CB = 256;   // columns per tile

DualGemvPlan dual_gemv_plan(int rows, int cols)
{
    DualGemvPlan p;
    p.rows = rows;
    p.cols = cols;
    p.nrb = rows > 0 ? ceil_div(rows, RB) : 0;
    p.ncb = cols > 0 ? ceil_div(cols, CB) : 0;
    return p;
}

// Tile (RB x CB) per block; lane l owns rows r0 + l + 32 i (i < 8), warp w
// owns columns c0 + w + 8 j (j < 32).  Per column: 8 coalesced 256-byte
// loads, 8 FMAs into the row partials of A x, 8 FMAs + a warp sum for the
// column's A^T r partial.
__global__ void __launch_bounds__(256)
k_dual_gemv(const double *__restrict__ A, int lda, int rows, int cols, const double *__restrict__ x,
            const double *__restrict__ r, double *__restrict__ pAx, double *__restrict__ pAtr)
{
    pdl_wait();
    pdl_trigger();
    __shared__ double red[8][RB + 1];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int rb = blockIdx.x, cb = blockIdx.y;
    const int r0 = rb * RB, c0 = cb * CB;
    double ax[8], rv[8];
#pragma unroll
    for (int i = 0; i < 8; i++) {
        const int row = r0 + lane + 32 * i;
        ax[i] = 0.0;
        rv[i] = row < rows ? r[row] : 0.0;
    }
    const int cend = min(CB, cols - c0);
#pragma unroll 2
    for (int jj = warp; jj < cend; jj += 8) {
        const int c = c0 + jj;
        const double *col = A + idx2(0, c, lda);
        const double xc = x[c];
        double a[8];
#pragma unroll
        for (int i = 0; i < 8; i++) {
            const int row = r0 + lane + 32 * i;
            a[i] = row < rows ? col[row] : 0.0;
        }
        double t = 0.0;
#pragma unroll
        for (int i = 0; i < 8; i++) {
            ax[i] = fma(a[i], xc, ax[i]);
            t = fma(a[i], rv[i], t);
        }
        t = warp_sum(t);
        if (lane == 0) pAtr[(size_t)rb * cols + c] = t;
    }
#pragma unroll
    for (int i = 0; i < 8; i++) red[warp][lane + 32 * i] = ax[i];
    __syncthreads();
    for (int e = threadIdx.x; e < RB; e += 256) {
        const int row = r0 + e;
        if (row < rows) {
            double s = 0.0;
#pragma unroll
            for (int w = 0; w < 8; w++) s += red[w][e];
            pAx[(size_t)cb * rows + row] = s;
        }
    }
}

cudaError_t dual_gemv(const double *A, int lda, int rows, int cols, const double *x, const double *r,
                      double *part_Ax, double *part_Atr, cudaStream_t s)
{
    if (rows <= 0 || cols <= 0) return cudaSuccess;
    dim3 grid(ceil_div(rows, RB), ceil_div(cols, CB));
    ProfScope ps(K_DUAL_GEMV, s);
    return pdl_launch(k_dual_gemv, grid, dim3(256), 0, s, A, lda, rows, cols, x, r, part_Ax, part_Atr);
}

// ------------------------------------------------------------------ finalize --

__device__ __forceinline__ double sum_parts(const double *p, int nparts, int stride, int i)
{
    double s = 0.0;
    for (int k = 0; k < nparts; k++) s += p[(size_t)k * stride + i];
    return s;
}

// Segments of the virtual index space: 0:f1 1:f2 2:f3 3:x 4:(r|y) 5:(v|z)
template <int KIND>
__global__ void __launch_bounds__(256)
k_resid_finalize(int n0, int n1, int n2, int n3, int n4, int n5,
                 const double *__restrict__ e0, const double *__restrict__ e1,
                 const double *__restrict__ vx, const double *__restrict__ v4, const double *__restrict__ v5,
                 const double *__restrict__ pA1, int kA1, const double *__restrict__ pA2, int kA2,
                 const double *__restrict__ pB1, int kB1, const double *__restrict__ pB2, int kB2,
                 double *__restrict__ f1, double *__restrict__ f2, double *__restrict__ f3,
                 double *__restrict__ normpart)
{
    pdl_wait();
    pdl_trigger();
    __shared__ double red[8][6];
    double sq[6] = {0, 0, 0, 0, 0, 0};
    const int total = n0 + n1 + n2 + n3 + n4 + n5;
    for (int t = blockIdx.x * 256 + threadIdx.x; t < total; t += gridDim.x * 256) {
        int i = t, seg = 0;
        if (i >= n0) { i -= n0; seg = 1;
            if (i >= n1) { i -= n1; seg = 2;
                if (i >= n2) { i -= n2; seg = 3;
                    if (i >= n3) { i -= n3; seg = 4;
                        if (i >= n4) { i -= n4; seg = 5; } } } } }
        double val;
        if (KIND == 0) {
            // LSE: e0 = b (m), e1 = d (p); v4 = r (m), v5 = v (p)
            // pA1 = A x partials (kA1 x m), pA2 = A^T r partials (kA2 x n),
            // pB1 = B x partials (kB1 x p), pB2 = B^T v partials (kB2 x n)
            if (seg == 0)      { val = e0[i] - v4[i] - sum_parts(pA1, kA1, n0, i); f1[i] = val; }
            else if (seg == 1) { val = e1[i] - sum_parts(pB1, kB1, n1, i); f2[i] = val; }
            else if (seg == 2) { val = -sum_parts(pA2, kA2, n2, i) + sum_parts(pB2, kB2, n2, i); f3[i] = val; }
            else if (seg == 3) val = vx[i];
            else if (seg == 4) val = v4[i];
            else               val = v5[i];
        } else {
            // GLS: e0 = d (n); v4 = y (p), v5 = z (n)
            // pA1 = W x partials (kA1 x n), pA2 = W^T z partials (kA2 x m),
            // pB1 = V y partials (kB1 x n), pB2 = V^T z partials (kB2 x p)
            if (seg == 0)      { val = -v4[i] + sum_parts(pB2, kB2, n0, i); f1[i] = val; }
            else if (seg == 1) { val = e0[i] - sum_parts(pA1, kA1, n1, i) - sum_parts(pB1, kB1, n1, i); f2[i] = val; }
            else if (seg == 2) { val = sum_parts(pA2, kA2, n2, i); f3[i] = val; }
            else if (seg == 3) val = vx[i];
            else if (seg == 4) val = v4[i];
            else               val = v5[i];
        }
#pragma unroll
        for (int k = 0; k < 6; k++) if (k == seg) sq[k] = fma(val, val, sq[k]);
    }
#pragma unroll
    for (int k = 0; k < 6; k++) sq[k] = warp_sum(sq[k]);
    if ((threadIdx.x & 31) == 0) {
#pragma unroll
        for (int k = 0; k < 6; k++) red[threadIdx.x >> 5][k] = sq[k];
    }
    __syncthreads();
    if (threadIdx.x < 6) {
        double s = 0.0;
        for (int w = 0; w < 8; w++) s += red[w][threadIdx.x];
        normpart[(size_t)blockIdx.x * 6 + threadIdx.x] = s;
    }
}

__global__ void k_norm_final(const double *__restrict__ normpart, int nb, double *__restrict__ norms2)
{
    pdl_wait();
    pdl_trigger();
    if (threadIdx.x < 6) {
        double s = 0.0;
        for (int b = 0; b < nb; b++) s += normpart[(size_t)b * 6 + threadIdx.x];
        norms2[threadIdx.x] = s;
    }
}

static int finalize_blocks(int total)
{
    int nb = ceil_div(total, 256 * 4);
    if (nb > 304) nb = 304;
    return nb < 1 ? 1 : nb;
}

cudaError_t lse_resid_finalize(int m, int n, int p, const double *b, const double *d, const double *x,
                        const double *r, const double *v, const double *pAx, int ncbA, const double *pAtr,
                        int nrbA, const double *pBx, int ncbB, const double *pBtv, int nrbB, double *f1,
                        double *f2, double *f3, double *normpart, double *norms2, cudaStream_t s)
{
    const int total = m + p + n + n + m + p;
    const int nb = finalize_blocks(total);
    ProfScope ps(K_FINALIZE, s);
    cudaError_t e = pdl_launch(k_resid_finalize<0>, dim3(nb), dim3(256), 0, s, m, p, n, n, m, p, b, d, x, r, v, pAx,
                               ncbA, pAtr, nrbA, pBx, ncbB, pBtv, nrbB, f1, f2, f3, normpart);
    if (e != cudaSuccess) return e;
    return pdl_launch(k_norm_final, dim3(1), dim3(32), 0, s, normpart, nb, norms2);
}

cudaError_t gls_resid_finalize(int n, int m, int p, const double *d, const double *x, const double *y,
                        const double *z, const double *pWx, int ncbW, const double *pWtz, int nrbW,
                        const double *pVy, int ncbV, const double *pVtz, int nrbV, double *f1, double *f2,
                        double *f3, double *normpart, double *norms2, cudaStream_t s)
{
    const int total = p + n + m + m + p + n;
    const int nb = finalize_blocks(total);
    ProfScope ps(K_FINALIZE, s);
    cudaError_t e = pdl_launch(k_resid_finalize<1>, dim3(nb), dim3(256), 0, s, p, n, m, m, p, n, d, nullptr, x, y, z,
                               pWx, ncbW, pWtz, nrbW, pVy, ncbV, pVtz, nrbV, f1, f2, f3, normpart);
    if (e != cudaSuccess) return e;
    return pdl_launch(k_norm_final, dim3(1), dim3(32), 0, s, normpart, nb, norms2);
}

} // namespace mpir
