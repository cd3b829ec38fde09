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

// ---------------------------------------------------------------------------
// Residuals in double-double (u_r = u^2, the u_r < u variant of the
// refinement: with it the forward error reaches about u instead of kappa u).
// Sums of FP64 products kept as unevaluated pairs (hi, lo) with the
// error-free transformations of Knuth (TwoSum) and the FMA product
// (TwoProd: a b = p + fma(a, b, -p) exactly); each accumulation adds the
// product's error term to the pair's low part (relative error O(u^2)).
// ---------------------------------------------------------------------------
struct DD { double hi, lo; };

// (the _rn intrinsics are never contracted into an FMA, which would break
// the error-free transformations)
__device__ __forceinline__ DD dd_two_sum(double a, double b)
{
    const double s = __dadd_rn(a, b), bb = __dsub_rn(s, a);
    return DD{s, __dadd_rn(__dsub_rn(a, __dsub_rn(s, bb)), __dsub_rn(b, bb))};
}
__device__ __forceinline__ DD dd_fast_two_sum(double a, double b)
{
    const double s = __dadd_rn(a, b);
    return DD{s, __dsub_rn(b, __dsub_rn(s, a))};
}
__device__ __forceinline__ DD dd_add(DD a, DD b)
{
    DD s = dd_two_sum(a.hi, b.hi);
    const DD t = dd_two_sum(a.lo, b.lo);
    s.lo = __dadd_rn(s.lo, t.hi);
    s = dd_fast_two_sum(s.hi, s.lo);
    s.lo = __dadd_rn(s.lo, t.lo);
    return dd_fast_two_sum(s.hi, s.lo);
}
// acc + a b
__device__ __forceinline__ DD dd_mac(DD acc, double a, double b)
{
    const double p = __dmul_rn(a, b);
    const double e = fma(a, b, -p);
    DD t = dd_two_sum(acc.hi, p);
    t.lo = __dadd_rn(t.lo, __dadd_rn(acc.lo, e));
    return dd_fast_two_sum(t.hi, t.lo);
}

// out[i] = sum_j M(i, j) x[j] (one thread per row; coalesced column walks)
__global__ void __launch_bounds__(256)
k_rowdot_dd(const double *__restrict__ M, int ld, int rows, int cols, const double *__restrict__ x,
            double *__restrict__ hi, double *__restrict__ lo)
{
    const int i = blockIdx.x * 256 + threadIdx.x;
    if (i >= rows) return;
    DD acc{0.0, 0.0};
    const double *row = M + i;
    for (int j = 0; j < cols; j++) acc = dd_mac(acc, row[(size_t)j * ld], x[j]);
    hi[i] = acc.hi;
    lo[i] = acc.lo;
}

// out[j] = sum_i M(i, j) r[i] (one warp per column)
__global__ void __launch_bounds__(256)
k_coldot_dd(const double *__restrict__ M, int ld, int rows, int cols, const double *__restrict__ r,
            double *__restrict__ hi, double *__restrict__ lo)
{
    const int j = blockIdx.x * 8 + (threadIdx.x >> 5), lane = threadIdx.x & 31;
    if (j >= cols) return;
    const double *col = M + (size_t)j * ld;
    DD acc{0.0, 0.0};
    for (int i = lane; i < rows; i += 32) acc = dd_mac(acc, col[i], r[i]);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        const DD other{__shfl_xor_sync(0xffffffffu, acc.hi, o), __shfl_xor_sync(0xffffffffu, acc.lo, o)};
        acc = dd_add(acc, other);
    }
    if (lane == 0) { hi[j] = acc.hi; lo[j] = acc.lo; }
}

// out = round(s0 a + s1 c + su u + sw w): a, c plain vectors, u, w
// double-double pairs (any of them NULL: absent); the signs are +-1, so the
// first sum is exact as a pair
__global__ void k_combine_dd(int n, const double *__restrict__ a, double s0, const double *__restrict__ c, double s1,
                             const double *__restrict__ uh, const double *__restrict__ ul, double su,
                             const double *__restrict__ wh, const double *__restrict__ wl, double sw,
                             double *__restrict__ out)
{
    const int i = blockIdx.x * 256 + threadIdx.x;
    if (i >= n) return;
    DD acc = dd_two_sum(a ? s0 * a[i] : 0.0, c ? s1 * c[i] : 0.0);
    if (uh) acc = dd_add(acc, DD{su * uh[i], su * ul[i]});
    if (wh) acc = dd_add(acc, DD{sw * wh[i], sw * wl[i]});
    out[i] = acc.hi;
}

// norms2[k] = sum of squares of vec[k] (length len[k]) for k < 6, one block
// each, fixed-order tree reduction
struct Vec6 { const double *v[6]; int len[6]; };
__global__ void __launch_bounds__(256) k_norms6(Vec6 V, double *__restrict__ norms2)
{
    __shared__ double red[256];
    const int k = blockIdx.x;
    double s = 0.0;
    if (V.v[k])
        for (int i = threadIdx.x; i < V.len[k]; i += 256) s = fma(V.v[k][i], V.v[k][i], s);
    red[threadIdx.x] = s;
    __syncthreads();
    for (int o = 128; o > 0; o >>= 1) {
        if (threadIdx.x < o) red[threadIdx.x] += red[threadIdx.x + o];
        __syncthreads();
    }
    if (threadIdx.x == 0) norms2[k] = red[0];
}

// out[0] += || a - b ||^2 (one block)
__global__ void __launch_bounds__(256) k_diffnorm2(const double *__restrict__ a, const double *__restrict__ b, int n,
                                                   double *__restrict__ out, int accumulate)
{
    __shared__ double red[256];
    double s = 0.0;
    for (int i = threadIdx.x; i < n; i += 256) {
        const double d = a[i] - b[i];
        s = fma(d, d, s);
    }
    red[threadIdx.x] = s;
    __syncthreads();
    for (int o = 128; o > 0; o >>= 1) {
        if (threadIdx.x < o) red[threadIdx.x] += red[threadIdx.x + o];
        __syncthreads();
    }
    if (threadIdx.x == 0) out[0] = (accumulate ? out[0] : 0.0) + red[0];
}

static int g256(int n) { return n > 0 ? ceil_div(n, 256) : 1; }

cudaError_t lse_resid_dd(int m, int n, int p, const double *A, int lda, const double *B, int ldb, const double *b,
                         const double *d, const double *x, const double *r, const double *v, double *scr,
                         double *f1, double *f2, double *f3, double *norms2, cudaStream_t s)
{
    // scr: A x (hi, lo: m each), B x (p each), A^T r (n each), B^T v (n each)
    double *axh = scr, *axl = axh + m, *bxh = axl + m, *bxl = bxh + p, *atrh = bxl + p, *atrl = atrh + n;
    double *btvh = atrl + n, *btvl = btvh + n;
    ProfScope ps(K_DUAL_GEMV, s);
    if (m > 0) {
        k_rowdot_dd<<<g256(m), 256, 0, s>>>(A, lda, m, n, x, axh, axl);
        k_coldot_dd<<<ceil_div(n, 8), 256, 0, s>>>(A, lda, m, n, r, atrh, atrl);
    }
    if (p > 0) {
        k_rowdot_dd<<<g256(p), 256, 0, s>>>(B, ldb, p, n, x, bxh, bxl);
        k_coldot_dd<<<ceil_div(n, 8), 256, 0, s>>>(B, ldb, p, n, v, btvh, btvl);
    }
    // f1 = b - r - A x, f2 = d - B x, f3 = -A^T r + B^T v
    if (m > 0) k_combine_dd<<<g256(m), 256, 0, s>>>(m, b, 1.0, r, -1.0, axh, axl, -1.0, nullptr, nullptr, 0.0, f1);
    if (p > 0)
        k_combine_dd<<<g256(p), 256, 0, s>>>(p, d, 1.0, nullptr, 0.0, bxh, bxl, -1.0, nullptr, nullptr, 0.0, f2);
    k_combine_dd<<<g256(n), 256, 0, s>>>(n, nullptr, 0.0, nullptr, 0.0, m > 0 ? atrh : nullptr, atrl, -1.0,
                                         p > 0 ? btvh : nullptr, btvl, 1.0, f3);
    Vec6 V{{m > 0 ? f1 : nullptr, p > 0 ? f2 : nullptr, f3, x, m > 0 ? r : nullptr, p > 0 ? v : nullptr},
           {m, p, n, n, m, p}};
    k_norms6<<<6, 256, 0, s>>>(V, norms2);
    return cudaGetLastError();
}

cudaError_t gls_resid_dd(int n, int m, int p, const double *W, int ldw, const double *V, int ldv, const double *d,
                         const double *x, const double *y, const double *z, double *scr, double *f1, double *f2,
                         double *f3, double *norms2, cudaStream_t s)
{
    // scr: W x, V y (hi, lo: n each), V^T z (p each), W^T z (m each)
    double *wxh = scr, *wxl = wxh + n, *vyh = wxl + n, *vyl = vyh + n, *vtzh = vyl + n, *vtzl = vtzh + p;
    double *wtzh = vtzl + p, *wtzl = wtzh + m;
    ProfScope ps(K_DUAL_GEMV, s);
    if (m > 0) {
        k_rowdot_dd<<<g256(n), 256, 0, s>>>(W, ldw, n, m, x, wxh, wxl);
        k_coldot_dd<<<ceil_div(m, 8), 256, 0, s>>>(W, ldw, n, m, z, wtzh, wtzl);
    }
    if (p > 0) {
        k_rowdot_dd<<<g256(n), 256, 0, s>>>(V, ldv, n, p, y, vyh, vyl);
        k_coldot_dd<<<ceil_div(p, 8), 256, 0, s>>>(V, ldv, n, p, z, vtzh, vtzl);
    }
    // f1 = -y + V^T z, f2 = d - W x - V y, f3 = W^T z
    if (p > 0)
        k_combine_dd<<<g256(p), 256, 0, s>>>(p, y, -1.0, nullptr, 0.0, vtzh, vtzl, 1.0, nullptr, nullptr, 0.0, f1);
    k_combine_dd<<<g256(n), 256, 0, s>>>(n, d, 1.0, nullptr, 0.0, m > 0 ? wxh : nullptr, wxl, -1.0,
                                         p > 0 ? vyh : nullptr, vyl, -1.0, f2);
    if (m > 0)
        k_combine_dd<<<g256(m), 256, 0, s>>>(m, nullptr, 0.0, nullptr, 0.0, wtzh, wtzl, 1.0, nullptr, nullptr, 0.0,
                                             f3);
    Vec6 Vv{{p > 0 ? f1 : nullptr, f2, m > 0 ? f3 : nullptr, m > 0 ? x : nullptr, p > 0 ? y : nullptr, z},
            {p, n, m, m, p, n}};
    k_norms6<<<6, 256, 0, s>>>(Vv, norms2);
    return cudaGetLastError();
}

cudaError_t diff_norm2(const double *a, const double *b, int n, double *out, int accumulate, cudaStream_t s)
{
    k_diffnorm2<<<1, 256, 0, s>>>(a, b, n, out, accumulate);
    return cudaGetLastError();
}

} // namespace mpir
