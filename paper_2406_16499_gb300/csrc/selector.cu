// selector.cu -- the learned precision / refinement selector: problem
// features with a Golub-Kahan-Lanczos condition sketch, and the MLP
// (16 -> 64 -> 64 -> 6, ReLU, softmax) with its training kernels.
//
// Features (16): log m, log n, log(p+1), n/m, p/n, kind, complex flag,
// log ||A||_F, log ||B||_F, log ||b||, log ||d||, log(||A||_F/||B||_F),
// log kappa^(A), log kappa^(B), log kappa^([A; B]), log(flop estimate)
// (GLS: log n, log m, log(p+1), m/n, n/p, kind 1, 0, log ||W||_F, log ||V||_F,
// log ||d||, 0, log(||W||/||V||), kappa^ of W, V and [W, V]).
// kappa^ = sigma_max(B_k) / sigma_min(B_k) of k = min(16, rows, columns)
// steps of Golub-Kahan-Lanczos bidiagonalization (FP32 vectors and
// products of the FP64 data; every new vector reorthogonalized once against
// the previous ones) from a given start vector, stopped early only at
// breakdown: an alpha or beta below 2^-26 of the largest one so far (the
// Krylov space is exhausted).  On tall blocks the Ritz values then follow the
// FP64 definition to within u_single ||M||_F up to kappa^ ~ 1e8; a
// rank-deficient block reads as kappa^ at the FP32 noise level (1e6-1e8).
// On a wide block FP32 rounding leaves components in the null space that
// grow by alpha/beta per step, so long sketches of wide blocks with
// alpha/beta well above 1 can drift.  The extreme singular values of the
// k x k bidiagonal come from FP32 bisection on its Golub-Kahan tridiagonal
// form (zero diagonal), which resolves them to a relative O(k u_single)
// however small they are.
//
// Blocks up to 16 CTAs' shared memory run with the stacked matrix resident
// in shared memory (k_features_sm); larger ones read it from an FP32 copy in
// global memory (k_features).
//
// MLP parameters are one FP32 array (layout below); every forward rounds
// the weights to bfloat16 and accumulates in FP32.
#include <cooperative_groups.h>

#include "common.cuh"
#include "kernels.h"
#include "mpir.h"
#include "selector.h"

namespace cg = cooperative_groups;

namespace mpir {

// ============================================================ features ==
constexpr int FT_THREADS = 512;
constexpr int FT_KMAX = 16;
constexpr float GKL_BREAKDOWN_F = 1.4901161e-08f;   // 2^-26: breakdown of the Krylov space only

struct FeatView {
    int kind;          // 0 LSE ([A; B], runs split rows), 1 GLS ([W, V], runs split columns)
    int R, C;          // stacked rows / columns
    int m, n, p;       // the API's dimensions
    const double *A;   // LSE A (m x n) / GLS W (n x m)
    const double *B;   // LSE B (p x n) / GLS V (n x p)
    int lda, ldb;

    __device__ __forceinline__ double at(int i, int j) const
    {
        if (kind == 0) return i < m ? A[i + (size_t)j * lda] : B[(i - m) + (size_t)j * ldb];
        return j < m ? A[i + (size_t)j * lda] : B[i + (size_t)(j - m) * ldb];
    }
    // f(j, a) for every column j of row i, in segments with plain strided
    // pointers (loads independent of the arithmetic, so they pipeline)
    template <typename F> __device__ __forceinline__ void row_each(int i, F f) const
    {
        if (kind == 0) {
            const double *pr = i < m ? A + i : B + (i - m);
            const size_t ld = i < m ? (size_t)lda : (size_t)ldb;
#pragma unroll 4
            for (int j = 0; j < C; j++) f(j, pr[(size_t)j * ld]);
        } else {
#pragma unroll 4
            for (int j = 0; j < m; j++) f(j, A[i + (size_t)j * lda]);
#pragma unroll 4
            for (int j = 0; j < p; j++) f(m + j, B[i + (size_t)j * ldb]);
        }
    }
    // f(i, a) for the rows lo + lane, lo + lane + 32, ... < hi of column j
    template <typename F> __device__ __forceinline__ void col_each(int j, int lo, int hi, int lane, F f) const
    {
        if (kind == 0) {
            const double *ca = A + (size_t)j * lda;
#pragma unroll 4
            for (int i = lo + lane; i < min(hi, m); i += 32) f(i, ca[i]);
            const double *cb = B + (size_t)j * ldb - m;
            const int s0 = max(lo, m);
#pragma unroll 4
            for (int i = s0 + lane; i < hi; i += 32) f(i, cb[i]);
        } else {
            const double *c = j < m ? A + (size_t)j * lda : B + (size_t)(j - m) * ldb;
#pragma unroll 4
            for (int i = lo + lane; i < hi; i += 32) f(i, c[i]);
        }
    }
    // run 0: A (W), 1: B (V), 2: stacked; membership of row i / column j
    __device__ __forceinline__ bool row_in(int r, int i) const
    {
        if (kind == 1 || r == 2) return true;
        return r == 0 ? i < m : i >= m;
    }
    __device__ __forceinline__ bool col_in(int r, int j) const
    {
        if (kind == 0 || r == 2) return true;
        return r == 0 ? j < m : j >= m;
    }
};

__device__ __forceinline__ double lg(double x) { return log(fmin(fmax(x, 1e-300), 1e300)); }

// The 16 features from the norms and the three condition sketches.
__device__ void feature_vector(const FeatView &V, double fA, double fB, double nb2, double nd2, const double *kap,
                               float *out)
{
    const double m = V.m, n = V.n, p = V.p;
    double f[16];
    if (V.kind == 0) {
        const double kA = fmin(m, n);
        const double fl = 2.0 * n * p * p - 2.0 * p * p * p / 3.0 + 4.0 * m * n * p + 2.0 * m * n * kA -
                          2.0 * kA * kA * kA / 3.0;
        const double ff[16] = {lg(m), lg(n), log(p + 1.0), n / m, p / n, 0.0, 0.0, lg(fA), lg(fB),
                               lg(sqrt(nb2)), lg(sqrt(nd2)), lg(fA) - lg(fB), lg(kap[0]), lg(kap[1]),
                               lg(kap[2]), lg(fl)};
        for (int q = 0; q < 16; q++) f[q] = ff[q];
    } else {
        const double kC = fmin(n, p);
        const double fl = 2.0 * n * m * m - 2.0 * m * m * m / 3.0 + 4.0 * n * m * p + 2.0 * p * n * kC -
                          2.0 * kC * kC * kC / 3.0;
        const double ff[16] = {lg(n), lg(m), log(p + 1.0), m / n, n / p, 1.0, 0.0, lg(fA), lg(fB),
                               lg(sqrt(nb2)), 0.0, lg(fA) - lg(fB), lg(kap[0]), lg(kap[1]),
                               lg(kap[2]), lg(fl)};
        for (int q = 0; q < 16; q++) f[q] = ff[q];
    }
    for (int q = 0; q < 16; q++) out[q] = (float)f[q];
}

// Number of eigenvalues below x of the Golub-Kahan tridiagonal (zero
// diagonal, squared off-diagonals e2[0 .. len-1]) in FP32: the ratio form of
// the Sturm sequence, a pivot of magnitude below pivmin replaced by -pivmin.
// Each step perturbs e2[i] and x by a few units of FP32 rounding, so the
// count is exact for a bidiagonal whose entries differ from the given ones
// by O(u_single) relatively, and the singular values it brackets carry a
// relative error of O(k u_single) (Demmel and Kahan's relative perturbation
// bound for bidiagonals).
__device__ __forceinline__ int gk_count_f(const float *e2, int len, float x, float pivmin)
{
    int c = 0;
    float q = -x;
    if (q < 0.f) c++;
    for (int i = 0; i < len; i++) {
        if (fabsf(q) < pivmin) q = -pivmin;
        q = -x - e2[i] / q;
        if (q < 0.f) c++;
    }
    return c;
}

// sigma_max / sigma_min of the three k x k upper bidiagonals (alpha[r],
// beta[r], kk[r] steps), by the whole block in FP32 (the FP64 units of this
// part are far too few for a Sturm-sequence search): the bidiagonal is
// scaled by a power of two to entries <= 1, the runs r = 0, 1, 2 take five
// warps each (160 multisection points per round), sigma_max on [0,
// Gershgorin bound] in 4 rounds (161^-4 < 2^-29), sigma_min first in log2
// scale on [sigma_max 2^-100, sigma_max] (3 rounds) and then linearly inside
// the bracket (2 rounds, below FP32 resolution).  kap[r] = sigma_max /
// sigma_min (infinite below 2^-100 sigma_max, 1 for an empty run).  Every
// thread of the block must call it.
__device__ void bidiag_cond_block(const double (*alpha)[FT_KMAX], const double (*beta)[FT_KMAX], const int *kk,
                                  double *kap)
{
    constexpr int G = 5, NP = G * 32;
    __shared__ unsigned bal[3][G];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int r = warp / G, g = warp % G;
    const bool act = r < 3;
    const int k = act ? kk[r] : 0;
    double amax = 0.0;
    for (int i = 0; i < k; i++) {
        amax = fmax(amax, fabs(alpha[r][i]));
        if (i < k - 1) amax = fmax(amax, fabs(beta[r][i]));
    }
    const double sc = amax > 0 ? exp2(-ceil(log2(amax))) : 1.0;     // entries scaled to <= 1
    float e2[2 * FT_KMAX];
    float hi = 0.f;
    for (int i = 0; i < k; i++) {
        const double a = alpha[r][i] * sc, b = i < k - 1 ? beta[r][i] * sc : 0.0, bp = i > 0 ? beta[r][i - 1] * sc : 0.0;
        e2[2 * i] = (float)(a * a);
        if (i < k - 1) e2[2 * i + 1] = (float)(b * b);
        hi = fmaxf(hi, (float)(fabs(a) + fabs(b) + fabs(bp)));
    }
    const int len = 2 * k - 1;
    const float pivmin = 1e-36f;
    const int pt = g * 32 + lane;
    auto first_true = [&](bool v) {
        const unsigned b = __ballot_sync(0xffffffffu, v);
        if (act && lane == 0) bal[r][g] = b;
        __syncthreads();
        int f = NP;
        if (act)
            for (int q = 0; q < G; q++)
                if (bal[r][q]) { f = q * 32 + __ffs(bal[r][q]) - 1; break; }
        __syncthreads();
        return f;
    };
    // bracket [lo, up] refined to the first of NP interior points where test holds
    auto section = [&](float &lo, float &up, bool holds) {
        const int f = first_true(holds);
        const float nlo = f == 0 ? lo : lo + (up - lo) * (float)f / (float)(NP + 1);
        const float nup = f == NP ? up : lo + (up - lo) * (float)(f + 1) / (float)(NP + 1);
        lo = nlo;
        up = nup;
    };
    const bool live = act && k > 0 && hi > 0.f;
    float lo = 0.f, up = hi;
    for (int round = 0; round < 4; round++) {
        const float x = lo + (up - lo) * (float)(pt + 1) / (float)(NP + 1);
        section(lo, up, live && gk_count_f(e2, len, x, pivmin) - k >= k);    // sigma_max < x
    }
    const float smax = up;
    float llo = live ? log2f(smax) - 100.f : 0.f, lup = live ? log2f(smax) : 0.f;
    const bool tiny = live && gk_count_f(e2, len, exp2f(llo), pivmin) - k >= 1;
    const bool go = live && !tiny;
    for (int round = 0; round < 3; round++) {
        const float y = llo + (lup - llo) * (float)(pt + 1) / (float)(NP + 1);
        section(llo, lup, go && gk_count_f(e2, len, exp2f(y), pivmin) - k >= 1);   // sigma_min < 2^y
    }
    float slo = exp2f(llo), sup = exp2f(lup);
    for (int round = 0; round < 2; round++) {
        const float x = slo + (sup - slo) * (float)(pt + 1) / (float)(NP + 1);
        section(slo, sup, go && gk_count_f(e2, len, x, pivmin) - k >= 1);          // sigma_min < x
    }
    if (act && g == 0 && lane == 0) kap[r] = !live ? 1.0 : tiny ? INFINITY : (double)smax / (double)sup;
    __syncthreads();
}

// One cluster; CTA `rank` owns stacked rows [r0, r1) of the u vectors and
// the column slice [c0, c1) of the v vectors.  ws (global):
// part[CS][3][C] (partial M^T u), U[3][KMAX][R], Vb[3][KMAX + 1][C].
// Every new u and v is reorthogonalized against the previous ones of its
// run (one classical Gram-Schmidt pass).
__global__ void __launch_bounds__(FT_THREADS, 1)
k_features(FeatView V, const double *__restrict__ s, const double *__restrict__ bv, int nbv,
           const double *__restrict__ dv, int ndv, double *__restrict__ ws, int k, float *__restrict__ out)
{
    extern __shared__ float vst[];             // 3 x C: the v vectors of the current step
    cg::cluster_group cl = cg::this_cluster();
    const int CS = (int)cl.num_blocks(), rank = (int)cl.block_rank();
    auto csync = [&]() { if (CS == 1) __syncthreads(); else cl.sync(); };
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    constexpr int NW = FT_THREADS / 32;
    constexpr int NS = 3 * FT_KMAX;            // reduction slots
    const int R = V.R, C = V.C;
    float *part = reinterpret_cast<float *>(ws);
    float *U = part + (size_t)CS * 3 * C;      // U[r][j][i] at U[(r * KMAX + j) * R + i]
    float *Vb = U + (size_t)3 * FT_KMAX * R;   // Vb[r][j][c] at Vb[(r * (KMAX + 1) + j) * C + c]
    float *M32 = Vb + (size_t)3 * (FT_KMAX + 1) * C;   // the stacked matrix in FP32, R x C, ld R
    auto Ui = [&](int r, int j) { return U + ((size_t)r * FT_KMAX + j) * R; };
    auto Vj = [&](int r, int j) { return Vb + ((size_t)r * (FT_KMAX + 1) + j) * C; };
    const int rows_per = ceil_div(R, CS);
    const int r0 = min(R, rank * rows_per), r1 = min(R, r0 + rows_per);
    const int cols_per = ceil_div(C, CS);
    const int c0 = min(C, rank * cols_per), c1 = min(C, c0 + cols_per);
    __shared__ float red[NW][NS];
    __shared__ float cred[NS];
    __shared__ float tot[NS];
    __shared__ double totd[2];                 // FP64 sums (Frobenius norms)
    __shared__ double alpha[3][FT_KMAX], beta[3][FT_KMAX];
    __shared__ int kk[3];

    // cluster sums of per-thread values v[0..ns) (results in tot[] on every CTA)
    // FP32 throughout: a warp-wide FP64 instruction costs tens of cycles here
    auto csum = [&](const float *v, int ns) {
        for (int q0 = 0; q0 < ns; q0 += 32) {       // 32 slots per transposed warp reduction
            float w32[32];
#pragma unroll
            for (int q = 0; q < 32; q++) w32[q] = q0 + q < ns ? v[q0 + q] : 0.f;
            const float t = warp_transpose_reduce<float, 32>(w32);
            if (q0 + lane < ns) red[warp][q0 + lane] = t;
        }
        __syncthreads();
        if (tid < ns) {
            float t = 0.f;
            for (int w = 0; w < NW; w++) t += red[w][tid];
            cred[tid] = t;
        }
        csync();
        if (tid < ns) {
            float t = 0.f;
            for (int q = 0; q < CS; q++) t += cl.map_shared_rank(cred, q)[tid];
            tot[tid] = t;
        }
        csync();
    };
    // FP64 cluster sum of two values (norms of the FP64 data)
    auto csum2d = [&](double a0, double a1) {
        a0 = warp_sum(a0);
        a1 = warp_sum(a1);
        __shared__ double rd[NW][2], cd[2];
        if (lane == 0) { rd[warp][0] = a0; rd[warp][1] = a1; }
        __syncthreads();
        if (tid < 2) {
            double t = 0.0;
            for (int w = 0; w < NW; w++) t += rd[w][tid];
            cd[tid] = t;
        }
        csync();
        if (tid < 2) {
            double t = 0.0;
            for (int q = 0; q < CS; q++) t += cl.map_shared_rank(cd, q)[tid];
            totd[tid] = t;
        }
        csync();
    };

    // ---- Frobenius norms of the two blocks
    {
        double v2[2] = {0.0, 0.0};
        for (int i = r0 + tid; i < r1; i += FT_THREADS)
            V.row_each(i, [&](int j, double a) {
                const bool first = V.kind == 0 ? i < V.m : j < V.m;
                if (first) v2[0] = fma(a, a, v2[0]); else v2[1] = fma(a, a, v2[1]);
                M32[i + (size_t)j * R] = (float)a;   // this CTA's rows, converted once
            });
        csum2d(v2[0], v2[1]);
    }
    const double fA = sqrt(totd[0]), fB = sqrt(totd[1]);
    // ---- start vectors: v_r = s restricted to run r's columns, normalized
    {
        float s2[3] = {0, 0, 0};
        for (int j = tid; j < C; j += FT_THREADS)
            for (int r = 0; r < 3; r++) if (V.col_in(r, j)) s2[r] = fmaf((float)s[j], (float)s[j], s2[r]);
        for (int r = 0; r < 3; r++) {
            const float t = warp_sum(s2[r]);
            if (lane == 0) red[warp][r] = t;
        }
        __syncthreads();
        if (tid < 3) {
            float t = 0.f;
            for (int w = 0; w < NW; w++) t += red[w][tid];
            tot[tid] = sqrtf(t);
            kk[tid] = 0;
        }
        __syncthreads();
        for (int j = c0 + tid; j < c1; j += FT_THREADS)
            for (int r = 0; r < 3; r++) Vj(r, 0)[j] = (V.col_in(r, j) && tot[r] > 0) ? (float)s[j] / tot[r] : 0.f;
        csync();
    }
    bool live[3];
    for (int r = 0; r < 3; r++) live[r] = (r == 1 && V.p == 0) ? false : true;
    if (V.kind == 1 && V.m == 0) live[0] = false;
    // rows and columns of each run's block; steps min(k, rows, columns)
    int rr[3], cc[3], klim[3];
    if (V.kind == 0) {
        rr[0] = V.m; rr[1] = V.p; rr[2] = V.m + V.p;
        cc[0] = cc[1] = cc[2] = V.n;
    } else {
        rr[0] = rr[1] = rr[2] = V.n;
        cc[0] = V.m; cc[1] = V.p; cc[2] = V.m + V.p;
    }
    bool wide[3];
    for (int r = 0; r < 3; r++) {
        klim[r] = min(k, min(rr[r], cc[r]));
        wide[r] = live[r] && rr[r] < cc[r];
    }
    // wide blocks: start from M^T M s (normalized), inside range(M^T), so the
    // Ritz values interlace the nonzero singular values
    if (wide[0] || wide[1] || wide[2]) {
        for (int e = tid; e < 3 * C; e += FT_THREADS) vst[e] = __ldcg(Vj(e / C, 0) + e % C);
        __syncthreads();
        for (int i = r0 + tid; i < r1; i += FT_THREADS) {
            float a3[3] = {0, 0, 0};
            const float *mr = M32 + i;
#pragma unroll 4
            for (int j = 0; j < C; j++) {
                const float a = mr[(size_t)j * R];
#pragma unroll
                for (int r = 0; r < 3; r++)
                    if (V.col_in(r, j)) a3[r] = fmaf(a, vst[r * C + j], a3[r]);
            }
            for (int r = 0; r < 3; r++)
                if (wide[r] && V.row_in(r, i)) Ui(r, 0)[i] = a3[r];
        }
        __syncthreads();
        for (int j = warp; j < C; j += NW) {
            float p3[3] = {0, 0, 0};
            const float *mc = M32 + (size_t)j * R;
#pragma unroll 4
            for (int i = r0 + lane; i < r1; i += 32) {
                const float a = mc[i];
#pragma unroll
                for (int r = 0; r < 3; r++)
                    if (wide[r] && V.row_in(r, i) && V.col_in(r, j)) p3[r] = fmaf(a, Ui(r, 0)[i], p3[r]);
            }
#pragma unroll
            for (int r = 0; r < 3; r++) p3[r] = warp_sum(p3[r]);
            if (lane == 0)
                for (int r = 0; r < 3; r++) part[((size_t)rank * 3 + r) * C + j] = p3[r];
        }
        csync();
        float n3[3] = {0, 0, 0};
        for (int j = c0 + tid; j < c1; j += FT_THREADS)
            for (int r = 0; r < 3; r++) {
                if (!wide[r]) continue;
                float w = 0.f;
                if (V.col_in(r, j))
                    for (int q = 0; q < CS; q++) w += __ldcg(part + ((size_t)q * 3 + r) * C + j);
                Vj(r, 0)[j] = w;
                n3[r] = fmaf(w, w, n3[r]);
            }
        csum(n3, 3);
        for (int j = c0 + tid; j < c1; j += FT_THREADS)
            for (int r = 0; r < 3; r++)
                if (wide[r]) Vj(r, 0)[j] = tot[r] > 0 ? Vj(r, 0)[j] * rsqrtf(tot[r]) : 0.f;
        csync();
    }
    float bprev[3] = {0, 0, 0}, big[3] = {0, 0, 0};
    float acc[NS];
    for (int t = 0; t < k; t++) {
        for (int r = 0; r < 3; r++) if (t >= klim[r]) live[r] = false;
        // u'_r = M_r v_t - beta u_{t-1} into U[r][t] (this CTA's rows)
        // the v vectors of this step, staged in shared memory once per CTA
        for (int e = tid; e < 3 * C; e += FT_THREADS) vst[e] = __ldcg(Vj(e / C, t) + e % C);
        float bpf[3];
        for (int r = 0; r < 3; r++) bpf[r] = bprev[r];
        __syncthreads();
        for (int i = r0 + tid; i < r1; i += FT_THREADS) {
            float a3[3] = {0, 0, 0};
            const float *mr = M32 + i;
#pragma unroll 4
            for (int j = 0; j < C; j++) {
                const float a = mr[(size_t)j * R];
#pragma unroll
                for (int r = 0; r < 3; r++)
                    if (V.col_in(r, j)) a3[r] = fmaf(a, vst[r * C + j], a3[r]);
            }
#pragma unroll
            for (int r = 0; r < 3; r++) {
                if (!live[r] || !V.row_in(r, i)) continue;
                Ui(r, t)[i] = a3[r] - (t > 0 ? bpf[r] * Ui(r, t - 1)[i] : 0.f);
            }
        }
        // classical Gram-Schmidt against U[r][0..t)
        for (int pass = 0; pass < 1 && t > 0; pass++) {
#pragma unroll
            for (int q = 0; q < NS; q++) acc[q] = 0.f;
            for (int i = r0 + tid; i < r1; i += FT_THREADS)
#pragma unroll
                for (int r = 0; r < 3; r++) {
                    if (!live[r] || !V.row_in(r, i)) continue;
                    const float x = Ui(r, t)[i];
#pragma unroll
                    for (int j = 0; j < FT_KMAX; j++)
                        if (j < t) acc[r * FT_KMAX + j] = fmaf(x, Ui(r, j)[i], acc[r * FT_KMAX + j]);
                }
            csum(acc, NS);
            for (int i = r0 + tid; i < r1; i += FT_THREADS)
                for (int r = 0; r < 3; r++) {
                    if (!live[r] || !V.row_in(r, i)) continue;
                    float x = Ui(r, t)[i];
                    for (int j = 0; j < t; j++) x = fmaf(-tot[r * FT_KMAX + j], Ui(r, j)[i], x);
                    Ui(r, t)[i] = x;
                }
        }
        {
            float nu[3] = {0, 0, 0};
            for (int i = r0 + tid; i < r1; i += FT_THREADS)
                for (int r = 0; r < 3; r++)
                    if (live[r] && V.row_in(r, i)) nu[r] = fmaf(Ui(r, t)[i], Ui(r, t)[i], nu[r]);
            csum(nu, 3);
        }
        float al[3];
        for (int r = 0; r < 3; r++) {
            al[r] = sqrtf(tot[r]);
            // breakdown: alpha negligible against the largest alpha / beta so far
            if (live[r] && !(al[r] > GKL_BREAKDOWN_F * (t == 0 ? al[r] : big[r]))) live[r] = false;
            if (live[r]) big[r] = fmaxf(big[r], al[r]);
            if (live[r] && tid == 0) { alpha[r][t] = al[r]; kk[r] = t + 1; }
        }
        {
            float inv[3];
            for (int r = 0; r < 3; r++) inv[r] = live[r] ? 1.f / al[r] : 0.f;
            for (int i = r0 + tid; i < r1; i += FT_THREADS)
                for (int r = 0; r < 3; r++)
                    if (live[r] && V.row_in(r, i)) Ui(r, t)[i] *= inv[r];
        }
        __syncthreads();
        if (t == k - 1) break;
        float alf[3];
        for (int r = 0; r < 3; r++) alf[r] = al[r];
        // partial M_r^T u_t over this CTA's rows (warp per column)
        for (int j = warp; j < C; j += NW) {
            float p3[3] = {0, 0, 0};
            const float *mc = M32 + (size_t)j * R;
#pragma unroll 4
            for (int i = r0 + lane; i < r1; i += 32) {
                const float a = mc[i];
#pragma unroll
                for (int r = 0; r < 3; r++)
                    if (live[r] && V.row_in(r, i) && V.col_in(r, j)) p3[r] = fmaf(a, Ui(r, t)[i], p3[r]);
            }
#pragma unroll
            for (int r = 0; r < 3; r++) p3[r] = warp_sum(p3[r]);
            if (lane == 0)
                for (int r = 0; r < 3; r++) part[((size_t)rank * 3 + r) * C + j] = p3[r];
        }
        csync();
        // w = sum of partials - alpha v_t on the column slice, into V[r][t+1]
        for (int j = c0 + tid; j < c1; j += FT_THREADS)
            for (int r = 0; r < 3; r++) {
                if (!live[r]) continue;
                float w = 0.f;
                if (V.col_in(r, j)) {
                    for (int q = 0; q < CS; q++) w += __ldcg(part + ((size_t)q * 3 + r) * C + j);
                    w -= alf[r] * Vj(r, t)[j];
                }
                Vj(r, t + 1)[j] = w;
            }
        // classical Gram-Schmidt against V[r][0..t]
        for (int pass = 0; pass < 1; pass++) {
#pragma unroll
            for (int q = 0; q < NS; q++) acc[q] = 0.f;
            for (int j = c0 + tid; j < c1; j += FT_THREADS)
#pragma unroll
                for (int r = 0; r < 3; r++) {
                    if (!live[r]) continue;
                    const float x = Vj(r, t + 1)[j];
#pragma unroll
                    for (int q = 0; q < FT_KMAX; q++)
                        if (q <= t) acc[r * FT_KMAX + q] = fmaf(x, Vj(r, q)[j], acc[r * FT_KMAX + q]);
                }
            csum(acc, NS);
            for (int j = c0 + tid; j < c1; j += FT_THREADS)
                for (int r = 0; r < 3; r++) {
                    if (!live[r]) continue;
                    float x = Vj(r, t + 1)[j];
                    for (int q = 0; q <= t; q++) x = fmaf(-tot[r * FT_KMAX + q], Vj(r, q)[j], x);
                    Vj(r, t + 1)[j] = x;
                }
        }
        {
            float nw[3] = {0, 0, 0};
            for (int j = c0 + tid; j < c1; j += FT_THREADS)
                for (int r = 0; r < 3; r++)
                    if (live[r]) nw[r] = fmaf(Vj(r, t + 1)[j], Vj(r, t + 1)[j], nw[r]);
            csum(nw, 3);
        }
        for (int r = 0; r < 3; r++) {
            const float b = sqrtf(tot[r]);
            if (live[r] && !(b > GKL_BREAKDOWN_F * big[r])) live[r] = false;
            if (live[r]) big[r] = fmaxf(big[r], b);
            if (live[r] && tid == 0) beta[r][t] = b;
            bprev[r] = b;
        }
        {
            float inv[3];
            for (int r = 0; r < 3; r++) inv[r] = live[r] ? 1.f / bprev[r] : 0.f;
            for (int j = c0 + tid; j < c1; j += FT_THREADS)
                for (int r = 0; r < 3; r++)
                    if (live[r]) Vj(r, t + 1)[j] *= inv[r];
        }
        csync();
    }
    __shared__ double kap_s[3];
    bidiag_cond_block(alpha, beta, kk, kap_s);
    if (rank == 0 && tid == 0) {
        double kap[3];
        for (int r = 0; r < 3; r++) kap[r] = kap_s[r];
        if (V.kind == 1 && V.m == 0) kap[0] = 1.0;
        if (V.kind == 0 && V.p == 0) kap[1] = 1.0;
        double nb2 = 0.0, nd2 = 0.0;
        for (int i = 0; i < nbv; i++) nb2 = fma(bv[i], bv[i], nb2);
        for (int i = 0; i < ndv; i++) nd2 = fma(dv[i], dv[i], nd2);
        feature_vector(V, fA, fB, nb2, nd2, kap, out);
    }
    csync();
}

// The same sketch with the stacked matrix resident in shared memory: CTA
// `rank` of the cluster holds rows [r0, r1) in FP32 (row stride C | 1) and
// the u vectors of those rows; every CTA keeps the full v vectors (shared
// memory, or a private global region when they do not fit) and repeats the
// v-side work (M^T u partials summed over the cluster in rank order, so all
// CTAs hold bitwise the same v).  Three cluster barriers per step: the u
// reorthogonalization sums, the u norms and the M^T u exchange.  Vectors of
// a run are kept zero outside its rows / columns.
__global__ void __launch_bounds__(FT_THREADS, 1)
k_features_sm(FeatView V, const double *__restrict__ s, const double *__restrict__ bv, int nbv,
              const double *__restrict__ dv, int ndv, float *__restrict__ gvh, int vh_smem, int k,
              float *__restrict__ out)
{
    extern __shared__ float fsm[];
    cg::cluster_group cl = cg::this_cluster();
    const int CS = (int)cl.num_blocks(), rank = (int)cl.block_rank();
    auto csync = [&]() { if (CS == 1) __syncthreads(); else cl.sync(); };
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    constexpr int NW = FT_THREADS / 32;
    constexpr int NS = 3 * FT_KMAX;
    const int R = V.R, C = V.C, ldc = C | 1;
    const int rp = ceil_div(R, CS);
    const int r0 = min(R, rank * rp), r1 = min(R, r0 + rp), nr = r1 - r0;
    float *Ms = fsm;                                        // nr x C, row stride ldc
    float *Uh = Ms + (size_t)rp * ldc;                      // U[r][j][il] at Uh[(r * KMAX + j) * rp + il]
    float *Pp = Uh + (size_t)3 * FT_KMAX * rp;              // [2][3][C] partial M^T u (ping-pong)
    float *vcur = Pp + (size_t)6 * C;                       // [3][C] staged v_t (global Vh only)
    float *Vh = vh_smem ? vcur : gvh + (size_t)rank * 3 * (FT_KMAX + 1) * C;
    auto U_ = [&](int r, int j) { return Uh + ((size_t)r * FT_KMAX + j) * rp; };
    auto V_ = [&](int r, int j) { return Vh + ((size_t)r * (FT_KMAX + 1) + j) * C; };
    __shared__ float red[NW][NS];
    __shared__ float cred[2][NS];
    __shared__ float tot[NS];
    __shared__ double redd[NW][2], credd[2];
    __shared__ double alpha[3][FT_KMAX], beta[3][FT_KMAX];
    __shared__ int kk[3];
    int cb = 0, pb = 0;

    // sums of per-thread values v[0..ns) over the block (and over the
    // cluster when `across`); the totals land in tot[] on every CTA
    auto reduce = [&](const float *v, int ns, bool across) {
        for (int q0 = 0; q0 < ns; q0 += 32) {
            float w32[32];
#pragma unroll
            for (int q = 0; q < 32; q++) w32[q] = q0 + q < ns ? v[q0 + q] : 0.f;
            const float t = warp_transpose_reduce<float, 32>(w32);
            if (q0 + lane < ns) red[warp][q0 + lane] = t;
        }
        __syncthreads();
        const bool cl_red = across && CS > 1;
        if (tid < ns) {
            float t = 0.f;
            for (int w = 0; w < NW; w++) t += red[w][tid];
            if (cl_red) cred[cb][tid] = t; else tot[tid] = t;
        }
        if (cl_red) {
            cl.sync();
            if (tid < ns) {
                float t = 0.f;
                for (int q = 0; q < CS; q++) t += cl.map_shared_rank(&cred[cb][0], q)[tid];
                tot[tid] = t;
            }
            cb ^= 1;
        }
        __syncthreads();
    };

    // ---- this CTA's rows into shared memory (FP32), FP64 Frobenius norms
    for (int e = tid; e < 3 * FT_KMAX * rp; e += FT_THREADS) Uh[e] = 0.f;
    {
        double v2[2] = {0.0, 0.0};
        for (int j = warp; j < C; j += NW)
            for (int il = lane; il < nr; il += 32) {
                const int i = r0 + il;
                const double a = V.at(i, j);
                const bool first = V.kind == 0 ? i < V.m : j < V.m;
                if (first) v2[0] = fma(a, a, v2[0]); else v2[1] = fma(a, a, v2[1]);
                Ms[(size_t)il * ldc + j] = (float)a;
            }
        v2[0] = warp_sum(v2[0]);
        v2[1] = warp_sum(v2[1]);
        if (lane == 0) { redd[warp][0] = v2[0]; redd[warp][1] = v2[1]; }
        __syncthreads();
        if (tid < 2) {
            double t = 0.0;
            for (int w = 0; w < NW; w++) t += redd[w][tid];
            credd[tid] = t;
        }
        csync();
        if (tid < 2) {
            double t = 0.0;
            for (int q = 0; q < CS; q++) t += cl.map_shared_rank(&credd[0], q)[tid];
            redd[0][tid] = t;
        }
        __syncthreads();
    }
    const double fA = sqrt(redd[0][0]), fB = sqrt(redd[0][1]);
    // ---- start vectors: v_r = s on run r's columns, normalized (every CTA)
    {
        float s2[3] = {0, 0, 0};
        for (int j = tid; j < C; j += FT_THREADS)
            for (int r = 0; r < 3; r++) if (V.col_in(r, j)) s2[r] = fmaf((float)s[j], (float)s[j], s2[r]);
        reduce(s2, 3, false);
        float nrm[3];
        for (int r = 0; r < 3; r++) nrm[r] = sqrtf(tot[r]);
        for (int j = tid; j < C; j += FT_THREADS)
            for (int r = 0; r < 3; r++) V_(r, 0)[j] = (V.col_in(r, j) && nrm[r] > 0) ? (float)s[j] / nrm[r] : 0.f;
        if (tid < 3) kk[tid] = 0;
    }
    bool live[3];
    for (int r = 0; r < 3; r++) live[r] = (r == 1 && V.p == 0) ? false : true;
    if (V.kind == 1 && V.m == 0) live[0] = false;
    int rr[3], cc[3], klim[3];
    if (V.kind == 0) {
        rr[0] = V.m; rr[1] = V.p; rr[2] = V.m + V.p;
        cc[0] = cc[1] = cc[2] = V.n;
    } else {
        rr[0] = rr[1] = rr[2] = V.n;
        cc[0] = V.m; cc[1] = V.p; cc[2] = V.m + V.p;
    }
    bool wide[3], any_wide = false;
    for (int r = 0; r < 3; r++) {
        klim[r] = min(k, min(rr[r], cc[r]));
        wide[r] = live[r] && rr[r] < cc[r];
        any_wide |= wide[r];
    }
    __syncthreads();

    // v_t of the three runs, read by the products with M
    auto vsrc = [&](int t) -> const float * {
        if (vh_smem) return nullptr;
        for (int e = tid; e < 3 * C; e += FT_THREADS) vcur[e] = V_(e / C, t)[e % C];
        __syncthreads();
        return vcur;
    };
    // dst_r[il] = (M_r v_r)[r0 + il] - c_r prev_r[il] on run r's rows (0 elsewhere)
    auto mv = [&](int t, int j_u, const bool *use, const float *c, int j_prev) {
        const float *vs = vsrc(t);
        const float *v0 = vs ? vs : V_(0, t), *v1 = vs ? vs + C : V_(1, t), *v2 = vs ? vs + 2 * C : V_(2, t);
        for (int il = warp; il < nr; il += NW) {
            const float *mr = Ms + (size_t)il * ldc;
            float a0 = 0.f, a1 = 0.f, a2 = 0.f;
#pragma unroll 4
            for (int j = lane; j < C; j += 32) {
                const float a = mr[j];
                a0 = fmaf(a, v0[j], a0);
                a1 = fmaf(a, v1[j], a1);
                a2 = fmaf(a, v2[j], a2);
            }
            a0 = warp_sum(a0);
            a1 = warp_sum(a1);
            a2 = warp_sum(a2);
            if (lane < 3) {
                const int r = lane;
                const float a = r == 0 ? a0 : r == 1 ? a1 : a2;
                if (use[r]) {
                    float x = 0.f;
                    if (V.row_in(r, r0 + il)) x = a - (j_prev >= 0 ? c[r] * U_(r, j_prev)[il] : 0.f);
                    U_(r, j_u)[il] = x;
                }
            }
        }
        __syncthreads();
    };
    // w_r = (M_r^T u_r) on run r's columns, summed over the cluster, minus
    // c_r v_r(t); written to V_(r, t_out) for the runs in use
    auto mtv = [&](int j_u, const bool *use, const float *c, int t_v, int t_out) {
        float *P = Pp + (size_t)pb * 3 * C;
        for (int j = tid; j < C; j += FT_THREADS) {
            float p0 = 0.f, p1 = 0.f, p2 = 0.f;
            const float *u0 = U_(0, j_u), *u1 = U_(1, j_u), *u2 = U_(2, j_u);
#pragma unroll 4
            for (int il = 0; il < nr; il++) {
                const float a = Ms[(size_t)il * ldc + j];
                p0 = fmaf(a, u0[il], p0);
                p1 = fmaf(a, u1[il], p1);
                p2 = fmaf(a, u2[il], p2);
            }
            P[j] = p0;
            P[C + j] = p1;
            P[2 * C + j] = p2;
        }
        csync();
        for (int j = tid; j < C; j += FT_THREADS)
            for (int r = 0; r < 3; r++) {
                if (!use[r]) continue;
                float w = 0.f;
                if (V.col_in(r, j)) {
                    for (int q = 0; q < CS; q++) w += cl.map_shared_rank(P, q)[(size_t)r * C + j];
                    if (t_v >= 0) w -= c[r] * V_(r, t_v)[j];
                }
                V_(r, t_out)[j] = w;
            }
        pb ^= 1;
    };

    // wide blocks: start from M^T M s (normalized), inside range(M^T)
    if (any_wide) {
        const float zero3[3] = {0.f, 0.f, 0.f};
        mv(0, 0, wide, zero3, -1);
        mtv(0, wide, zero3, -1, 0);
        float n3[3] = {0, 0, 0};
        for (int j = tid; j < C; j += FT_THREADS)
            for (int r = 0; r < 3; r++) if (wide[r]) n3[r] = fmaf(V_(r, 0)[j], V_(r, 0)[j], n3[r]);
        reduce(n3, 3, false);
        float sc[3];
        for (int r = 0; r < 3; r++) sc[r] = tot[r] > 0 ? rsqrtf(tot[r]) : 0.f;
        for (int j = tid; j < C; j += FT_THREADS)
            for (int r = 0; r < 3; r++) if (wide[r]) V_(r, 0)[j] *= sc[r];
        for (int e = tid; e < 3 * FT_KMAX * rp; e += FT_THREADS) Uh[e] = 0.f;
        __syncthreads();
    }

    float bprev[3] = {0, 0, 0}, big[3] = {0, 0, 0};
    float acc[NS];
    for (int t = 0; t < k; t++) {
        for (int r = 0; r < 3; r++) if (t >= klim[r]) live[r] = false;
        // u'_r = M_r v_t - beta u_{t-1}
        mv(t, t, live, bprev, t > 0 ? t - 1 : -1);
        // classical Gram-Schmidt against U[r][0..t) (sums over the cluster)
        if (t > 0) {
#pragma unroll
            for (int q = 0; q < NS; q++) acc[q] = 0.f;
            for (int il = tid; il < nr; il += FT_THREADS)
#pragma unroll
                for (int r = 0; r < 3; r++) {
                    if (!live[r]) continue;
                    const float x = U_(r, t)[il];
#pragma unroll
                    for (int j = 0; j < FT_KMAX; j++)
                        if (j < t) acc[r * FT_KMAX + j] = fmaf(x, U_(r, j)[il], acc[r * FT_KMAX + j]);
                }
            reduce(acc, NS, true);
            for (int il = tid; il < nr; il += FT_THREADS)
                for (int r = 0; r < 3; r++) {
                    if (!live[r]) continue;
                    float x = U_(r, t)[il];
                    for (int j = 0; j < t; j++) x = fmaf(-tot[r * FT_KMAX + j], U_(r, j)[il], x);
                    U_(r, t)[il] = x;
                }
        }
        {
            float nu[3] = {0, 0, 0};
            for (int il = tid; il < nr; il += FT_THREADS)
                for (int r = 0; r < 3; r++)
                    if (live[r]) nu[r] = fmaf(U_(r, t)[il], U_(r, t)[il], nu[r]);
            reduce(nu, 3, true);
        }
        float al[3];
        for (int r = 0; r < 3; r++) {
            al[r] = sqrtf(tot[r]);
            if (live[r] && !(al[r] > GKL_BREAKDOWN_F * (t == 0 ? al[r] : big[r]))) live[r] = false;
            if (live[r]) big[r] = fmaxf(big[r], al[r]);
            if (live[r] && tid == 0) { alpha[r][t] = al[r]; kk[r] = t + 1; }
        }
        {
            float inv[3];
            for (int r = 0; r < 3; r++) inv[r] = live[r] ? 1.f / al[r] : 0.f;
            for (int il = tid; il < nr; il += FT_THREADS)
                for (int r = 0; r < 3; r++)
                    if (live[r]) U_(r, t)[il] *= inv[r];
        }
        __syncthreads();
        if (t == k - 1) break;
        // w = M_r^T u_t - alpha v_t into V[r][t+1]
        mtv(t, live, al, t, t + 1);
        // classical Gram-Schmidt against V[r][0..t] (every CTA, same columns per thread)
#pragma unroll
        for (int q = 0; q < NS; q++) acc[q] = 0.f;
        for (int j = tid; j < C; j += FT_THREADS)
#pragma unroll
            for (int r = 0; r < 3; r++) {
                if (!live[r]) continue;
                const float x = V_(r, t + 1)[j];
#pragma unroll
                for (int q = 0; q < FT_KMAX; q++)
                    if (q <= t) acc[r * FT_KMAX + q] = fmaf(x, V_(r, q)[j], acc[r * FT_KMAX + q]);
            }
        reduce(acc, NS, false);
        for (int j = tid; j < C; j += FT_THREADS)
            for (int r = 0; r < 3; r++) {
                if (!live[r]) continue;
                float x = V_(r, t + 1)[j];
                for (int q = 0; q <= t; q++) x = fmaf(-tot[r * FT_KMAX + q], V_(r, q)[j], x);
                V_(r, t + 1)[j] = x;
            }
        {
            float nw[3] = {0, 0, 0};
            for (int j = tid; j < C; j += FT_THREADS)
                for (int r = 0; r < 3; r++)
                    if (live[r]) nw[r] = fmaf(V_(r, t + 1)[j], V_(r, t + 1)[j], nw[r]);
            reduce(nw, 3, false);
        }
        for (int r = 0; r < 3; r++) {
            const float b = sqrtf(tot[r]);
            if (live[r] && !(b > GKL_BREAKDOWN_F * big[r])) live[r] = false;
            if (live[r]) big[r] = fmaxf(big[r], b);
            if (live[r] && tid == 0) beta[r][t] = b;
            bprev[r] = b;
        }
        {
            float inv[3];
            for (int r = 0; r < 3; r++) inv[r] = live[r] ? 1.f / bprev[r] : 0.f;
            for (int j = tid; j < C; j += FT_THREADS)
                for (int r = 0; r < 3; r++)
                    if (live[r]) V_(r, t + 1)[j] *= inv[r];
        }
        __syncthreads();
    }
    // every CTA runs the (identical) bisection; rank 0 writes the features
    __shared__ double kap_s[3];
    bidiag_cond_block(alpha, beta, kk, kap_s);
    if (rank == 0) {
        double b2 = 0.0, d2 = 0.0;
        for (int i = tid; i < nbv; i += FT_THREADS) b2 = fma(bv[i], bv[i], b2);
        for (int i = tid; i < ndv; i += FT_THREADS) d2 = fma(dv[i], dv[i], d2);
        b2 = warp_sum(b2);
        d2 = warp_sum(d2);
        if (lane == 0) { redd[warp][0] = b2; redd[warp][1] = d2; }
        __syncthreads();
        if (tid == 0) {
            double nb2 = 0.0, nd2 = 0.0;
            for (int w = 0; w < NW; w++) { nb2 += redd[w][0]; nd2 += redd[w][1]; }
            double kap[3];
            for (int r = 0; r < 3; r++) kap[r] = kap_s[r];
            if (V.kind == 1 && V.m == 0) kap[0] = 1.0;
            if (V.kind == 0 && V.p == 0) kap[1] = 1.0;
            feature_vector(V, fA, fB, nb2, nd2, kap, out);
        }
    }
    csync();
}

size_t features_ws_doubles(int R, int C)
{   // FP32 words / 2: partials, U, V and the FP32 copy of the stacked matrix
    // (global-memory variant), or the per-CTA v histories of the
    // shared-memory variant, whichever is larger
    const size_t words = (size_t)16 * 3 * C + (size_t)3 * FT_KMAX * R + (size_t)3 * (FT_KMAX + 1) * C +
                         (size_t)R * C + 128;
    const size_t vh = (size_t)16 * 3 * (FT_KMAX + 1) * C + 128;
    return (std::max(words, vh) + 1) / 2;
}

// Launch shape of the shared-memory variant: cluster size (a power of two,
// about 16k matrix entries per CTA, at most 16) and whether the v histories
// fit in shared memory.  0: the stacked matrix does not fit in 16 CTAs.
static int fsm_shape(int R, int C, size_t limit, bool *vh_smem, size_t *smem)
{
    const double elems = (double)R * C;
    int cs = 1;
    while (cs < 16 && elems > 16384.0 * cs) cs *= 2;
    for (; cs <= 16; cs *= 2) {
        const size_t rp = (size_t)ceil_div(R, cs), ldc = (size_t)(C | 1);
        const size_t base = rp * ldc + (size_t)3 * FT_KMAX * rp + (size_t)6 * C;
        const size_t with_vh = (base + (size_t)3 * (FT_KMAX + 1) * C) * sizeof(float);
        const size_t without = (base + (size_t)3 * C) * sizeof(float);
        if (with_vh <= limit) { *vh_smem = true; *smem = with_vh; return cs; }
        if (without <= limit) { *vh_smem = false; *smem = without; return cs; }
    }
    return 0;
}

int features_launch(int kind, int m, int n, int p, const double *A, int lda, const double *B, int ldb,
                    const double *s, const double *bv, int nbv, const double *dv, int ndv, int k, double *ws,
                    float *out, cudaStream_t st)
{
    FeatView V;
    V.kind = kind;
    V.m = m; V.n = n; V.p = p;
    V.A = A; V.B = B; V.lda = lda; V.ldb = ldb;
    if (kind == 0) { V.R = m + p; V.C = n; } else { V.R = n; V.C = m + p; }
    if (k < 1 || k > FT_KMAX) return MPIR_UNSUP();
    // shared-memory variant while the stacked matrix fits in a cluster
    static PerDeviceOnce once_sm;
    static size_t sm_limit = 0;
    once_sm([&] {
        cudaFuncAttributes fa{};
        int optin = 0, dev = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
        if (cudaFuncGetAttributes(&fa, k_features_sm) == cudaSuccess && optin > (int)fa.sharedSizeBytes) {
            sm_limit = (size_t)optin - fa.sharedSizeBytes;
            cudaFuncSetAttribute(k_features_sm, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
            cudaFuncSetAttribute(k_features_sm, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm_limit);
        }
        cudaGetLastError();
    });
    bool vh_smem = false;
    size_t smem = 0;
    const int want = sm_limit ? fsm_shape(V.R, V.C, sm_limit, &vh_smem, &smem) : 0;
    if (want > 0 && cluster_size_for((const void *)k_features_sm, FT_THREADS, smem, want) == want) {
        cudaLaunchConfig_t cfg = {};
        cfg.gridDim = dim3(want, 1, 1);
        cfg.blockDim = dim3(FT_THREADS, 1, 1);
        cfg.dynamicSmemBytes = smem;
        cfg.stream = st;
        cudaLaunchAttribute at[1];
        at[0].id = cudaLaunchAttributeClusterDimension;
        at[0].val.clusterDim.x = want;
        at[0].val.clusterDim.y = 1;
        at[0].val.clusterDim.z = 1;
        cfg.attrs = at;
        cfg.numAttrs = 1;
        ProfScope ps(K_SELECTOR, st);
        cudaError_t e = cudaLaunchKernelEx(&cfg, k_features_sm, V, s, bv, nbv, dv, ndv, (float *)ws,
                                           vh_smem ? 1 : 0, k, out);
        return e == cudaSuccess ? 0 : MPIR_CUDA_ERROR;
    }
    // larger blocks: the matrix stays in global memory (L2)
    auto kern = k_features;
    static PerDeviceOnce once;
    once([&] {
        cudaFuncSetAttribute(kern, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
        cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, 160 * 1024);
    });
    smem = (size_t)3 * V.C * sizeof(float);
    if (smem > 160 * 1024) return MPIR_UNSUP();
    const double elems = (double)V.R * V.C;
    int wantg = std::max(1, std::min(16, (int)(elems / 262144.0) + 1));
    const int cs = cluster_size_for((const void *)kern, FT_THREADS, smem, wantg);
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(cs, 1, 1);
    cfg.blockDim = dim3(FT_THREADS, 1, 1);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = st;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeClusterDimension;
    at[0].val.clusterDim.x = cs;
    at[0].val.clusterDim.y = 1;
    at[0].val.clusterDim.z = 1;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    ProfScope ps(K_SELECTOR, st);
    cudaError_t e = cudaLaunchKernelEx(&cfg, kern, V, s, bv, nbv, dv, ndv, ws, k, out);
    return e == cudaSuccess ? 0 : MPIR_CUDA_ERROR;
}

// ================================================================= MLP ==
// Parameter layout (FP32): W1 [64][16], b1 [64], W2 [64][64], b2 [64],
// W3 [6][64], b3 [6]; row-major weights (W[o][i] multiplies input i into
// output o).
constexpr int OW1 = 0, OB1 = 1024, OW2 = 1088, OB2 = 5184, OW3 = 5248, OB3 = 5632;
constexpr int MLP_THREADS = 256;

__device__ __forceinline__ float bf16_rne(float x)
{   // nearest bfloat16, ties to even (finite inputs)
    unsigned u = __float_as_uint(x);
    u = (u + 0x7FFFu + ((u >> 16) & 1u)) & 0xFFFF0000u;
    return __uint_as_float(u);
}

// Warp per sample: forward with bfloat16 weights and FP32 accumulation; with
// labels also the output deltas of the mean cross-entropy and the hidden
// deltas, stored per sample for the gradient kernel.
// acts (per sample, 262 floats): x[16] h1[64] h2[64] d1[64] d2[64] d3[6]
constexpr int ACT = 16 + 64 + 64 + 64 + 64 + 6;

__global__ void __launch_bounds__(MLP_THREADS)
k_mlp_sample(const float *__restrict__ P, const float *__restrict__ X, int count, const int *__restrict__ y,
             float *__restrict__ prob, float *__restrict__ acts, float *__restrict__ loss)
{
    __shared__ float w[MLP_PARAMS];
    for (int e = threadIdx.x; e < MLP_PARAMS; e += MLP_THREADS) {
        const bool bias = (e >= OB1 && e < OW2) || (e >= OB2 && e < OW3) || e >= OB3;
        w[e] = bias ? P[e] : bf16_rne(P[e]);
    }
    __syncthreads();
    const int lane = threadIdx.x & 31;
    const int nw = gridDim.x * (MLP_THREADS / 32);
    for (int smp = blockIdx.x * (MLP_THREADS / 32) + (threadIdx.x >> 5); smp < count; smp += nw) {
        const float xl = lane < 16 ? X[(size_t)smp * 16 + lane] : 0.f;
        float z1[2], h1[2], z2[2], h2[2];
#pragma unroll
        for (int q = 0; q < 2; q++) {
            const int o = lane + 32 * q;
            float a = w[OB1 + o];
#pragma unroll
            for (int i = 0; i < 16; i++) a = fmaf(w[OW1 + o * 16 + i], __shfl_sync(0xffffffffu, xl, i), a);
            z1[q] = a;
            h1[q] = fmaxf(a, 0.f);
        }
#pragma unroll
        for (int q = 0; q < 2; q++) {
            const int o = lane + 32 * q;
            float a = w[OB2 + o];
#pragma unroll
            for (int i = 0; i < 64; i++) {
                const float hi = __shfl_sync(0xffffffffu, h1[i >> 5], i & 31);
                a = fmaf(w[OW2 + o * 64 + i], hi, a);
            }
            z2[q] = a;
            h2[q] = fmaxf(a, 0.f);
        }
        float z3[NCLASS];
#pragma unroll
        for (int c = 0; c < NCLASS; c++) {
            float a = fmaf(w[OW3 + c * 64 + lane], h2[0], w[OW3 + c * 64 + lane + 32] * h2[1]);
            z3[c] = warp_sum(a) + w[OB3 + c];
        }
        float mx = z3[0];
#pragma unroll
        for (int c = 1; c < NCLASS; c++) mx = fmaxf(mx, z3[c]);
        float pr[NCLASS], se = 0.f;
#pragma unroll
        for (int c = 0; c < NCLASS; c++) { pr[c] = expf(z3[c] - mx); se += pr[c]; }
#pragma unroll
        for (int c = 0; c < NCLASS; c++) pr[c] /= se;
        if (prob && lane < NCLASS) {
            float v = 0.f;
#pragma unroll
            for (int c = 0; c < NCLASS; c++) if (c == lane) v = pr[c];
            prob[(size_t)smp * NCLASS + lane] = v;
        }
        if (!y) continue;
        const int lab = y[smp];
        float d3[NCLASS];
#pragma unroll
        for (int c = 0; c < NCLASS; c++) d3[c] = (pr[c] - (c == lab ? 1.f : 0.f)) / (float)count;
        float d2[2], d1[2];
#pragma unroll
        for (int q = 0; q < 2; q++) {
            const int j = lane + 32 * q;
            float a = 0.f;
#pragma unroll
            for (int c = 0; c < NCLASS; c++) a = fmaf(w[OW3 + c * 64 + j], d3[c], a);
            d2[q] = z2[q] > 0.f ? a : 0.f;
        }
#pragma unroll
        for (int q = 0; q < 2; q++) {
            const int i = lane + 32 * q;
            float a = 0.f;
#pragma unroll
            for (int j = 0; j < 64; j++) {
                const float dj = __shfl_sync(0xffffffffu, d2[j >> 5], j & 31);
                a = fmaf(w[OW2 + j * 64 + i], dj, a);
            }
            d1[q] = z1[q] > 0.f ? a : 0.f;
        }
        float *act = acts + (size_t)smp * ACT;
        if (lane < 16) act[lane] = xl;
#pragma unroll
        for (int q = 0; q < 2; q++) {
            act[16 + lane + 32 * q] = h1[q];
            act[80 + lane + 32 * q] = h2[q];
            act[144 + lane + 32 * q] = d1[q];
            act[208 + lane + 32 * q] = d2[q];
        }
        if (lane < NCLASS) {
            float v = 0.f;
#pragma unroll
            for (int c = 0; c < NCLASS; c++) if (c == lane) v = d3[c];
            act[272 + lane] = v;
        }
        if (lane == 0 && loss) {
            float pl = 0.f;
#pragma unroll
            for (int c = 0; c < NCLASS; c++) if (c == lab) pl = pr[c];
            loss[smp] = -logf(fmaxf(pl, 1e-30f));
        }
    }
}

// Gradient of every parameter: a sum over the samples in their order.
__global__ void k_mlp_grad(const float *__restrict__ acts, int count, float *__restrict__ grad)
{
    const int e = blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= MLP_PARAMS) return;
    int dofs, aofs;       // delta offset, activation offset (-1: bias)
    if (e < OB1) { dofs = 144 + e / 16; aofs = e % 16; }
    else if (e < OW2) { dofs = 144 + (e - OB1); aofs = -1; }
    else if (e < OB2) { dofs = 208 + (e - OW2) / 64; aofs = 16 + (e - OW2) % 64; }
    else if (e < OW3) { dofs = 208 + (e - OB2); aofs = -1; }
    else if (e < OB3) { dofs = 272 + (e - OW3) / 64; aofs = 80 + (e - OW3) % 64; }
    else { dofs = 272 + (e - OB3); aofs = -1; }
    float g = 0.f;
    for (int s = 0; s < count; s++) {
        const float *a = acts + (size_t)s * ACT;
        g = fmaf(a[dofs], aofs >= 0 ? a[aofs] : 1.f, g);
    }
    grad[e] = g;
}

__global__ void k_mlp_adam(float *__restrict__ P, float *__restrict__ M, float *__restrict__ Vv,
                           const float *__restrict__ g, float lr, float c1, float c2)
{
    const int e = blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= MLP_PARAMS) return;
    const float b1 = 0.9f, b2 = 0.999f, eps = 1e-8f;
    const float m = b1 * M[e] + (1.f - b1) * g[e];
    const float v = b2 * Vv[e] + (1.f - b2) * g[e] * g[e];
    M[e] = m;
    Vv[e] = v;
    P[e] -= lr * (m / c1) / (sqrtf(v / c2) + eps);
}

__global__ void k_sum(const float *__restrict__ x, int n, float *__restrict__ out)
{
    __shared__ float red[32];
    float s = 0.f;
    for (int i = threadIdx.x; i < n; i += blockDim.x) s += x[i];
    s = warp_sum(s);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
    __syncthreads();
    if (threadIdx.x == 0) {
        float t = 0.f;
        for (int w = 0; w < (int)(blockDim.x >> 5); w++) t += red[w];
        out[0] = t / (float)n;
    }
}

size_t mlp_ws_floats(int count) { return (size_t)count * ACT + (size_t)count + MLP_PARAMS + 64; }

int mlp_forward(const float *P, const float *X, int count, float *prob, cudaStream_t s)
{
    if (count <= 0) return 0;
    const int grid = std::min(ceil_div(count, MLP_THREADS / 32), 1216);
    ProfScope ps(K_SELECTOR, s);
    k_mlp_sample<<<grid, MLP_THREADS, 0, s>>>(P, X, count, nullptr, prob, nullptr, nullptr);
    return cudaGetLastError() == cudaSuccess ? 0 : MPIR_CUDA_ERROR;
}

int mlp_train_step(float *P, float *M, float *Vv, int t, float lr, const float *X, const int *y, int count,
                   float *ws, float *grad_out, float *loss_out, cudaStream_t s)
{
    if (count <= 0 || t < 1) return MPIR_UNSUP();
    float *acts = ws, *lossv = acts + (size_t)count * ACT, *grad = lossv + count;
    if (grad_out) grad = grad_out;
    const int grid = std::min(ceil_div(count, MLP_THREADS / 32), 1216);
    {
        ProfScope ps(K_SELECTOR, s);
        k_mlp_sample<<<grid, MLP_THREADS, 0, s>>>(P, X, count, y, nullptr, acts, lossv);
    }
    {
        ProfScope ps(K_SELECTOR, s);
        k_mlp_grad<<<ceil_div(MLP_PARAMS, 128), 128, 0, s>>>(acts, count, grad);
    }
    if (loss_out) {
        ProfScope ps(K_SELECTOR, s);
        k_sum<<<1, 256, 0, s>>>(lossv, count, loss_out);
    }
    if (M && Vv && lr > 0.f) {
        const float c1 = 1.f - powf(0.9f, (float)t), c2 = 1.f - powf(0.999f, (float)t);
        ProfScope ps(K_SELECTOR, s);
        k_mlp_adam<<<ceil_div(MLP_PARAMS, 128), 128, 0, s>>>(P, M, Vv, grad, lr, c1, c2);
    }
    return cudaGetLastError() == cudaSuccess ? 0 : MPIR_CUDA_ERROR;
}

} // namespace mpir
