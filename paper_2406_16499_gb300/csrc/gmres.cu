// gmres.cu -- restarted GMRES in FP64 (Sec. 5; Sec. 6.1: GMRES runs in
// double precision) for the preconditioned correction systems of GMRES-IR.
//
// The engine is generic over the operator (a LinOp supplied by the solver:
// M_l F~ M_r with the block-diagonal split preconditioners).  Per inner
// step one thread-block cluster does the whole Arnoldi step:
//   * classical Gram-Schmidt applied twice (CGS2): h = V^T w, w -= V h,
//     repeated once, H(:, j) = h1 + h2 -- two cluster-wide reductions of
//     j+1 dot products each instead of the j+1 sequential ones of modified
//     Gram-Schmidt;
//   * ||w|| and the normalization of the new basis vector;
//   * the Givens rotations of the small least-squares problem (H, g) and the
//     residual estimate |g(j+1)|, which the host reads to decide the stop.
// Cluster partial sums are combined in rank order, so runs are bitwise
// reproducible.  At the end of a cycle one kernel solves the small upper
// triangular system H y = g and adds V y to the iterate.
#include <cooperative_groups.h>

#include "common.cuh"
#include "kernels.h"
#include "gmres.h"
#include "mpir.h"

namespace cg = cooperative_groups;

namespace mpir {

constexpr int AR_THREADS = 512;
constexpr int AR_WARPS = AR_THREADS / 32;

size_t gmres_ws_bytes(int N, int R)
{
    const size_t ldv = (size_t)rup32(N);
    size_t b = 0;
    auto add = [&](size_t count) { b = (b + 255) & ~(size_t)255; b += count * sizeof(double); };
    add(ldv * (R + 1));          // basis
    add((size_t)(R + 1) * R);    // H
    add(R); add(R); add(R + 1);  // cs, sn, g
    add(8);                      // residual estimate + norms
    add(4096);                   // norm partials
    add(ldv); add(ldv);          // r, tmp
    return (b + 255) & ~(size_t)255;
}

GmresWs gmres_layout(void *base, int N, int R)
{
    GmresWs w{};
    w.N = N;
    w.R = R;
    w.ldv = (size_t)rup32(N);
    uintptr_t p = (uintptr_t)base;
    auto take = [&](size_t count) {
        p = (p + 255) & ~(uintptr_t)255;
        double *q = reinterpret_cast<double *>(p);
        p += count * sizeof(double);
        return q;
    };
    w.Vb = take(w.ldv * (R + 1));
    w.H = take((size_t)(R + 1) * R);
    w.cs = take(R); w.sn = take(R); w.g = take(R + 1);
    w.est = take(8);
    w.part = take(4096);
    w.r = take(w.ldv); w.tmp = take(w.ldv);
    return w;
}

// ------------------------------------------------------------ Arnoldi --
// Cluster of CS CTAs; CTA `rank` owns rows [rank*slice, min(N, (rank+1)*slice))
// of every vector and keeps its slice of w in shared memory.
__global__ void __launch_bounds__(AR_THREADS, 1)
k_arnoldi_cgs2(double *__restrict__ Vb, size_t ldv, int N, int j, int R, double *__restrict__ H,
               double *__restrict__ cs, double *__restrict__ sn, double *__restrict__ g,
               double *__restrict__ est, int slice)
{
    extern __shared__ double wsl[];
    __shared__ double part[GMRES_MAX_RESTART + 2];
    __shared__ double hs[GMRES_MAX_RESTART + 1];
    __shared__ double hacc[GMRES_MAX_RESTART + 1];
    __shared__ double red[AR_WARPS];
    __shared__ double nrm_s;
    cg::cluster_group cl = cg::this_cluster();
    const int ncta = (int)cl.num_blocks(), rank = (int)cl.block_rank();
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int s0 = rank * slice;
    const int len = max(0, min(N, s0 + slice) - s0);
    double *w = Vb + (size_t)(j + 1) * ldv + s0;
    for (int i = tid; i < len; i += AR_THREADS) wsl[i] = w[i];
    if (tid <= j) hacc[tid] = 0.0;
    __syncthreads();
    for (int pass = 0; pass < 2; pass++) {
        // partial dots of the owned slice: warp k handles basis vector k
        for (int k = warp; k <= j; k += AR_WARPS) {
            const double *vk = Vb + (size_t)k * ldv + s0;
            double acc = 0.0;
            for (int i = lane; i < len; i += 32) acc = fma(vk[i], wsl[i], acc);
            acc = warp_sum(acc);
            if (lane == 0) part[k] = acc;
        }
        cl.sync();
        if (tid <= j) {
            double h = 0.0;
            for (int r = 0; r < ncta; r++) h += cl.map_shared_rank(part, r)[tid];
            hs[tid] = h;
            hacc[tid] += h;
        }
        cl.sync();   // remote reads of `part` done; hs visible to the CTA
        for (int i = tid; i < len; i += AR_THREADS) {
            double d = 0.0;
            for (int k = 0; k <= j; k++) d = fma(hs[k], Vb[(size_t)k * ldv + s0 + i], d);
            wsl[i] -= d;
        }
        __syncthreads();
    }
    // ||w||
    double sq = 0.0;
    for (int i = tid; i < len; i += AR_THREADS) sq = fma(wsl[i], wsl[i], sq);
    sq = warp_sum(sq);
    if (lane == 0) red[warp] = sq;
    __syncthreads();
    if (tid == 0) {
        double t = 0.0;
        for (int k = 0; k < AR_WARPS; k++) t += red[k];
        part[GMRES_MAX_RESTART + 1] = t;
    }
    cl.sync();
    if (tid == 0) {
        double t = 0.0;
        for (int r = 0; r < ncta; r++) t += cl.map_shared_rank(part, r)[GMRES_MAX_RESTART + 1];
        nrm_s = sqrt(t);
    }
    cl.sync();       // every remote read done before any CTA exits
    const double nrm = nrm_s;
    // a zero norm (breakdown) leaves w as it is; the residual estimate is 0
    // then and the cycle ends
    for (int i = tid; i < len; i += AR_THREADS) w[i] = nrm > 0.0 ? wsl[i] / nrm : wsl[i];
    if (rank == 0 && tid == 0) {
        double *hc = H + (size_t)j * (R + 1);
        for (int i = 0; i <= j; i++) hc[i] = hacc[i];
        hc[j + 1] = nrm;
        for (int i = 0; i < j; i++) {
            const double t = cs[i] * hc[i] + sn[i] * hc[i + 1];
            hc[i + 1] = -sn[i] * hc[i] + cs[i] * hc[i + 1];
            hc[i] = t;
        }
        const double den = hypot(hc[j], hc[j + 1]);
        cs[j] = den != 0.0 ? hc[j] / den : 1.0;
        sn[j] = den != 0.0 ? hc[j + 1] / den : 0.0;
        hc[j] = den;
        hc[j + 1] = 0.0;
        g[j + 1] = -sn[j] * g[j];
        g[j] = cs[j] * g[j];
        est[0] = fabs(g[j + 1]);
    }
}

static int arnoldi_step(GmresWs &w, int j, cudaStream_t s)
{
    auto kern = k_arnoldi_cgs2;
    static PerDeviceOnce once;
    once([&] {
        cudaFuncSetAttribute(kern, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
        cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, 160 * 1024);
    });
    int want = ceil_div(w.N, 1024);
    if (want > 16) want = 16;
    if (want < 1) want = 1;
    int ncta = cluster_size_for((const void *)kern, AR_THREADS, (size_t)ceil_div(w.N, want) * sizeof(double), want);
    const int slice = ceil_div(w.N, ncta);
    ncta = ceil_div(w.N, slice);
    const size_t smem = (size_t)slice * sizeof(double);
    if (smem > 160 * 1024) return MPIR_UNSUP();
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(ncta, 1, 1);
    cfg.blockDim = dim3(AR_THREADS, 1, 1);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = s;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeClusterDimension;
    at[0].val.clusterDim.x = ncta;
    at[0].val.clusterDim.y = 1;
    at[0].val.clusterDim.z = 1;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    ProfScope ps(K_GMRES, s);
    cudaError_t e = cudaLaunchKernelEx(&cfg, kern, w.Vb, w.ldv, w.N, j, w.R, w.H, w.cs, w.sn, w.g, w.est, slice);
    return e == cudaSuccess ? 0 : MPIR_CUDA_ERROR;
}

// ------------------------------------------------- cycle start / update --
// V0 = r / beta0, g = [beta0, 0, ...]
__global__ void k_gmres_start(const double *__restrict__ r, double *__restrict__ v0, int N, double beta0,
                              double *__restrict__ g, int R)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < N) v0[i] = r[i] / beta0;
    if (i <= R) g[i] = i == 0 ? beta0 : 0.0;
}

// x += V(:, 0:jend) y with H(0:jend, 0:jend) y = g(0:jend) (upper triangular
// after the rotations); every block solves the small system itself.
__global__ void __launch_bounds__(256)
k_gmres_update(const double *__restrict__ Vb, size_t ldv, int N, int jend, int R, const double *__restrict__ H,
               const double *__restrict__ g, double *__restrict__ x)
{
    __shared__ double y[GMRES_MAX_RESTART];
    if (threadIdx.x == 0) {
        for (int i = jend - 1; i >= 0; i--) {
            double t = g[i];
            for (int k = i + 1; k < jend; k++) t -= H[i + (size_t)k * (R + 1)] * y[k];
            y[i] = t / H[i + (size_t)i * (R + 1)];
        }
    }
    __syncthreads();
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < N; i += gridDim.x * blockDim.x) {
        double d = 0.0;
        for (int k = 0; k < jend; k++) d = fma(Vb[(size_t)k * ldv + i], y[k], d);
        x[i] += d;
    }
}

// out = a - b
__global__ void k_gmres_sub(const double *__restrict__ a, const double *__restrict__ b, double *__restrict__ out,
                            int N)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < N) out[i] = a[i] - b[i];
}

// out[i] = c0 * base[i] + c1 * sum_k P1[k * st1 + i] + c2 * sum_k P2[k * st2 + i]
__global__ void k_combine_parts(double *__restrict__ out, int n, double c0, const double *__restrict__ base,
                                double c1, const double *__restrict__ P1, int k1, int st1, double c2,
                                const double *__restrict__ P2, int k2, int st2)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    double v = base ? c0 * base[i] : 0.0;
    if (P1) {
        double t = 0.0;
        for (int k = 0; k < k1; k++) t += P1[(size_t)k * st1 + i];
        v = fma(c1, t, v);
    }
    if (P2) {
        double t = 0.0;
        for (int k = 0; k < k2; k++) t += P2[(size_t)k * st2 + i];
        v = fma(c2, t, v);
    }
    out[i] = v;
}

void combine_parts(double *out, int n, double c0, const double *base, double c1, const double *P1, int k1,
                   int st1, double c2, const double *P2, int k2, int st2, cudaStream_t s)
{
    if (n <= 0) return;
    ProfScope ps(K_ELEMWISE, s);
    k_combine_parts<<<ceil_div(n, 256), 256, 0, s>>>(out, n, c0, base, c1, P1, k1, st1, c2, P2, k2, st2);
}

// ||v||_2 of a device vector, read back through the pinned buffer.
static int dev_norm(const double *v, int N, GmresWs &w, double *hbuf, cudaStream_t s, double *out)
{
    absmax_sumsq(v, std::max(N, 1), N, 1, w.part, w.est + 2, s);
    cudaMemcpyAsync(hbuf, w.est + 2, 2 * sizeof(double), cudaMemcpyDeviceToHost, s);
    if (cudaStreamSynchronize(s) != cudaSuccess) return MPIR_CUDA_ERROR;
    *out = sqrt(hbuf[1]);
    return 0;
}

static int read_est(GmresWs &w, double *hbuf, cudaStream_t s, double *out)
{
    cudaMemcpyAsync(hbuf, w.est, sizeof(double), cudaMemcpyDeviceToHost, s);
    if (cudaStreamSynchronize(s) != cudaSuccess) return MPIR_CUDA_ERROR;
    *out = hbuf[0];
    return 0;
}

#define GRC(x) do { int _rc = (x); if (_rc) return _rc; } while (0)

int gmres_solve(LinOp &op, const double *rhs, double *x, GmresWs &w, double tol, int maxit, double *hbuf,
                cudaStream_t s, int *iters, double *rel_out)
{
    const int N = w.N, R = w.R;
    if (R < 1 || R > GMRES_MAX_RESTART) return MPIR_UNSUP();
    *iters = 0;
    *rel_out = 0.0;
    cudaMemsetAsync(x, 0, sizeof(double) * N, s);
    double nb = 0.0;
    GRC(dev_norm(rhs, N, w, hbuf, s, &nb));
    if (!(nb > 0.0)) return std::isfinite(nb) ? 0 : MPIR_NONFINITE;
    cudaMemcpyAsync(w.r, rhs, sizeof(double) * N, cudaMemcpyDeviceToDevice, s);
    int total = 0;
    double rel = 1.0;
    const int nbk = ceil_div(N, 256);
    while (total < maxit) {
        double beta0 = 0.0;
        GRC(dev_norm(w.r, N, w, hbuf, s, &beta0));
        if (!std::isfinite(beta0)) return MPIR_NONFINITE;
        if (beta0 <= tol * nb) break;
        {
            ProfScope ps(K_GMRES, s);
            k_gmres_start<<<ceil_div(std::max(N, R + 1), 256), 256, 0, s>>>(w.r, w.Vb, N, beta0, w.g, R);
        }
        int jend = 0;
        for (int j = 0; j < R; j++) {
            GRC(op.apply(w.Vb + (size_t)j * w.ldv, w.Vb + (size_t)(j + 1) * w.ldv));
            GRC(arnoldi_step(w, j, s));
            total++;
            jend = j + 1;
            double est = 0.0;
            GRC(read_est(w, hbuf, s, &est));
            if (!std::isfinite(est)) return MPIR_NONFINITE;
            if (est <= tol * nb || total >= maxit) break;
        }
        {
            ProfScope ps(K_GMRES, s);
            k_gmres_update<<<std::min(nbk, 152), 256, 0, s>>>(w.Vb, w.ldv, N, jend, R, w.H, w.g, x);
        }
        // true residual of the cycle's iterate
        GRC(op.apply(x, w.tmp));
        {
            ProfScope ps(K_ELEMWISE, s);
            k_gmres_sub<<<nbk, 256, 0, s>>>(rhs, w.tmp, w.r, N);
        }
        double nr = 0.0;
        GRC(dev_norm(w.r, N, w, hbuf, s, &nr));
        rel = nr / nb;
        if (!std::isfinite(rel)) return MPIR_NONFINITE;
        if (rel <= tol) break;
    }
    *iters = total;
    *rel_out = rel;
    return cudaGetLastError() == cudaSuccess ? 0 : MPIR_CUDA_ERROR;
}

} // namespace mpir
