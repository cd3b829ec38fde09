// vec.cu -- the vector side of the correction solve (Alg. 1 / Alg. 3):
// reflector-set applications to one vector (xORMQR on a vector), blocked
// triangular solves (xTRSV), matrix-vector products (xGEMV) and the
// elementwise conversions between the FP64 working vectors and the
// factor-precision vectors.
#include "common.cuh"
#include "kernels.h"
#include "mpir.h"

namespace mpir {

static int coop_grid(const void *kern, int threads, size_t smem, int want)
{
    int dev = 0, sms = 0, per = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, kern, threads, smem);
    int cap = sms * (per > 0 ? per : 1);
    return want < cap ? want : cap;
}

// ---------------------------------------------------------------------------
// x <- Z^T x (trans = 1: blocks in order, factor I - V Tw^T V^T) or
// x <- Z x  (trans = 0: blocks in reverse order, factor I - V Tw V^T).
// Cooperative grid; block g owns rows [g*slice, (g+1)*slice) of x, kept in
// shared memory.  Per reflector block: partial V^T x over the owned rows ->
// global partials -> grid barrier -> every block sums the partials in the
// same fixed order, applies Tw, updates its rows.  One barrier per block.
// ---------------------------------------------------------------------------
template <typename T, int NB>
__global__ void __launch_bounds__(256)
k_vec_apply(const T *__restrict__ V, int ldv, int M, int K, const T *__restrict__ Tw, int trans,
            T *__restrict__ x, int slice, T *__restrict__ part, GridBarrier gb)
{
    extern __shared__ unsigned char smem_raw[];
    T *xs = reinterpret_cast<T *>(smem_raw);
    __shared__ T red_s[8][32];
    __shared__ T w_s[NB];
    __shared__ T wp_s[NB];
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int G = gridDim.x;
    const int s0 = blockIdx.x * slice;
    const int s1 = min(s0 + slice, M);
    for (int i = s0 + tid; i < s1; i += 256) xs[i - s0] = x[i];
    __syncthreads();
    const int nblk = ceil_div(K, NB);
    for (int t = 0; t < nblk; t++) {
        const int b = trans ? t : nblk - 1 - t;
        const int j0 = b * NB;
        const int kb = min(NB, K - j0);
        const int par = t & 1;
        T acc[NB];
#pragma unroll
        for (int c = 0; c < NB; c++) acc[c] = T(0);
        for (int i = max(s0, j0) + tid; i < s1; i += 256) {
            const T xi = xs[i - s0];
#pragma unroll
            for (int c = 0; c < NB; c++) {
                const int j = j0 + c;
                T v = T(0);
                if (c < kb) v = i > j ? V[idx2(i, j, ldv)] : (i == j ? T(1) : T(0));
                acc[c] = fma(v, xi, acc[c]);
            }
        }
        T ws = warp_transpose_reduce<T, NB>(acc);
        if (lane < NB) red_s[warp][lane] = ws;
        __syncthreads();
        if (warp == 0 && lane < NB) {
            T tsum = T(0);
            for (int w = 0; w < 8; w++) tsum += red_s[w][lane];
            part[((size_t)par * G + blockIdx.x) * NB + lane] = tsum;
        }
        if (!grid_sync(gb, G)) return;
        // every block: w = sum over blocks (fixed order), then w' = X w
        {
            const int c = tid % NB, g0 = tid / NB, gs = 256 / NB;
            T tsum = T(0);
            for (int g = g0; g < G; g += gs) tsum += part[((size_t)par * G + g) * NB + c];
            // reuse red_s as a [gs][NB] scratch (gs * NB == 256 == 8 * 32)
            T *scr = &red_s[0][0];
            scr[g0 * NB + c] = tsum;
            __syncthreads();
            if (tid < NB) {
                T s = T(0);
                for (int g = 0; g < gs; g++) s += scr[g * NB + tid];
                w_s[tid] = s;
            }
            __syncthreads();
            if (tid < NB) {
                T s = T(0);
                for (int k = 0; k < kb; k++) {
                    // X(i,k) = Tw(k,i) when trans, Tw(i,k) otherwise
                    const T xk = trans ? Tw[(size_t)b * NB * NB + k + (size_t)tid * NB]
                                       : Tw[(size_t)b * NB * NB + tid + (size_t)k * NB];
                    s = fma(xk, w_s[k], s);
                }
                wp_s[tid] = tid < kb ? s : T(0);
            }
            __syncthreads();
        }
        for (int i = max(s0, j0) + tid; i < s1; i += 256) {
            T d = T(0);
#pragma unroll
            for (int c = 0; c < NB; c++) {
                const int j = j0 + c;
                T v = T(0);
                if (c < kb) v = i > j ? V[idx2(i, j, ldv)] : (i == j ? T(1) : T(0));
                d = fma(v, wp_s[c], d);
            }
            xs[i - s0] -= d;
        }
        __syncthreads();
    }
    for (int i = s0 + tid; i < s1; i += 256) x[i] = xs[i - s0];
}

template <typename T>
int apply_reflectors_vec(const T *V, int ldv, int M, int K, const T *Tw, int trans, T *x,
                         const DevScratch &sc, cudaStream_t s)
{
    constexpr int NB = panel_nb<T>();
    if (K <= 0 || M <= 0) return 0;
    auto kern = k_vec_apply<T, NB>;
    int want = ceil_div(M, 128);
    int slice = 0;
    size_t smem = 0;
    int G = 1;
    for (int it = 0; it < 3; it++) {
        G = want < 1 ? 1 : want;
        slice = ceil_div(M, G);
        smem = (size_t)slice * sizeof(T);
        int cap = coop_grid((const void *)kern, 256, smem, G);
        if (cap >= G) break;
        want = cap;
    }
    slice = ceil_div(M, G);
    smem = (size_t)slice * sizeof(T);
    if ((size_t)2 * G * NB * sizeof(T) > sc.part_bytes || smem > 200 * 1024) return MPIR_UNSUP();
    if (smem > 48 * 1024) cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    GridBarrier gb{sc.barrier, sc.err};
    T *part = reinterpret_cast<T *>(sc.part);
    void *args[] = {(void *)&V, (void *)&ldv, (void *)&M, (void *)&K, (void *)&Tw, (void *)&trans,
                    (void *)&x, (void *)&slice, (void *)&part, (void *)&gb};
    ProfScope ps(K_VEC_APPLY, s);
    cudaError_t e = cudaLaunchCooperativeKernel((const void *)kern, dim3(G), dim3(256), args, smem, s);
    return e == cudaSuccess ? 0 : MPIR_CUDA_ERROR;
}

// ---------------------------------------------------------------------------
// Cluster version of the reflector-set application, used whenever the
// blocks' compact-WY factors are available at width NBV (128 for the
// two-level FP32 factorization).  One thread-block cluster; CTA r owns rows
// [r*slice, (r+1)*slice) of x in shared memory.  Per block of NBV
// reflectors:
//   1. each warp forms partial dots v_c^T x over the CTA's rows for its
//      columns (coalesced column reads of V);
//   2. cluster barrier; every CTA sums the partials of all CTAs from
//      distributed shared memory in rank order (identical on every CTA);
//   3. w' = X w with X = Tw^T (trans) or Tw, Tw staged in shared memory;
//   4. x_i -= sum_c v_c(i) w'_c on the CTA's rows.
// One cluster barrier per NBV reflectors (partials double-buffered).
// ---------------------------------------------------------------------------
constexpr int VEC_CL_THREADS = 512;

template <typename TS, typename T, int NBV>
__global__ void __launch_bounds__(VEC_CL_THREADS, 1)
k_vec_apply_cl(const TS *__restrict__ V, int ldv, int M, int K, const TS *__restrict__ Tw, int trans,
               T *__restrict__ x, int slice)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    T *Ts = reinterpret_cast<T *>(smem_raw);          // NBV x NBV, X(i,k) at i + k*NBV
    T *xs = Ts + NBV * NBV;                           // slice
    __shared__ T pbuf[2][NBV];
    __shared__ T wv[NBV];
    __shared__ T wp[NBV];
    cg::cluster_group cluster = cg::this_cluster();
    const int cs = (int)cluster.num_blocks();
    const int crank = (int)cluster.block_rank();
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    constexpr int NWARP = VEC_CL_THREADS / 32;
    const int s0 = crank * slice;
    const int s1 = min(s0 + slice, M);
    for (int i = s0 + tid; i < s1; i += VEC_CL_THREADS) xs[i - s0] = x[i];
    __syncthreads();
    const int nblk = ceil_div(K, NBV);
    for (int t = 0; t < nblk; t++) {
        const int b = trans ? t : nblk - 1 - t;
        const int j0 = b * NBV;
        const int kb = min(NBV, K - j0);
        const int par = t & 1;
        // stage X (used after the barrier)
        const TS *Tb = Tw + (size_t)b * NBV * NBV;
        for (int e = tid; e < NBV * NBV; e += VEC_CL_THREADS) {
            const int i = e % NBV, k = e / NBV;
            const T tv = (T)Tb[i + (size_t)k * NBV];
            if (trans) Ts[k + i * NBV] = tv; else Ts[i + k * NBV] = tv;
        }
        // 1. partial dots (rows unrolled by 4 for memory-level parallelism)
        for (int c = warp; c < NBV; c += NWARP) {
            T acc = T(0);
            if (c < kb) {
                const int j = j0 + c;
                const TS *vc = V + (size_t)j * ldv;
                const int ib = max(s0, j);
                for (int i0 = ib; i0 < s1; i0 += 128) {
                    T vv[4], xx[4];
#pragma unroll
                    for (int u = 0; u < 4; u++) {
                        const int i = i0 + lane + 32 * u;
                        vv[u] = i < s1 ? (i == j ? T(1) : (T)vc[i]) : T(0);
                        xx[u] = i < s1 ? xs[i - s0] : T(0);
                    }
#pragma unroll
                    for (int u = 0; u < 4; u++) acc = fma(vv[u], xx[u], acc);
                }
            }
            acc = warp_sum(acc);
            if (lane == 0) pbuf[par][c] = acc;
        }
        cluster.sync();
        // 2. cluster-wide sums
        if (tid < NBV) {
            T wsum = T(0);
            for (int r = 0; r < cs; r++) wsum += *cluster.map_shared_rank(&pbuf[par][tid], r);
            wv[tid] = wsum;
        }
        __syncthreads();
        // 3. w' = X w
        if (tid < NBV) {
            T sacc = T(0);
            for (int k = 0; k < kb; k++) sacc = fma(Ts[tid + k * NBV], wv[k], sacc);
            wp[tid] = tid < kb ? sacc : T(0);
        }
        __syncthreads();
        // 4. update the owned rows (wp[c] = 0 for c >= kb; 16 loads in flight)
        for (int i = max(s0, j0) + tid; i < s1; i += VEC_CL_THREADS) {
            T d = T(0);
            const int cmax = min(kb, i - j0 + 1);
            for (int c0 = 0; c0 < cmax; c0 += 16) {
                T vv[16];
#pragma unroll
                for (int u = 0; u < 16; u++) {
                    const int c = c0 + u, j = j0 + c;
                    vv[u] = c < cmax ? (i == j ? T(1) : (T)V[(size_t)j * ldv + i]) : T(0);
                }
#pragma unroll
                for (int u = 0; u < 16; u++) d = fma(vv[u], wp[(c0 + u) & (NBV - 1)], d);
            }
            xs[i - s0] -= d;
        }
        __syncthreads();
    }
    for (int i = s0 + tid; i < s1; i += VEC_CL_THREADS) x[i] = xs[i - s0];
    cluster.sync();   // keep shared memory alive until every remote read is done
}

template <typename TS, typename T, int NBV>
static int launch_vec_apply_cl(const TS *V, int ldv, int M, int K, const TS *Tw, int trans, T *x, cudaStream_t s)
{
    auto kern = k_vec_apply_cl<TS, T, NBV>;
    int want = ceil_div(M, 256);
    if (want > 16) want = 16;
    const size_t tsz = (size_t)NBV * NBV * sizeof(T);
    static PerDeviceOnce once;
    once([&] {
        cudaFuncSetAttribute(kern, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
        cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)(tsz + 64 * 1024));
    });
    int cs = cluster_size_for((const void *)kern, VEC_CL_THREADS, tsz + (size_t)ceil_div(M, want) * sizeof(T), want);
    int slice = ceil_div(M, cs);
    size_t smem = tsz + (size_t)slice * sizeof(T);
    if (smem > tsz + 64 * 1024) return MPIR_UNSUP();
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(cs, 1, 1);
    cfg.blockDim = dim3(VEC_CL_THREADS, 1, 1);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = s;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeClusterDimension;
    at[0].val.clusterDim.x = cs;
    at[0].val.clusterDim.y = 1;
    at[0].val.clusterDim.z = 1;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    ProfScope ps(K_VEC_APPLY, s);
    cudaError_t e = cudaLaunchKernelEx(&cfg, kern, V, ldv, M, K, Tw, trans, x, slice);
    return e == cudaSuccess ? 0 : MPIR_CUDA_ERROR;
}

template <typename TS, typename T>
int apply_reflectors_vec_blk(const TS *V, int ldv, int M, int K, const TS *Tw, int nbv, int trans, T *x,
                             cudaStream_t s)
{
    if (K <= 0 || M <= 0) return 0;
    if (nbv == 128) return launch_vec_apply_cl<TS, T, 128>(V, ldv, M, K, Tw, trans, x, s);
    if (nbv == 32) return launch_vec_apply_cl<TS, T, 32>(V, ldv, M, K, Tw, trans, x, s);
    if (nbv == 16) return launch_vec_apply_cl<TS, T, 16>(V, ldv, M, K, Tw, trans, x, s);
    return MPIR_UNSUP();
}

// ---------------------------------------------------------------------------
// Inverses of the 32 x 32 diagonal blocks of an upper triangular N x N
// matrix (one warp per block, lane j solves column j by back substitution;
// a partial last block is padded with the identity).  Zero pivot -> bit 1 of
// *status.  Used by the cluster triangular solve below; the inverse of a
// leading principal part of a block is the leading part of its inverse, so
// solves of any leading n <= N reuse them.
// ---------------------------------------------------------------------------
template <typename TS, typename T>
__global__ void __launch_bounds__(32)
k_invert_diag32(const TS *__restrict__ U, int ldu, int N, T *__restrict__ Dinv, int *__restrict__ status)
{
    __shared__ T Us[32][33];
    __shared__ T Xs[32][33];
    const int lane = threadIdx.x, blk = blockIdx.x, r0 = blk * 32;
    for (int c = 0; c < 32; c++) {
        T v;
        if (r0 + lane < N && r0 + c < N) v = lane <= c ? (T)U[idx2(r0 + lane, r0 + c, ldu)] : T(0);
        else v = lane == c ? T(1) : T(0);
        Us[lane][c] = v;
    }
    __syncwarp();
    const int j = lane;
    for (int i = 31; i >= 0; i--) {
        T val = T(0);
        if (i <= j) {
            T sum = i == j ? T(1) : T(0);
            for (int k = i + 1; k <= j; k++) sum = fma(-Us[i][k], Xs[k][j], sum);
            const T d = Us[i][i];
            if (d == T(0)) atomicOr(status, 2);
            val = sum / d;
        }
        Xs[i][j] = val;
    }
    __syncwarp();
    for (int i = 0; i < 32; i++) Dinv[(size_t)blk * 1024 + i + 32 * j] = Xs[i][j];
}

template <typename TS, typename T>
void invert_diag32_mixed(const TS *U, int ldu, int N, T *Dinv, int *status, cudaStream_t s)
{
    if (N <= 0) return;
    ProfScope ps(K_TRSV, s);
    k_invert_diag32<TS, T><<<ceil_div(N, 32), 32, 0, s>>>(U, ldu, N, Dinv, status);
}

template <typename T>
void invert_diag32(const T *U, int ldu, int N, T *Dinv, int *status, cudaStream_t s)
{
    invert_diag32_mixed<T, T>(U, ldu, N, Dinv, status, s);
}

// ---------------------------------------------------------------------------
// Cluster triangular solve with an upper triangular U (n x n):
//   trans = 0: U x = b  (32-row blocks from the bottom)
//   trans = 1: U^T x = b (32-row blocks from the top)
// CTA r owns rows [r*slice, (r+1)*slice) of x (slice a multiple of 32, at
// most 1024 = two rows per thread).  Per diagonal block: every thread first
// issues the loads of the block column of U for its rows (independent of
// x); the owner forms x_blk = D b_blk with the pre-inverted diagonal block
// D (or by substitution when no inverses are given) and publishes it;
// cluster barrier; every CTA reads x_blk through distributed shared memory
// and updates its unsolved rows.  One cluster barrier per 32 rows.
// ---------------------------------------------------------------------------
template <typename TS, typename T>
__global__ void __launch_bounds__(VEC_CL_THREADS, 1)
k_trsv_cl(const TS *__restrict__ U, int ldu, int n, int trans, T *__restrict__ x, int slice,
          const T *__restrict__ Dinv, int *__restrict__ status)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    T *xs = reinterpret_cast<T *>(smem_raw);
    __shared__ T xb[2][32];
    __shared__ T xl[32];
    __shared__ T dg[32][33];
    cg::cluster_group cluster = cg::this_cluster();
    const int crank = (int)cluster.block_rank();
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int s0 = crank * slice;
    const int s1 = min(s0 + slice, n);
    for (int i = s0 + tid; i < s1; i += VEC_CL_THREADS) xs[i - s0] = x[i];
    __syncthreads();
    const int nblk = ceil_div(n, 32);
    for (int t = 0; t < nblk; t++) {
        const int blk = trans ? t : nblk - 1 - t;
        const int r0 = blk * 32;
        const int bs = min(32, n - r0);
        const int par = t & 1;
        const int owner = r0 / slice;
        // rows this thread updates after the barrier, and their U entries
        const int lo = trans ? max(s0, r0 + bs) : s0;
        const int hi = trans ? s1 : min(s1, r0);
        constexpr int TROWS = sizeof(T) == 4 ? 2 : 1;    // rows prefetched per thread
        const int ia = s0 + tid, ib = s0 + tid + VEC_CL_THREADS;
        const bool va = ia >= lo && ia < hi, vb = TROWS > 1 && ib >= lo && ib < hi;
        T ua[32], ub[TROWS > 1 ? 32 : 1];
#pragma unroll
        for (int c = 0; c < 32; c++)
            ua[c] = (va && c < bs) ? (T)(trans ? U[idx2(r0 + c, ia, ldu)] : U[idx2(ia, r0 + c, ldu)]) : T(0);
        if (TROWS > 1) {
#pragma unroll
            for (int c = 0; c < 32; c++)
                ub[c % (TROWS > 1 ? 32 : 1)] =
                    (vb && c < bs) ? (T)(trans ? U[idx2(r0 + c, ib, ldu)] : U[idx2(ib, r0 + c, ldu)]) : T(0);
        }
        if (crank == owner && warp == 0) {
            T rhs = lane < bs ? xs[r0 + lane - s0] : T(0);
            T xv = T(0);
            if (Dinv) {
                const T *D = Dinv + (size_t)blk * 1024;
                T drow[32];
#pragma unroll
                for (int k = 0; k < 32; k++) drow[k] = trans ? D[k + 32 * lane] : D[lane + 32 * k];
#pragma unroll
                for (int k = 0; k < 32; k++) xv = fma(drow[k], __shfl_sync(0xffffffffu, rhs, k), xv);
                if (lane >= bs) xv = T(0);
            } else {
#pragma unroll
                for (int c = 0; c < 32; c++)
                    dg[lane][c] = (c < bs && lane < bs) ? (T)U[idx2(r0 + lane, r0 + c, ldu)] : T(0);
                __syncwarp();
                if (!trans) {
                    for (int c = bs - 1; c >= 0; c--) {
                        const T dcc = dg[c][c];
                        T xc = __shfl_sync(0xffffffffu, rhs, c);
                        if (dcc == T(0) && lane == 0) atomicOr(status, 2);
                        xc = xc / dcc;
                        if (lane == c) xv = xc;
                        if (lane < c) rhs = fma(-dg[lane][c], xc, rhs);
                    }
                } else {
                    for (int c = 0; c < bs; c++) {
                        const T dcc = dg[c][c];
                        T xc = __shfl_sync(0xffffffffu, rhs, c);
                        if (dcc == T(0) && lane == 0) atomicOr(status, 2);
                        xc = xc / dcc;
                        if (lane == c) xv = xc;
                        if (lane > c && lane < bs) rhs = fma(-dg[c][lane], xc, rhs);
                    }
                }
            }
            if (lane < bs) xs[r0 + lane - s0] = xv;
            xb[par][lane] = lane < bs ? xv : T(0);
        }
        cluster.sync();
        if (tid < 32) xl[tid] = *cluster.map_shared_rank(&xb[par][tid], owner);
        __syncthreads();
        if (va) {
            T d = T(0);
#pragma unroll
            for (int c = 0; c < 32; c++) d = fma(ua[c], xl[c], d);
            xs[ia - s0] -= d;
        }
        if (TROWS > 1 && vb) {
            T d = T(0);
#pragma unroll
            for (int c = 0; c < 32; c++) d = fma(ub[c % (TROWS > 1 ? 32 : 1)], xl[c], d);
            xs[ib - s0] -= d;
        }
        __syncthreads();
    }
    for (int i = s0 + tid; i < s1; i += VEC_CL_THREADS) x[i] = xs[i - s0];
    cluster.sync();
}

// ---------------------------------------------------------------------------
// Blocked triangular solve with an upper triangular U (n x n):
//   trans = 0: U x = b  (blocks of 32 from the bottom)
//   trans = 1: U^T x = b (blocks of 32 from the top)
// Cooperative grid; block g owns a slice of rows of x (multiple of 32).
// Step per diagonal block: its owner solves the 32 x 32 triangle in one warp
// and publishes the 32 values; grid barrier; every block subtracts the
// block column's contribution from its own not-yet-solved rows.
// ---------------------------------------------------------------------------
template <typename TS, typename T>
__global__ void __launch_bounds__(256)
k_trsv_upper(const TS *__restrict__ U, int ldu, int n, int trans, T *__restrict__ x, int slice,
             T *__restrict__ xbuf, int *__restrict__ status, GridBarrier gb)
{
    extern __shared__ unsigned char smem_raw[];
    T *xs = reinterpret_cast<T *>(smem_raw);
    __shared__ T xb[32];
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int G = gridDim.x;
    const int s0 = blockIdx.x * slice;
    const int s1 = min(s0 + slice, n);
    for (int i = s0 + tid; i < s1; i += 256) xs[i - s0] = x[i];
    __syncthreads();
    const int nblk = ceil_div(n, 32);
    for (int t = 0; t < nblk; t++) {
        const int blk = trans ? t : nblk - 1 - t;
        const int r0 = blk * 32;
        const int bs = min(32, n - r0);
        const int par = t & 1;
        if (r0 >= s0 && r0 < s1 && warp == 0) {
            T rhs = lane < bs ? xs[r0 + lane - s0] : T(0);
            T xv = T(0);
            if (!trans) {
                for (int c = bs - 1; c >= 0; c--) {
                    const T dcc = (T)U[idx2(r0 + c, r0 + c, ldu)];
                    T xc = __shfl_sync(0xffffffffu, rhs, c);
                    if (dcc == T(0)) { if (lane == 0) atomicOr(status, 2); }
                    xc = xc / dcc;
                    if (lane == c) xv = xc;
                    if (lane < c) rhs = fma(-(T)U[idx2(r0 + lane, r0 + c, ldu)], xc, rhs);
                }
            } else {
                for (int c = 0; c < bs; c++) {
                    const T dcc = (T)U[idx2(r0 + c, r0 + c, ldu)];
                    T xc = __shfl_sync(0xffffffffu, rhs, c);
                    if (dcc == T(0)) { if (lane == 0) atomicOr(status, 2); }
                    xc = xc / dcc;
                    if (lane == c) xv = xc;
                    if (lane > c && lane < bs) rhs = fma(-(T)U[idx2(r0 + c, r0 + lane, ldu)], xc, rhs);
                }
            }
            if (lane < bs) {
                xs[r0 + lane - s0] = xv;
                xbuf[par * 32 + lane] = xv;
            }
        }
        if (!grid_sync(gb, G)) return;
        if (tid < 32) xb[tid] = tid < bs ? xbuf[par * 32 + tid] : T(0);
        __syncthreads();
        if (!trans) {
            // rows i < r0: x_i -= sum_c U(i, r0+c) xb_c
            const int hi = min(s1, r0);
            for (int i = s0 + tid; i < hi; i += 256) {
                T d = T(0);
                for (int c = 0; c < bs; c++) d = fma((T)U[idx2(i, r0 + c, ldu)], xb[c], d);
                xs[i - s0] -= d;
            }
        } else {
            // rows i >= r0 + bs: x_i -= sum_c U(r0+c, i) xb_c
            const int lo = max(s0, r0 + bs);
            for (int i = lo + tid; i < s1; i += 256) {
                const TS *ucol = U + idx2(r0, i, ldu);
                T d = T(0);
                for (int c = 0; c < bs; c++) d = fma((T)ucol[c], xb[c], d);
                xs[i - s0] -= d;
            }
        }
        __syncthreads();
    }
    for (int i = s0 + tid; i < s1; i += 256) x[i] = xs[i - s0];
}

template <typename TS, typename T>
static int trsv_upper_cl(const TS *U, int ldu, int n, int trans, T *x, const DevScratch &sc, cudaStream_t s,
                         const T *Dinv)
{
    auto kern = k_trsv_cl<TS, T>;
    const int nblk = ceil_div(n, 32);
    int want = ceil_div(nblk, 8);            // 256 rows per CTA
    if (want > 16) want = 16;
    static PerDeviceOnce once;
    once([&] {
        cudaFuncSetAttribute(kern, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
        cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, 128 * 1024);
    });
    int cs = cluster_size_for((const void *)kern, VEC_CL_THREADS, (size_t)ceil_div(nblk, want) * 32 * sizeof(T), want);
    const int slice = ceil_div(nblk, cs) * 32;
    cs = ceil_div(n, slice);
    const size_t smem = (size_t)slice * sizeof(T);
    if (slice > (sizeof(T) == 4 ? 2 : 1) * VEC_CL_THREADS) return -1;   // rows a thread can prefetch
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(cs, 1, 1);
    cfg.blockDim = dim3(VEC_CL_THREADS, 1, 1);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = s;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeClusterDimension;
    at[0].val.clusterDim.x = cs;
    at[0].val.clusterDim.y = 1;
    at[0].val.clusterDim.z = 1;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    ProfScope ps(K_TRSV, s);
    cudaError_t e = cudaLaunchKernelEx(&cfg, kern, U, ldu, n, trans, x, slice, Dinv, sc.status);
    return e == cudaSuccess ? 0 : MPIR_CUDA_ERROR;
}

template <typename TS, typename T>
static int trsv_dispatch(const TS *U, int ldu, int n, int trans, T *x, const DevScratch &sc, cudaStream_t s,
                         const T *Dinv)
{
    if (n <= 0) return 0;
    {
        const int rc = trsv_upper_cl<TS, T>(U, ldu, n, trans, x, sc, s, Dinv);
        if (rc >= 0) return rc;          // -1: too large for one cluster, use the grid version
    }
    auto kern = k_trsv_upper<TS, T>;
    const int nblk = ceil_div(n, 32);
    int want = ceil_div(nblk, 4);          // 128 rows per block
    int G = want;
    size_t smem = 0;
    int slice = 0;
    for (int it = 0; it < 3; it++) {
        G = want < 1 ? 1 : want;
        slice = ceil_div(nblk, G) * 32;
        smem = (size_t)slice * sizeof(T);
        int cap = coop_grid((const void *)kern, 256, smem, G);
        if (cap >= G) break;
        want = cap;
    }
    slice = ceil_div(nblk, G) * 32;
    G = ceil_div(n, slice);
    smem = (size_t)slice * sizeof(T);
    if (smem > 200 * 1024 || (size_t)64 * sizeof(T) > sc.part_bytes) return MPIR_UNSUP();
    if (smem > 48 * 1024) cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    GridBarrier gb{sc.barrier, sc.err};
    T *xbuf = reinterpret_cast<T *>(sc.part);
    int *status = sc.status;
    void *args[] = {(void *)&U, (void *)&ldu, (void *)&n, (void *)&trans, (void *)&x, (void *)&slice,
                    (void *)&xbuf, (void *)&status, (void *)&gb};
    ProfScope ps(K_TRSV, s);
    cudaError_t e = cudaLaunchCooperativeKernel((const void *)kern, dim3(G), dim3(256), args, smem, s);
    return e == cudaSuccess ? 0 : MPIR_CUDA_ERROR;
}

template <typename T>
int trsv_upper(const T *U, int ldu, int n, int trans, T *x, const DevScratch &sc, cudaStream_t s, const T *Dinv)
{
    return trsv_dispatch<T, T>(U, ldu, n, trans, x, sc, s, Dinv);
}

// Mixed-precision solve: U stored as TS, arithmetic and x in T (FP32 factors
// applied in FP64 by GMRES-IR).  Dinv (optional, type T): inverses of the
// diagonal blocks from invert_diag32_mixed; else substitution.
template <typename TS, typename T>
int trsv_upper_mixed(const TS *U, int ldu, int n, int trans, T *x, const DevScratch &sc, cudaStream_t s,
                     const T *Dinv)
{
    return trsv_dispatch<TS, T>(U, ldu, n, trans, x, sc, s, Dinv);
}

// ---------------------------------------------------------------------------
// gemv.  trans = 0: 32 rows per block (lanes), 8 warps split the columns.
//        trans = 1: one warp per output column.
// upper_mask: M(i, j) treated as 0 when i > j + diag_off.
// ---------------------------------------------------------------------------
template <typename TS, typename T>
__global__ void __launch_bounds__(256)
k_gemv_n(const TS *__restrict__ M, int ld, int rows, int cols, T alpha, const T *__restrict__ x,
         T beta, T *__restrict__ y, int upper_mask, int diag_off)
{
    pdl_wait();
    pdl_trigger();
    __shared__ T red[8][33];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int i = blockIdx.x * 32 + lane;
    T acc = T(0);
    if (i < rows) {
        int jlo = 0;
        if (upper_mask) jlo = max(0, i - diag_off);
        for (int j = warp; j < cols; j += 8)
            if (j >= jlo) acc = fma((T)M[idx2(i, j, ld)], x[j], acc);
    }
    red[warp][lane] = acc;
    __syncthreads();
    if (warp == 0 && i < rows) {
        T s = T(0);
        for (int w = 0; w < 8; w++) s += red[w][lane];
        y[i] = (beta == T(0) ? T(0) : beta * y[i]) + alpha * s;
    }
}

template <typename TS, typename T>
__global__ void __launch_bounds__(256)
k_gemv_t(const TS *__restrict__ M, int ld, int rows, int cols, T alpha, const T *__restrict__ x,
         T beta, T *__restrict__ y, int upper_mask, int diag_off)
{
    pdl_wait();
    pdl_trigger();
    const int lane = threadIdx.x & 31;
    const int j = blockIdx.x * 8 + (threadIdx.x >> 5);
    if (j >= cols) return;
    int ihi = rows;
    if (upper_mask) ihi = min(rows, j + diag_off + 1);
    const TS *col = M + idx2(0, j, ld);
    T acc = T(0);
    for (int i = lane; i < ihi; i += 32) acc = fma((T)col[i], x[i], acc);
    acc = warp_sum(acc);
    if (lane == 0) y[j] = (beta == T(0) ? T(0) : beta * y[j]) + alpha * acc;
}

template <typename TS, typename T>
int gemv_mixed(const TS *M, int ld, int rows, int cols, int trans, T alpha, const T *x, T beta, T *y,
               int upper_mask, int diag_off, cudaStream_t s)
{
    if ((!trans && rows <= 0) || (trans && cols <= 0)) return 0;
    ProfScope ps(K_GEMV, s);
    if (!trans) {
        pdl_launch(k_gemv_n<TS, T>, dim3(ceil_div(rows, 32)), dim3(256), 0, s, M, ld, rows, cols, alpha, x, beta, y, upper_mask,
                                                        diag_off);
    } else {
        pdl_launch(k_gemv_t<TS, T>, dim3(ceil_div(cols, 8)), dim3(256), 0, s, M, ld, rows, cols, alpha, x, beta, y, upper_mask,
                                                       diag_off);
    }
    return cudaGetLastError() == cudaSuccess ? 0 : MPIR_CUDA_ERROR;
}

template <typename T>
int gemv(const T *M, int ld, int rows, int cols, int trans, T alpha, const T *x, T beta, T *y,
         int upper_mask, int diag_off, cudaStream_t s)
{
    return gemv_mixed<T, T>(M, ld, rows, cols, trans, alpha, x, beta, y, upper_mask, diag_off, s);
}

// ------------------------------------------------------------ elementwise --

template <typename Ts, typename Td>
__global__ void k_vcopy(const Ts *__restrict__ src, Td *__restrict__ dst, int n, double scale, int rev,
                        const double *__restrict__ dscale)
{
    pdl_wait();
    pdl_trigger();
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    const double g = dscale ? scale * dscale[0] : scale;
    if (i < n) dst[i] = (Td)(g * (double)src[rev ? n - 1 - i : i]);
}

__global__ void __launch_bounds__(256)
k_pow2_normalizer(const double *__restrict__ u, int nu, double a1, const double *__restrict__ w, int nw,
                  double a2, double *__restrict__ out)
{
    pdl_wait();
    pdl_trigger();
    __shared__ double red[8];
    double mx = 0.0;
    for (int i = threadIdx.x; i < nu; i += 256) mx = fmax(mx, fabs(a1 * u[i]));
    for (int i = threadIdx.x; i < nw; i += 256) mx = fmax(mx, fabs(a2 * w[i]));
    for (int o = 16; o > 0; o >>= 1) mx = fmax(mx, __shfl_xor_sync(0xffffffffu, mx, o));
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = mx;
    __syncthreads();
    if (threadIdx.x == 0) {
        for (int k = 1; k < 8; k++) mx = fmax(mx, red[k]);
        double g = 1.0;
        if (mx > 0.0 && isfinite(mx)) g = ldexp(1.0, -(ilogb(mx) + 1));
        out[0] = g;
        out[1] = 1.0 / g;
    }
}

void pow2_normalizer(const double *u, int nu, double a1, const double *w, int nw, double a2, double *out,
                     cudaStream_t s)
{
    ProfScope ps(K_NORM, s);
    pdl_launch(k_pow2_normalizer, dim3(1), dim3(256), 0, s, u, nu, a1, w, nw, a2, out);
}

template <typename Ts>
__global__ void k_vaxpy(const Ts *__restrict__ src, double *__restrict__ dst, int n, double scale, int rev,
                        const double *__restrict__ dscale)
{
    pdl_wait();
    pdl_trigger();
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    const double sc = dscale ? scale * *dscale : scale;
    if (i < n) dst[i] += sc * (double)src[rev ? n - 1 - i : i];
}

template <typename Ts, typename Td>
void vcopy(const Ts *src, Td *dst, int n, double scale, int rev, cudaStream_t s, const double *dscale)
{
    if (n <= 0) return;
    ProfScope ps(K_ELEMWISE, s);
    pdl_launch(k_vcopy<Ts, Td>, dim3(ceil_div(n, 256)), dim3(256), 0, s, src, dst, n, scale, rev, dscale);
}

template <typename Ts>
void vaxpy(const Ts *src, double *dst, int n, double scale, int rev, cudaStream_t s, const double *dscale)
{
    if (n <= 0) return;
    ProfScope ps(K_ELEMWISE, s);
    pdl_launch(k_vaxpy<Ts>, dim3(ceil_div(n, 256)), dim3(256), 0, s, src, dst, n, scale, rev, dscale);
}

void vzero(void *dst, size_t bytes, cudaStream_t s)
{
    if (bytes) cudaMemsetAsync(dst, 0, bytes, s);
}

// Tiled conversion with optional transpose / reversal: 64 x 64 tiles through
// shared memory, so that a warp reads 32 consecutive source entries and
// writes 32 consecutive destination entries (each tile column a 256- or
// 512-byte run), and every thread has its 16 loads in flight before the
// tile barrier.
constexpr int MC_T = 64;
template <typename Ts, typename Td>
__global__ void __launch_bounds__(256)
k_mconvert(const Ts *__restrict__ src, int lds, Td *__restrict__ dst, int ldd, int rows_d, int cols_d,
           int transpose, int rev_r, int rev_c, double scale, const double *__restrict__ rs, int rs_rev)
{
    auto rsc = [&](int i) { return rs ? scale * rs[rs_rev ? rows_d - 1 - i : i] : scale; };
    __shared__ Ts tile[MC_T][MC_T + 1];
    const int bi = blockIdx.x * MC_T, bj = blockIdx.y * MC_T;
    const int tx = threadIdx.x & (MC_T - 1), ty = threadIdx.x / MC_T;   // 64 x 4
    // destination tile (bi.., bj..): source index for dst (i, j) is
    // (ri, ci) = transpose ? (j', i') : (i', j')
    if (!transpose) {
        const int i = bi + tx;
        const int ip = rev_r ? rows_d - 1 - i : i;
        Ts v[MC_T / 4];
#pragma unroll
        for (int k = 0; k < MC_T / 4; k++) {
            const int j = bj + ty + 4 * k;
            const int jp = rev_c ? cols_d - 1 - j : j;
            v[k] = (i < rows_d && j < cols_d) ? src[idx2(ip, jp, lds)] : Ts(0);
        }
        if (i < rows_d) {
            const double sc = rsc(i);
#pragma unroll
            for (int k = 0; k < MC_T / 4; k++) {
                const int j = bj + ty + 4 * k;
                if (j < cols_d) dst[idx2(i, j, ldd)] = (Td)(sc * (double)v[k]);
            }
        }
        return;
    }
    // transpose: read source rows (j') contiguous along j' for fixed i'
    {
        const int j = bj + tx;
        const int jp = rev_c ? cols_d - 1 - j : j;
        Ts v[MC_T / 4];
#pragma unroll
        for (int k = 0; k < MC_T / 4; k++) {
            const int i = bi + ty + 4 * k;          // load element needed by dst(i, j)
            const int ip = rev_r ? rows_d - 1 - i : i;
            v[k] = (i < rows_d && j < cols_d) ? src[idx2(jp, ip, lds)] : Ts(0);
        }
#pragma unroll
        for (int k = 0; k < MC_T / 4; k++) tile[ty + 4 * k][tx] = v[k];
    }
    __syncthreads();
    const int i = bi + tx;
    if (i < rows_d) {
        const double sc = rsc(i);
#pragma unroll
        for (int k = 0; k < MC_T / 4; k++) {
            const int j = bj + ty + 4 * k;
            if (j < cols_d) dst[idx2(i, j, ldd)] = (Td)(sc * (double)tile[tx][ty + 4 * k]);
        }
    }
}

template <typename Ts, typename Td>
void mconvert(const Ts *src, int lds, Td *dst, int ldd, int rows_d, int cols_d, int transpose, int rev_r,
              int rev_c, double scale, cudaStream_t s, const double *rs, int rs_rev)
{
    if (rows_d <= 0 || cols_d <= 0) return;
    dim3 grid(ceil_div(rows_d, MC_T), ceil_div(cols_d, MC_T));
    ProfScope ps(K_CONVERT, s);
    k_mconvert<Ts, Td><<<grid, 256, 0, s>>>(src, lds, dst, ldd, rows_d, cols_d, transpose, rev_r, rev_c,
                                           scale, rs, rs_rev);
}

template <typename T>
__global__ void __launch_bounds__(256) k_vdiag(T *__restrict__ v, const double *__restrict__ D, int n, int rev)
{
    const int i = blockIdx.x * 256 + threadIdx.x;
    if (i < n) v[i] = (T)((double)v[i] * D[rev ? n - 1 - i : i]);
}

template <typename T>
void vdiag(T *v, const double *D, int n, int rev, cudaStream_t s)
{
    if (n <= 0 || !D) return;
    ProfScope ps(K_ELEMWISE, s);
    k_vdiag<T><<<ceil_div(n, 256), 256, 0, s>>>(v, D, n, rev);
}

// One warp per column j: the column maxima of A and B, then D[j].
__global__ void __launch_bounds__(256)
k_colscale(const double *__restrict__ A, int lda, int rows_a, const double *__restrict__ B, int ldb, int rows_b,
           int n, double a1, double a2, double *__restrict__ D)
{
    const int j = blockIdx.x * 8 + (threadIdx.x >> 5), lane = threadIdx.x & 31;
    if (j >= n) return;
    double ma = 0.0, mb = 0.0;
    for (int i = lane; i < rows_a; i += 32) ma = fmax(ma, fabs(A[idx2(i, j, lda)]));
    for (int i = lane; i < rows_b; i += 32) mb = fmax(mb, fabs(B[idx2(i, j, ldb)]));
    for (int o = 16; o > 0; o >>= 1) {
        ma = fmax(ma, __shfl_xor_sync(0xffffffffu, ma, o));
        mb = fmax(mb, __shfl_xor_sync(0xffffffffu, mb, o));
    }
    if (lane == 0) {
        const double mx = fmax(a1 * ma, a2 * mb);
        double d = 1.0;
        if (mx > 0.0 && isfinite(mx)) {
            int e;
            frexp(mx, &e);                 // mx = f 2^e, f in [0.5, 1)
            d = ldexp(1.0, -e);
        }
        D[j] = d;
    }
}

void colscale_pow2(const double *A, int lda, int rows_a, const double *B, int ldb, int rows_b, int n, double a1,
                   double a2, double *D, cudaStream_t s)
{
    if (n <= 0) return;
    ProfScope ps(K_NORM, s);
    k_colscale<<<ceil_div(n, 8), 256, 0, s>>>(A, lda, rows_a, B, ldb, rows_b, n, a1, a2, D);
}

// max|A| and sum of squares, two-stage deterministic reduction.
__global__ void __launch_bounds__(256)
k_absmax_sumsq(const double *__restrict__ A, int lda, int rows, int cols, double *__restrict__ part)
{
    __shared__ double smax[8], ssq[8];
    double mx = 0.0, sq = 0.0;
    const size_t total = (size_t)rows * cols;
    for (size_t e = (size_t)blockIdx.x * 256 + threadIdx.x; e < total; e += (size_t)gridDim.x * 256) {
        const int i = (int)(e % rows), j = (int)(e / rows);
        const double a = A[idx2(i, j, lda)];
        mx = fmax(mx, fabs(a));
        sq = fma(a, a, sq);
    }
    for (int o = 16; o > 0; o >>= 1) {
        mx = fmax(mx, __shfl_xor_sync(0xffffffffu, mx, o));
        sq += __shfl_xor_sync(0xffffffffu, sq, o);
    }
    if ((threadIdx.x & 31) == 0) { smax[threadIdx.x >> 5] = mx; ssq[threadIdx.x >> 5] = sq; }
    __syncthreads();
    if (threadIdx.x == 0) {
        for (int w = 1; w < 8; w++) { mx = fmax(mx, smax[w]); sq += ssq[w]; }
        part[2 * blockIdx.x] = mx;
        part[2 * blockIdx.x + 1] = sq;
    }
}

__global__ void k_absmax_sumsq_final(const double *__restrict__ part, int nb, double *__restrict__ out)
{
    __shared__ double smax[32], ssq[32];
    double mx = 0.0, sq = 0.0;
    for (int b = threadIdx.x; b < nb; b += 32) { mx = fmax(mx, part[2 * b]); sq += part[2 * b + 1]; }
    smax[threadIdx.x] = mx;
    ssq[threadIdx.x] = sq;
    __syncwarp();
    if (threadIdx.x == 0) {
        for (int w = 1; w < 32; w++) { mx = fmax(mx, smax[w]); sq += ssq[w]; }
        out[0] = mx;
        out[1] = sq;
    }
}

void absmax_sumsq(const double *A, int lda, int rows, int cols, double *part, double *out, cudaStream_t s)
{
    if (rows <= 0 || cols <= 0) { cudaMemsetAsync(out, 0, 2 * sizeof(double), s); return; }
    const size_t total = (size_t)rows * cols;
    int nb = (int)((total + 256 * 8 - 1) / (256 * 8));
    if (nb > 1216) nb = 1216;
    if (nb < 1) nb = 1;
    ProfScope ps(K_NORM, s);
    k_absmax_sumsq<<<nb, 256, 0, s>>>(A, lda, rows, cols, part);
    k_absmax_sumsq_final<<<1, 32, 0, s>>>(part, nb, out);
}

// ---------------------------------------------------------- instantiations --
template int apply_reflectors_vec<float>(const float *, int, int, int, const float *, int, float *,
                                         const DevScratch &, cudaStream_t);
template int apply_reflectors_vec<double>(const double *, int, int, int, const double *, int, double *,
                                          const DevScratch &, cudaStream_t);
template int apply_reflectors_vec_blk<float, float>(const float *, int, int, int, const float *, int, int, float *,
                                                    cudaStream_t);
template int apply_reflectors_vec_blk<double, double>(const double *, int, int, int, const double *, int, int,
                                                      double *, cudaStream_t);
template int apply_reflectors_vec_blk<float, double>(const float *, int, int, int, const float *, int, int,
                                                     double *, cudaStream_t);
template int trsv_upper_mixed<float, double>(const float *, int, int, int, double *, const DevScratch &,
                                             cudaStream_t, const double *);
template void invert_diag32_mixed<float, double>(const float *, int, int, double *, int *, cudaStream_t);
template void invert_diag32_mixed<double, double>(const double *, int, int, double *, int *, cudaStream_t);
template int gemv_mixed<float, double>(const float *, int, int, int, int, double, const double *, double,
                                       double *, int, int, cudaStream_t);
template int trsv_upper_mixed<double, double>(const double *, int, int, int, double *, const DevScratch &,
                                              cudaStream_t, const double *);
template int gemv_mixed<double, double>(const double *, int, int, int, int, double, const double *, double,
                                        double *, int, int, cudaStream_t);
template int trsv_upper<float>(const float *, int, int, int, float *, const DevScratch &, cudaStream_t,
                               const float *);
template int trsv_upper<double>(const double *, int, int, int, double *, const DevScratch &, cudaStream_t,
                                const double *);
template void invert_diag32<float>(const float *, int, int, float *, int *, cudaStream_t);
template void invert_diag32<double>(const double *, int, int, double *, int *, cudaStream_t);
template int gemv<float>(const float *, int, int, int, int, float, const float *, float, float *, int, int,
                         cudaStream_t);
template int gemv<double>(const double *, int, int, int, int, double, const double *, double, double *, int,
                          int, cudaStream_t);
template void vcopy<double, float>(const double *, float *, int, double, int, cudaStream_t, const double *);
template void vcopy<double, double>(const double *, double *, int, double, int, cudaStream_t, const double *);
template void vcopy<float, double>(const float *, double *, int, double, int, cudaStream_t, const double *);
template void vcopy<float, float>(const float *, float *, int, double, int, cudaStream_t, const double *);
template void vaxpy<float>(const float *, double *, int, double, int, cudaStream_t, const double *);
template void vaxpy<double>(const double *, double *, int, double, int, cudaStream_t, const double *);
template void mconvert<double, float>(const double *, int, float *, int, int, int, int, int, int, double,
                                      cudaStream_t, const double *, int);
template void mconvert<double, double>(const double *, int, double *, int, int, int, int, int, int, double,
                                      cudaStream_t, const double *, int);
template void mconvert<float, float>(const float *, int, float *, int, int, int, int, int, int, double,
                                      cudaStream_t, const double *, int);
template void mconvert<float, double>(const float *, int, double *, int, int, int, int, int, int, double,
                                      cudaStream_t, const double *, int);

} // namespace mpir

namespace mpir {
template void vdiag<double>(double *, const double *, int, int, cudaStream_t);
template void vdiag<float>(float *, const double *, int, int, cudaStream_t);
} // namespace mpir
