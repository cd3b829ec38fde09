// wyapply.cu -- reflector-set application to one vector with the aggregated
// compact-WY factor Tf of the whole set (built by geqrf, qr.cu):
//     x <- (I - V op(Tf) V^T) x,   op(Tf) = Tf^T (Z^T x) or Tf (Z x),
// as three passes that each span the whole GPU and read their matrix once:
//     y  = V^T x         column dots, one warp per reflector;
//     w' = op(Tf) y      column dots (Tf^T) or row products (Tf);
//     x -= V w'          row products over 64-column chunks, then a sum of
//                        the chunk partials in a fixed order (deterministic).
// This is the vector side of every correction solve (Sec. 3, Alg. 3 / 4:
// the orthogonal factors of the generalized factorizations applied to the
// residual vectors); the blocked form applies one 128-reflector block after
// the other, each block a dependent step.
#include "common.cuh"
#include "kernels.h"
#include "mpir.h"

namespace mpir {

constexpr int WY_RT = 256;     // rows per tile of the row products (one per thread)
constexpr int WY_CC = 64;      // columns per chunk of the row products
constexpr int WY_U = 16;       // independent loads in flight per thread

// Whether tile (rows from i0) x chunk (columns from c0) of the row products
// meets the nonzero triangle: mode 0, unit lower trapezoid (j <= i); mode 1,
// upper triangle (j >= i).  The final sums use the same predicate.
template <int MODE>
__host__ __device__ __forceinline__ bool wy_chunk_valid(int i0, int c0, int nrow, int ncol)
{
    if (MODE == 0) return c0 <= min(i0 + WY_RT, nrow) - 1;
    return min(c0 + WY_CC, ncol) - 1 >= i0;
}

// Column dots, one warp per column j < ncol:
//   mode 0 (V): out_j = v_j + sum_{j < i < len} A(i, j) v_i   (unit diagonal; R above is not read)
//   mode 1 (Tf^T): out_j = sum_{k <= j} A(k, j) v_k
template <typename TS, typename T, int MODE>
__global__ void __launch_bounds__(256)
k_wy_coldot(const TS *__restrict__ A, int lda, int ncol, int len, const T *__restrict__ v, T *__restrict__ out)
{
    pdl_wait();
    pdl_trigger();
    const int lane = threadIdx.x & 31;
    const int j = blockIdx.x * 8 + (threadIdx.x >> 5);
    if (j >= ncol) return;
    const TS *col = A + (size_t)j * lda;
    const int lo = MODE == 0 ? j + 1 : 0;
    const int hi = MODE == 0 ? len : j + 1;
    T acc = T(0);
    for (int i0 = lo; i0 < hi; i0 += 32 * WY_U) {
        TS a[WY_U];
        T b[WY_U];
#pragma unroll
        for (int u = 0; u < WY_U; u++) {
            const int i = i0 + lane + 32 * u;
            a[u] = i < hi ? col[i] : TS(0);
            b[u] = i < hi ? v[i] : T(0);
        }
#pragma unroll
        for (int u = 0; u < WY_U; u++) acc = fma((T)a[u], b[u], acc);
    }
    acc = warp_sum(acc);
    if (lane == 0) out[j] = MODE == 0 ? acc + v[j] : acc;
}

// Row products: part[c * nrow + i] = sum_{j in chunk c} A~(i, j) w_j with
//   mode 0 (V): A~(i, j) = A(i, j) for j < i, 1 for j = i, 0 for j > i;
//   mode 1 (Tf): A~(i, j) = A(i, j) for j >= i, 0 below.
// Thread = row (coalesced column segments); grid (row tiles, chunks); a
// tile/chunk pair off the triangle returns without writing.
template <typename TS, typename T, int MODE>
__global__ void __launch_bounds__(WY_RT)
k_wy_rowprod(const TS *__restrict__ A, int lda, int nrow, int ncol, const T *__restrict__ w, T *__restrict__ part)
{
    pdl_wait();
    pdl_trigger();
    const int i0 = blockIdx.x * WY_RT, c0 = blockIdx.y * WY_CC;
    if (!wy_chunk_valid<MODE>(i0, c0, nrow, ncol)) return;
    __shared__ T ws[WY_CC];
    const int tid = threadIdx.x;
    const int cn = min(WY_CC, ncol - c0);
    if (tid < WY_CC) ws[tid] = tid < cn ? w[c0 + tid] : T(0);
    __syncthreads();
    const int i = i0 + tid;
    if (i >= nrow) return;
    T acc = T(0);
    for (int j0 = c0; j0 < c0 + cn; j0 += WY_U) {
        TS a[WY_U];
#pragma unroll
        for (int u = 0; u < WY_U; u++) {
            const int j = j0 + u;
            bool nz = j < c0 + cn && (MODE == 0 ? j <= i : j >= i);
            a[u] = nz ? ((MODE == 0 && j == i) ? TS(1) : A[(size_t)j * lda + i]) : TS(0);
        }
#pragma unroll
        for (int u = 0; u < WY_U; u++) acc = fma((T)a[u], ws[(j0 + u - c0) & (WY_CC - 1)], acc);
    }
    part[(size_t)blockIdx.y * nrow + i] = acc;
}

// mode 0: x_i -= sum over the valid chunks; mode 1: x_i = that sum.
template <typename T, int MODE>
__global__ void __launch_bounds__(256)
k_wy_final(const T *__restrict__ part, int nrow, int ncol, T *__restrict__ x)
{
    pdl_wait();
    pdl_trigger();
    const int i = blockIdx.x * 256 + threadIdx.x;
    if (i >= nrow) return;
    const int i0 = (i / WY_RT) * WY_RT;
    const int nch = ceil_div(ncol, WY_CC);
    T sum = T(0);
    for (int c = 0; c < nch; c++)
        if (wy_chunk_valid<MODE>(i0, c * WY_CC, nrow, ncol)) sum += part[(size_t)c * nrow + i];
    if (MODE == 0) x[i] -= sum; else x[i] = sum;
}

static size_t rup256(size_t b) { return (b + 255) & ~(size_t)255; }

size_t wy_apply_ws_bytes(int M, int K)
{
    if (M < 1) M = 1;
    if (K < 1) K = 1;
    const size_t e = sizeof(double);
    const size_t nch = (size_t)ceil_div(K, WY_CC);
    return 2 * rup256((size_t)K * e) + rup256(nch * (size_t)(M > K ? M : K) * e);
}

template <typename TS, typename T>
static int wy_apply_one(const TS *V, int ldv, int M, int K, const TS *Tf, int ldt, int trans, T *x, void *ws,
                        cudaStream_t s)
{
    unsigned char *b = static_cast<unsigned char *>(ws);
    T *y = reinterpret_cast<T *>(b);
    T *wp = reinterpret_cast<T *>(b + rup256((size_t)K * sizeof(double)));
    T *part = reinterpret_cast<T *>(b + 2 * rup256((size_t)K * sizeof(double)));
    const int nch = ceil_div(K, WY_CC);
    {
        ProfScope ps(K_VEC_APPLY, s);
        pdl_launch(k_wy_coldot<TS, T, 0>, dim3(ceil_div(K, 8)), dim3(256), 0, s, V, ldv, K, M, x, y);
    }
    if (trans) {
        ProfScope ps(K_VEC_APPLY, s);
        pdl_launch(k_wy_coldot<TS, T, 1>, dim3(ceil_div(K, 8)), dim3(256), 0, s, Tf, ldt, K, K, y, wp);
    } else {
        {
            ProfScope ps(K_VEC_APPLY, s);
            pdl_launch(k_wy_rowprod<TS, T, 1>, dim3(ceil_div(K, WY_RT), nch), dim3(WY_RT), 0, s, Tf, ldt, K, K, y, part);
        }
        ProfScope ps(K_VEC_APPLY, s);
        pdl_launch(k_wy_final<T, 1>, dim3(ceil_div(K, 256)), dim3(256), 0, s, part, K, K, wp);
    }
    {
        ProfScope ps(K_VEC_APPLY, s);
        pdl_launch(k_wy_rowprod<TS, T, 0>, dim3(ceil_div(M, WY_RT), nch), dim3(WY_RT), 0, s, V, ldv, M, K, wp, part);
    }
    {
        ProfScope ps(K_VEC_APPLY, s);
        pdl_launch(k_wy_final<T, 0>, dim3(ceil_div(M, 256)), dim3(256), 0, s, part, M, K, x);
    }
    return cudaGetLastError() == cudaSuccess ? 0 : MPIR_CUDA_ERROR;
}

// The aggregated factor holds one compact-WY factor per segment of WY_SEG
// reflectors (the factorization couples each outer block only to the
// earlier blocks of its segment): Q = Q_0 Q_1 ..., segment g acting on rows
// and columns from g WY_SEG on.  Q^T x runs the segments first to last,
// Q x last to first.
template <typename TS, typename T>
int wy_apply_vec(const TS *V, int ldv, int M, int K, const TS *Tf, int ldt, int trans, T *x, void *ws,
                 cudaStream_t s)
{
    if (K <= 0 || M <= 0) return 0;
    if (K > M || ldv < M || ldt < K || !ws) return MPIR_UNSUP();
    const int nseg = ceil_div(K, WY_SEG);
    for (int k = 0; k < nseg; k++) {
        const int g = trans ? k : nseg - 1 - k;
        const int S = g * WY_SEG, E = std::min(K, S + WY_SEG);
        const int rc = wy_apply_one<TS, T>(V + idx2(S, S, ldv), ldv, M - S, E - S, Tf + idx2(S, S, ldt), ldt, trans,
                                           x + S, ws, s);
        if (rc) return rc;
    }
    return 0;
}

template int wy_apply_vec<float, float>(const float *, int, int, int, const float *, int, int, float *, void *,
                                        cudaStream_t);
template int wy_apply_vec<float, double>(const float *, int, int, int, const float *, int, int, double *, void *,
                                         cudaStream_t);

} // namespace mpir
