// qr.cu -- blocked Householder QR on GB300: cluster panel kernels with
// st.async column messages, cluster inner updates, tensor-core outer
// updates with look-ahead, and the aggregated compact-WY factor of the whole
// reflector set.  The generalized factorizations of the paper (GRQ for LSE,
// GQR for GLS, Lemma 4.5 / 4.6) are built from this one QR: an RQ
// factorization of C is a QR factorization of the reversed transpose of C
// (the host driver forms that copy), so every reflector is a column of a
// column-major matrix and every access below is coalesced.
#include "common.cuh"
#include "gemm_tc.h"
#include "kernels.h"
#include "mpir.h"

namespace mpir {

constexpr int PANEL_NT = 512;
constexpr int PANEL_RPT = 2;                      // rows held per thread
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
// Cluster message passing of the panel: every CTA pushes its column message
// into every CTA's shared memory with st.async, which signals the
// receiver's mbarrier (complete_tx); the receiver announces the bytes it
// expects one column ahead, so no message can arrive before its count.

__device__ __forceinline__ uint32_t pq_smem(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ uint32_t pq_mapa(uint32_t addr, int rank)
{
    uint32_t r;
    asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(r) : "r"(addr), "r"(rank));
    return r;
}

__device__ __forceinline__ void pq_st_async(uint32_t raddr, float4 v, uint32_t rbar)
{
    asm volatile("st.async.shared::cluster.mbarrier::complete_tx::bytes.v4.f32 [%0], {%1, %2, %3, %4}, [%5];"
                 ::"r"(raddr), "f"(v.x), "f"(v.y), "f"(v.z), "f"(v.w), "r"(rbar) : "memory");
}

__device__ __forceinline__ void pq_expect_tx(uint32_t bar, uint32_t bytes)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes) : "memory");
}

// Bounded wait on the phase of parity `parity`; false on timeout.  Polls
// with test_wait (no suspension of the waiting warp between polls).
constexpr uint32_t PANEL_POLL_LIMIT = 1u << 26;
__device__ __forceinline__ bool pq_wait(uint32_t bar, uint32_t parity)
{
    for (uint32_t it = 0; it < PANEL_POLL_LIMIT; it++) {
        uint32_t done;
        asm volatile("{\n\t.reg .pred p;\n\t"
                     "mbarrier.test_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
                     "selp.u32 %0, 1, 0, p;\n\t}"
                     : "=r"(done)
                     : "r"(bar), "r"(parity)
                     : "memory");
        if (done) return true;
    }
    return false;
}

// v[k] for a warp-uniform k by a log-depth select tree (N a power of two):
// N - 1 selects, dependency depth log2(N), compile-time register indices.
template <typename T, int N>
__device__ __forceinline__ T pq_select(const T (&v)[N], int k)
{
    T t[N];
#pragma unroll
    for (int c = 0; c < N; c++) t[c] = v[c];
#pragma unroll
    for (int w = 1; w < N; w *= 2)
#pragma unroll
        for (int c = 0; c < N; c += 2 * w) t[c] = (k & w) ? t[c + w] : t[c];
    return t[0];
}

// Compact-WY factor of a panel from its Gram entries (one warp, lane k
// forms column k):  Tw = (triu(G, 1) + diag(1 / tau))^{-1}, i.e.
//   T(k, k) = tau_k,  T(i, k) = -tau_i sum_{c > i} G(i, c) T(c, k)  (i < k).
// Column k lives in registers (t[c] = 0 for c > k) and the recurrence is
// fully unrolled, so the only serial chain is one product per row; the G
// entries are warp-broadcast shared-memory reads.
template <typename T, int NB, int LDG>
__device__ __forceinline__ void panel_T_from_gram(const T (*G_s)[LDG], const T *tau_s, int kpanel, T *Tw)
{
    const int k = threadIdx.x & 31;
    T t[NB];
#pragma unroll
    for (int i = NB - 1; i >= 0; i--) {
        T sum = T(0);
#pragma unroll
        for (int c = i + 1; c < NB; c++) sum = fma(G_s[i][c], t[c], sum);
        const T ti = i == k ? tau_s[i] : -tau_s[i] * sum;
        t[i] = (i <= k && k < kpanel) ? ti : T(0);
    }
    if (k < NB) {
#pragma unroll
        for (int i = 0; i < NB; i++) Tw[i + (size_t)k * NB] = t[i];
    }
}

template <typename T, int NB, int NT, int RPT>
__global__ void __launch_bounds__(NT, 1)
k_panel_qr(T *__restrict__ A, int lda, int M, int j0, int ncols, int chunk,
           T *__restrict__ tau, T *__restrict__ Tw, int *__restrict__ err)
{
    constexpr int NW = NT / 32;
    cg::cluster_group cluster = cg::this_cluster();
    const int cs = (int)cluster.num_blocks();
    const int crank = (int)cluster.block_rank();
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int L = M - j0;
    const int kpanel = min(ncols, L);

    // column message of a CTA: its partial sums (NB) and its part of the
    // pivot row (NB; nonzero on rank 0 only), 16-byte vectors
    constexpr int MSG = 2 * NB;
    constexpr int NV = MSG * (int)sizeof(T) / 16;
    static_assert(MSG * sizeof(T) % 16 == 0, "message of whole 16-byte vectors");
    __shared__ T red_s[2][NW][32];
    __shared__ __align__(16) T xbuf[NW][MSG];               // each warp's copy of the message
    __shared__ __align__(16) T gbuf[2][16][MSG];
    __shared__ __align__(8) unsigned long long mbar[2];
    __shared__ T prow[2][NB];
    __shared__ __align__(16) T coefw[NW][NB];
    __shared__ T G_s[NB][NB + 1];
    __shared__ T tau_s[NB];

    const int row_base = crank * chunk;
    const int row_end = min(row_base + chunk, L);
    const uint32_t msg_bytes = (uint32_t)(cs * MSG * sizeof(T));
    bool timed_out = false;
    // Gram entries beyond the panel stay zero (the T recurrence reads them)
    for (int e = tid; e < NB * (NB + 1); e += NT) (&G_s[0][0])[e] = T(0);
    if (cs > 1) {
        if (tid == 0) {
            asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(pq_smem(&mbar[0])) : "memory");
            asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(pq_smem(&mbar[1])) : "memory");
            asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
            pq_expect_tx(pq_smem(&mbar[0]), msg_bytes);        // column 0
        }
        cluster.sync();                                         // barriers ready before any message
    }
    int rr[RPT];
    T a[RPT][NB];
#pragma unroll
    for (int q = 0; q < RPT; q++) {
        int r = row_base + tid + q * NT;
        rr[q] = r < row_end ? r : -1;
    }
#pragma unroll
    for (int c = 0; c < NB; c++) {
        const T *col = A + idx2(j0, j0 + c, lda);
#pragma unroll
        for (int q = 0; q < RPT; q++)
            a[q][c] = (rr[q] >= 0 && c < ncols) ? col[rr[q]] : T(0);
    }

    // Runtime column loop (a fully unrolled loop overflows the instruction
    // cache); register-array indices stay compile-time through predication.
#pragma unroll 1
    for (int kk = 0; kk < kpanel; kk++) {
        const int par = kk & 1;
        // pivot-column value of each owned row (select tree, no dynamic index)
        T akk[RPT];
#pragma unroll
        for (int q = 0; q < RPT; q++) akk[q] = pq_select<T, NB>(a[q], kk);
        // the reduction runs in halves of H columns to bound the number of
        // live accumulators (registers hold the panel itself)
        constexpr int H = NB > 16 ? 16 : NB;
#pragma unroll
        for (int h0 = 0; h0 < NB; h0 += H) {
            T acc[H];
#pragma unroll
            for (int c = 0; c < H; c++) acc[c] = T(0);
#pragma unroll
            for (int q = 0; q < RPT; q++) {
                const T ak = rr[q] > kk ? akk[q] : T(0);   // rows below the pivot
#pragma unroll
                for (int c = 0; c < H; c++) acc[c] = fma(ak, a[q][h0 + c], acc[c]);
            }
            T wsum = warp_transpose_reduce<T, H>(acc);
            if (lane < H) red_s[par][warp][h0 + lane] = wsum;
        }
#pragma unroll
        for (int q = 0; q < RPT; q++) {
            if (rr[q] == kk) {
#pragma unroll
                for (int c = 0; c < NB; c++) prow[par][c] = a[q][c];
            }
        }
        // the next column's message count is announced before this column's
        // messages leave (no CTA can send column kk+1 before it has ours)
        if (cs > 1 && tid == 0 && kk + 1 < kpanel) pq_expect_tx(pq_smem(&mbar[par ^ 1]), msg_bytes);
        __syncthreads();
        // every warp forms the column totals and the coefficients itself
        T tot = T(0), pj = T(0);
        if (cs == 1) {
            if (lane < NB) {
#pragma unroll
                for (int w = 0; w < NW; w++) tot += red_s[par][w][lane];
                pj = prow[par][lane];
            }
        } else {
            // every warp forms the CTA's message and sends it to its share
            // of the destinations (ranks warp, warp + NW, ...)
            if (lane < NB) {
                T t = T(0);
#pragma unroll
                for (int w = 0; w < NW; w++) t += red_s[par][w][lane];
                xbuf[warp][lane] = t;
                xbuf[warp][NB + lane] = crank == 0 ? prow[par][lane] : T(0);
            }
            __syncwarp();
            if (lane < NV) {
                const float4 v = reinterpret_cast<const float4 *>(&xbuf[warp][0])[lane];
                const uint32_t dst = pq_smem(&gbuf[par][crank][0]) + 16 * lane;
                const uint32_t bar = pq_smem(&mbar[par]);
                for (int r = warp; r < cs; r += NW) pq_st_async(pq_mapa(dst, r), v, pq_mapa(bar, r));
            }
            // after a timeout the remaining columns skip their waits (the
            // error flag reports the panel; the kernel still ends promptly)
            if (!timed_out && !pq_wait(pq_smem(&mbar[par]), (uint32_t)(kk >> 1) & 1u)) timed_out = true;
            if (lane < NB) {
                T t2 = T(0), p2 = T(0);
                int r = 0;
                for (; r + 1 < cs; r += 2) {
                    tot += gbuf[par][r][lane];
                    t2 += gbuf[par][r + 1][lane];
                    pj += gbuf[par][r][NB + lane];
                    p2 += gbuf[par][r + 1][NB + lane];
                }
                if (r < cs) { tot += gbuf[par][r][lane]; pj += gbuf[par][r][NB + lane]; }
                tot += t2;
                pj += p2;
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
        if (lane < NB) coefw[warp][lane] = lane > kk ? tv * dot : T(0);
        if (warp == 0) {
            if (lane < kk) G_s[lane][kk] = dot;
            if (lane == 0) tau_s[kk] = tv;
        }
        __syncwarp();
        // branch-free update: f = v_i (scale * a(i,kk) below the pivot, 1 on
        // the pivot row, 0 above); a(i, c) -= coef_c * f (coef_c = 0 for
        // c <= kk); the pivot column becomes v (or beta on the pivot row)
        // groups of 8 columns wholly left of the pivot are untouched (warp-
        // uniform branch)
#pragma unroll
        for (int q = 0; q < RPT; q++) {
            const bool below = rr[q] > kk, piv = rr[q] == kk;
            const T sk = akk[q] * scale;
            const T f = below ? sk : (piv ? T(1) : T(0));
            const T newk = below ? sk : (piv ? beta : akk[q]);
#pragma unroll
            for (int g = 0; g < NB; g += 8) {
                if (g + 7 >= kk) {
#pragma unroll
                    for (int c = g; c < g + 8; c++) {
                        const T upd = fma(-coefw[warp][c], f, a[q][c]);
                        a[q][c] = (c == kk) ? newk : upd;
                    }
                }
            }
        }
    }
    __syncthreads();

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
        panel_T_from_gram<T, NB, NB + 1>(G_s, tau_s, kpanel, Tw);
    }
    if (timed_out) atomicOr(err, 8);
    if (cs > 1) cluster.sync();   // no CTA leaves while messages to it may be in flight
}

// ---------------------------------------------------------------------------
// FP32 panel with two threads per row (k_panel_qr's algorithm, same column
// message protocol): lane pair (2r, 2r+1) of a warp holds row r's columns
// 0..15 and 16..31.  Every per-column chain (pivot select, products, the
// warp reduction, the update) is half as long, and a CTA has twice the warps
// to hide latency.  The warp reduction exchanges only between lanes of the
// same half (xor 16, 8, 4, 2), leaving lane l with the warp total of column
// 16 (l & 1) + (l >> 1).  NT threads hold NT / 2 rows.
// ---------------------------------------------------------------------------
template <int NT>
__global__ void __launch_bounds__(NT, 1)
k_panel_qr2(float *__restrict__ A, int lda, int M, int j0, int ncols, int chunk, float *__restrict__ tau,
            float *__restrict__ Tw, int *__restrict__ err)
{
    constexpr int NB = 32, HB = 16;
    constexpr int NW = NT / 32;
    cg::cluster_group cluster = cg::this_cluster();
    const int cs = (int)cluster.num_blocks();
    const int crank = (int)cluster.block_rank();
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int h = lane & 1;                              // this thread's half of the row
    const int L = M - j0;
    const int kpanel = min(ncols, L);
    constexpr int MSG = 2 * NB;
    constexpr int NV = MSG * (int)sizeof(float) / 16;
    __shared__ float red_s[2][NW][32];
    __shared__ __align__(16) float xbuf[NW][MSG];
    __shared__ __align__(16) float gbuf[2][16][MSG];
    __shared__ __align__(8) unsigned long long mbar[2];
    __shared__ float prow[2][NB];
    __shared__ __align__(16) float coefw[NW][NB];
    __shared__ float G_s[NB][NB + 1];
    __shared__ float tau_s[NB];

    const int row_base = crank * chunk;
    const int row_end = min(row_base + chunk, L);
    const uint32_t msg_bytes = (uint32_t)(cs * MSG * sizeof(float));
    bool timed_out = false;
    for (int e = tid; e < NB * (NB + 1); e += NT) (&G_s[0][0])[e] = 0.f;
    if (cs > 1) {
        if (tid == 0) {
            asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(pq_smem(&mbar[0])) : "memory");
            asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(pq_smem(&mbar[1])) : "memory");
            asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
            pq_expect_tx(pq_smem(&mbar[0]), msg_bytes);
        }
        cluster.sync();
    }
    // programmatic dependent launch: everything above overlaps the previous
    // kernel's tail; its results are read only after this wait
    pdl_wait();
    pdl_trigger();
    const int r = row_base + warp * 16 + (lane >> 1);
    const int rr = r < row_end ? r : -1;
    float a[HB];
#pragma unroll
    for (int c = 0; c < HB; c++) {
        const int cc = HB * h + c;
        a[c] = (rr >= 0 && cc < ncols) ? A[idx2(j0 + rr, j0 + cc, lda)] : 0.f;
    }
    const int col_of_lane = HB * h + (lane >> 1);        // column total this lane ends with

#pragma unroll 1
    for (int kk = 0; kk < kpanel; kk++) {
        const int par = kk & 1;
        // pivot value of the row: select in the half that holds column kk,
        // exchanged within the lane pair
        const float vsel = pq_select<float, HB>(a, kk & (HB - 1));
        const float vother = __shfl_xor_sync(0xffffffffu, vsel, 1);
        const float akk = (h == (kk >> 4)) ? vsel : vother;
        float acc[HB];
        {
            const float ak = rr > kk ? akk : 0.f;        // rows below the pivot
#pragma unroll
            for (int c = 0; c < HB; c++) acc[c] = ak * a[c];
        }
        // transpose-reduce over the 16 lanes of the same half
#pragma unroll
        for (int sft = HB / 2; sft >= 1; sft >>= 1) {
            const int m = 2 * sft;
            const bool upper = (lane & m) != 0;
#pragma unroll
            for (int i = 0; i < sft; i++) {
                const float send = upper ? acc[i] : acc[i + sft];
                const float keep = upper ? acc[i + sft] : acc[i];
                acc[i] = keep + __shfl_xor_sync(0xffffffffu, send, m);
            }
        }
        red_s[par][warp][col_of_lane] = acc[0];
        if (rr == kk) {
#pragma unroll
            for (int c = 0; c < HB; c++) prow[par][HB * h + c] = a[c];
        }
        if (cs > 1 && tid == 0 && kk + 1 < kpanel) pq_expect_tx(pq_smem(&mbar[par ^ 1]), msg_bytes);
        __syncthreads();
        float tot = 0.f, pj = 0.f;
        if (cs == 1) {
#pragma unroll
            for (int w = 0; w < NW; w++) tot += red_s[par][w][lane];
            pj = prow[par][lane];
        } else {
            {
                float t = 0.f;
#pragma unroll
                for (int w = 0; w < NW; w++) t += red_s[par][w][lane];
                xbuf[warp][lane] = t;
                xbuf[warp][NB + lane] = crank == 0 ? prow[par][lane] : 0.f;
            }
            __syncwarp();
            if (lane < NV) {
                const float4 v = reinterpret_cast<const float4 *>(&xbuf[warp][0])[lane];
                const uint32_t dst = pq_smem(&gbuf[par][crank][0]) + 16 * lane;
                const uint32_t bar = pq_smem(&mbar[par]);
                for (int q = warp; q < cs; q += NW) pq_st_async(pq_mapa(dst, q), v, pq_mapa(bar, q));
            }
            if (!timed_out && !pq_wait(pq_smem(&mbar[par]), (uint32_t)(kk >> 1) & 1u)) timed_out = true;
            float t2 = 0.f, p2 = 0.f;
            int q = 0;
            for (; q + 1 < cs; q += 2) {
                tot += gbuf[par][q][lane];
                t2 += gbuf[par][q + 1][lane];
                pj += gbuf[par][q][NB + lane];
                p2 += gbuf[par][q + 1][NB + lane];
            }
            if (q < cs) { tot += gbuf[par][q][lane]; pj += gbuf[par][q][NB + lane]; }
            tot += t2;
            pj += p2;
        }
        const float alpha = __shfl_sync(0xffffffffu, pj, kk);
        const float sp = __shfl_sync(0xffffffffu, tot, kk);
        float beta, tv, scale;
        if (sp == 0.f) {
            tv = 0.f; beta = alpha; scale = 1.f;
        } else {
            const float nrm = sqrtf(alpha * alpha + sp);
            beta = alpha >= 0.f ? -nrm : nrm;
            tv = (beta - alpha) / beta;
            scale = 1.f / (alpha - beta);
        }
        const float dot = pj + scale * tot;
        coefw[warp][lane] = lane > kk ? tv * dot : 0.f;
        if (warp == 0) {
            if (lane < kk) G_s[lane][kk] = dot;
            if (lane == 0) tau_s[kk] = tv;
        }
        __syncwarp();
        {
            const bool below = rr > kk, piv = rr == kk;
            const float sk = akk * scale;
            const float f = below ? sk : (piv ? 1.f : 0.f);
            const float newk = below ? sk : (piv ? beta : akk);
            const int kloc = kk - HB * h;                 // pivot index in this half (may be out of range)
#pragma unroll
            for (int q = 0; q < HB / 4; q++) {
                const float4 cw = *reinterpret_cast<const float4 *>(&coefw[warp][HB * h + 4 * q]);
                const float cv[4] = {cw.x, cw.y, cw.z, cw.w};
#pragma unroll
                for (int u = 0; u < 4; u++) {
                    const int c = 4 * q + u;
                    const float upd = fmaf(-cv[u], f, a[c]);
                    a[c] = (c == kloc) ? newk : upd;
                }
            }
        }
    }
    __syncthreads();

    float *Aw = A;
    asm volatile("" : "+l"(Aw));
    if (rr >= 0) {
#pragma unroll
        for (int c = 0; c < HB; c++) {
            const int cc = HB * h + c;
            if (cc < ncols) Aw[idx2(j0 + rr, j0 + cc, lda)] = a[c];
        }
    }
    if (crank == 0 && warp == 0) {
        if (lane < kpanel) tau[j0 + lane] = tau_s[lane];
        panel_T_from_gram<float, NB, NB + 1>(G_s, tau_s, kpanel, Tw);
    }
    if (timed_out) atomicOr(err, 8);
    if (cs > 1) cluster.sync();
}

// ---------------------------------------------------------------------------
// Panels taller than one 16-CTA cluster holds (the row chunks of
// k_panel_qr on more CTAs than a cluster allows): the same column step with
// the cluster message replaced by a global-memory exchange.  Each CTA
// writes its partial sums and its part of the pivot row to gx (two parity
// slots of gridDim.x x 2 NB), a bounded grid barrier follows (cooperative
// launch: all CTAs are resident), and every CTA sums the slots in rank
// order (L2 reads), so all CTAs hold bitwise the same column totals.
// ---------------------------------------------------------------------------
struct PanelGrid {
    void *gx;               // 2 x PANEL_GRID_MAX x 2 NB elements of the panel type
    unsigned int *bar;      // grid barrier: [0] arrivals (zero between launches), [1] generation
};
constexpr int PANEL_GRID_MAX = 160;              // CTAs (one per SM)

template <typename T, int NB, int NT, int RPT>
__global__ void __launch_bounds__(NT, 1)
k_panel_qr_grid(T *__restrict__ A, int lda, int M, int j0, int ncols, int chunk, T *__restrict__ tau,
                T *__restrict__ Tw, int *__restrict__ err, T *__restrict__ gx, GridBarrier gb)
{
    constexpr int NW = NT / 32;
    const int G = (int)gridDim.x, rank = (int)blockIdx.x;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int L = M - j0;
    const int kpanel = min(ncols, L);
    __shared__ T red_s[2][NW][32];
    __shared__ T rsum[NW][2][32];
    __shared__ T prow[2][NB];
    __shared__ __align__(16) T coefw[NW][NB];
    __shared__ T G_s[NB][NB + 1];
    __shared__ T tau_s[NB];

    const int row_base = rank * chunk;
    const int row_end = min(row_base + chunk, L);
    bool timed_out = false;
    for (int e = tid; e < NB * (NB + 1); e += NT) (&G_s[0][0])[e] = T(0);
    int rr[RPT];
    T a[RPT][NB];
#pragma unroll
    for (int q = 0; q < RPT; q++) {
        const int r = row_base + tid + q * NT;
        rr[q] = r < row_end ? r : -1;
    }
#pragma unroll
    for (int c = 0; c < NB; c++) {
        const T *col = A + idx2(j0, j0 + c, lda);
#pragma unroll
        for (int q = 0; q < RPT; q++) a[q][c] = (rr[q] >= 0 && c < ncols) ? col[rr[q]] : T(0);
    }
#pragma unroll 1
    for (int kk = 0; kk < kpanel; kk++) {
        const int par = kk & 1;
        T akk[RPT];
#pragma unroll
        for (int q = 0; q < RPT; q++) akk[q] = pq_select<T, NB>(a[q], kk);
        constexpr int H = NB > 16 ? 16 : NB;
#pragma unroll
        for (int h0 = 0; h0 < NB; h0 += H) {
            T acc[H];
#pragma unroll
            for (int c = 0; c < H; c++) acc[c] = T(0);
#pragma unroll
            for (int q = 0; q < RPT; q++) {
                const T ak = rr[q] > kk ? akk[q] : T(0);
#pragma unroll
                for (int c = 0; c < H; c++) acc[c] = fma(ak, a[q][h0 + c], acc[c]);
            }
            T wsum = warp_transpose_reduce<T, H>(acc);
            if (lane < H) red_s[par][warp][h0 + lane] = wsum;
        }
#pragma unroll
        for (int q = 0; q < RPT; q++) {
            if (rr[q] == kk) {
#pragma unroll
                for (int c = 0; c < NB; c++) prow[par][c] = a[q][c];
            }
        }
        __syncthreads();
        T *slot = gx + ((size_t)par * PANEL_GRID_MAX + rank) * 2 * NB;
        if (warp == 0 && lane < NB) {
            T t = T(0);
#pragma unroll
            for (int w = 0; w < NW; w++) t += red_s[par][w][lane];
            slot[lane] = t;
            slot[NB + lane] = rank == 0 ? prow[par][lane] : T(0);
        }
        // after a timeout the remaining columns skip the barrier (the error
        // flag reports the panel; the kernel still ends promptly)
        if (!timed_out && !grid_sync(gb, (unsigned)G)) timed_out = true;
        // rank-order sums: warp w takes ranks w, w + NW, ...; then over warps
        {
            T t = T(0), pp = T(0);
            if (lane < NB)
                for (int q = warp; q < G; q += NW) {
                    const T *sq = gx + ((size_t)par * PANEL_GRID_MAX + q) * 2 * NB;
                    t += __ldcg(sq + lane);
                    pp += __ldcg(sq + NB + lane);
                }
            rsum[warp][0][lane] = t;
            rsum[warp][1][lane] = pp;
        }
        __syncthreads();
        T tot = T(0), pj = T(0);
        if (lane < NB) {
#pragma unroll
            for (int w = 0; w < NW; w++) { tot += rsum[w][0][lane]; pj += rsum[w][1][lane]; }
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
        if (lane < NB) coefw[warp][lane] = lane > kk ? tv * dot : T(0);
        if (warp == 0) {
            if (lane < kk) G_s[lane][kk] = dot;
            if (lane == 0) tau_s[kk] = tv;
        }
        __syncwarp();
#pragma unroll
        for (int q = 0; q < RPT; q++) {
            const bool below = rr[q] > kk, piv = rr[q] == kk;
            const T sk = akk[q] * scale;
            const T f = below ? sk : (piv ? T(1) : T(0));
            const T newk = below ? sk : (piv ? beta : akk[q]);
#pragma unroll
            for (int g = 0; g < NB; g += 8) {
                if (g + 7 >= kk) {
#pragma unroll
                    for (int c = g; c < g + 8; c++) {
                        const T upd = fma(-coefw[warp][c], f, a[q][c]);
                        a[q][c] = (c == kk) ? newk : upd;
                    }
                }
            }
        }
    }
    __syncthreads();
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
    if (rank == 0 && warp == 0) {
        if (lane < kpanel) tau[j0 + lane] = tau_s[lane];
        panel_T_from_gram<T, NB, NB + 1>(G_s, tau_s, kpanel, Tw);
    }
    if (timed_out) atomicOr(err, 8);
}

// ---------------------------------------------------------------------------
// FP32 panel with column pairs (k_panel_qr's layout and message protocol,
// one message round per two columns).  A round for columns kk, kk+1 sums,
// over the rows below kk+1,
//     S1[c] = sum_i a(i,kk) a(i,c),   S2[c] = sum_i a(i,kk+1) a(i,c)   (all c),
// and broadcasts the pivot rows P1 = a(kk,:), P2 = a(kk+1,:).  Reflector kk
// is the single-column one with row kk+1 added back (S1 + P2[kk] P2).  It
// changes column c below row kk+1 into a(:,c) - g_c w (w = a(:,kk), g_c =
// scale1 tau1 dot1[c]; column kk itself into scale1 w), so the sums the
// second reflector needs expand into S1, S2 and the g's:
//     sum a'(i,kk+1) a'(i,c) = S2[c] - g_c S1[kk+1] - g S1[c] + g g_c S1[kk]
// (g = g_{kk+1}), and its pivot row is P2 - g_c P2[kk].  That downdate
// cancels when column kk+1 is nearly parallel to column kk: where its
// squared norm below the pivot falls under 1/16 of S2[kk+1], the round
// applies reflector kk only and the next round starts at kk+1.  Every warp
// of every CTA evaluates the same totals in the same order, so the choice
// is uniform over the cluster.
// ---------------------------------------------------------------------------
constexpr float PAIR_GUARD = 0.0625f;

__device__ __forceinline__ void pair_reflector(float alpha, float sp, float &tv, float &beta, float &scale)
{
    if (sp == 0.f) {
        tv = 0.f; beta = alpha; scale = 1.f;
    } else {
        const float nrm = sqrtf(alpha * alpha + sp);
        beta = alpha >= 0.f ? -nrm : nrm;
        tv = (beta - alpha) / beta;
        scale = 1.f / (alpha - beta);
    }
}

template <int NT, int RPT>
__global__ void __launch_bounds__(NT, 1)
k_panel_qr_pair(float *__restrict__ A, int lda, int M, int j0, int ncols, int chunk, float *__restrict__ tau,
                float *__restrict__ Tw, int *__restrict__ err)
{
    constexpr int NB = 32, H = 16;
    constexpr int NW = NT / 32;
    cg::cluster_group cluster = cg::this_cluster();
    const int cs = (int)cluster.num_blocks();
    const int crank = (int)cluster.block_rank();
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int L = M - j0;
    const int kpanel = min(ncols, L);
    constexpr int MSG = 4 * NB;                          // S1, S2, P1, P2
    static_assert(MSG * sizeof(float) / 16 == 32, "one 16-byte vector per lane");
    __shared__ float red_s[2][NW][2 * NB];
    __shared__ __align__(16) float xbuf[NW][MSG];
    __shared__ __align__(16) float gbuf[2][16][MSG];
    __shared__ __align__(8) unsigned long long mbar[2];
    __shared__ float prow[2][2][NB];
    __shared__ __align__(16) float coefw[NW][2][NB];
    __shared__ float G_s[NB][NB + 1];
    __shared__ float tau_s[NB];

    const int row_base = crank * chunk;
    const int row_end = min(row_base + chunk, L);
    const uint32_t msg_bytes = (uint32_t)(cs * MSG * sizeof(float));
    bool timed_out = false;
    for (int e = tid; e < NB * (NB + 1); e += NT) (&G_s[0][0])[e] = 0.f;
    if (cs > 1) {
        if (tid == 0) {
            asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(pq_smem(&mbar[0])) : "memory");
            asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(pq_smem(&mbar[1])) : "memory");
            asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
            pq_expect_tx(pq_smem(&mbar[0]), msg_bytes);        // round 0
        }
        cluster.sync();
    }
    int rr[RPT];
    float a[RPT][NB];
#pragma unroll
    for (int q = 0; q < RPT; q++) {
        const int r = row_base + tid + q * NT;
        rr[q] = r < row_end ? r : -1;
    }
#pragma unroll
    for (int c = 0; c < NB; c++) {
        const float *col = A + idx2(j0, j0 + c, lda);
#pragma unroll
        for (int q = 0; q < RPT; q++) a[q][c] = (rr[q] >= 0 && c < ncols) ? col[rr[q]] : 0.f;
    }

    int rnd = 0;
#pragma unroll 1
    for (int kk = 0; kk < kpanel; rnd++) {
        const int par = rnd & 1;
        const bool two = kk + 1 < kpanel;
        const int kb = two ? kk + 1 : kk;                 // the sums run over rows below kb
        float ak1[RPT], ak2[RPT];
#pragma unroll
        for (int q = 0; q < RPT; q++) {
            ak1[q] = pq_select<float, NB>(a[q], kk);
            ak2[q] = two ? pq_select<float, NB>(a[q], kk + 1) : 0.f;
        }
#pragma unroll
        for (int h0 = 0; h0 < NB; h0 += H) {
            float acc1[H], acc2[H];
#pragma unroll
            for (int c = 0; c < H; c++) { acc1[c] = 0.f; acc2[c] = 0.f; }
#pragma unroll
            for (int q = 0; q < RPT; q++) {
                const bool bel = rr[q] > kb;
                const float x1 = bel ? ak1[q] : 0.f, x2 = bel ? ak2[q] : 0.f;
#pragma unroll
                for (int c = 0; c < H; c++) {
                    acc1[c] = fmaf(x1, a[q][h0 + c], acc1[c]);
                    acc2[c] = fmaf(x2, a[q][h0 + c], acc2[c]);
                }
            }
            const float w1 = warp_transpose_reduce<float, H>(acc1);
            const float w2 = warp_transpose_reduce<float, H>(acc2);
            if (lane < H) {
                red_s[par][warp][h0 + lane] = w1;
                red_s[par][warp][NB + h0 + lane] = w2;
            }
        }
#pragma unroll
        for (int q = 0; q < RPT; q++) {
            if (rr[q] == kk) {
#pragma unroll
                for (int c = 0; c < NB; c++) prow[par][0][c] = a[q][c];
            }
            if (two && rr[q] == kk + 1) {
#pragma unroll
                for (int c = 0; c < NB; c++) prow[par][1][c] = a[q][c];
            }
        }
        // a next round exists whenever a column follows kk (if this round
        // takes two columns and none is left, the count is never used)
        if (cs > 1 && tid == 0 && kk + 1 < kpanel) pq_expect_tx(pq_smem(&mbar[par ^ 1]), msg_bytes);
        __syncthreads();
        float tot1 = 0.f, tot2 = 0.f, pj1 = 0.f, pj2 = 0.f;
        if (cs == 1) {
#pragma unroll
            for (int w = 0; w < NW; w++) { tot1 += red_s[par][w][lane]; tot2 += red_s[par][w][NB + lane]; }
            pj1 = prow[par][0][lane];
            pj2 = two ? prow[par][1][lane] : 0.f;
        } else {
            {
                float t1 = 0.f, t2 = 0.f;
#pragma unroll
                for (int w = 0; w < NW; w++) { t1 += red_s[par][w][lane]; t2 += red_s[par][w][NB + lane]; }
                xbuf[warp][lane] = t1;
                xbuf[warp][NB + lane] = t2;
                xbuf[warp][2 * NB + lane] = crank == 0 ? prow[par][0][lane] : 0.f;
                xbuf[warp][3 * NB + lane] = (crank == 0 && two) ? prow[par][1][lane] : 0.f;
            }
            __syncwarp();
            {
                const float4 v = reinterpret_cast<const float4 *>(&xbuf[warp][0])[lane];
                const uint32_t dst = pq_smem(&gbuf[par][crank][0]) + 16 * lane;
                const uint32_t bar = pq_smem(&mbar[par]);
                for (int q = warp; q < cs; q += NW) pq_st_async(pq_mapa(dst, q), v, pq_mapa(bar, q));
            }
            if (!timed_out && !pq_wait(pq_smem(&mbar[par]), (uint32_t)(rnd >> 1) & 1u)) timed_out = true;
            for (int q = 0; q < cs; q++) {
                tot1 += gbuf[par][q][lane];
                tot2 += gbuf[par][q][NB + lane];
                pj1 += gbuf[par][q][2 * NB + lane];
                pj2 += gbuf[par][q][3 * NB + lane];
            }
        }
        // reflector kk (row kk+1 added back to its sums)
        const float alpha1 = __shfl_sync(0xffffffffu, pj1, kk);
        const float pk1 = __shfl_sync(0xffffffffu, pj2, kk);          // a(kk+1, kk); 0 without a pair
        const float sp1 = fmaf(pk1, pk1, __shfl_sync(0xffffffffu, tot1, kk));
        float tau1, beta1, scale1;
        pair_reflector(alpha1, sp1, tau1, beta1, scale1);
        const float dot1 = fmaf(scale1, fmaf(pk1, pj2, tot1), pj1);
        const float coef1 = lane > kk ? tau1 * dot1 : 0.f;
        // reflector kk+1 from the downdated sums
        const int k2 = two ? kk + 1 : kk;
        const float gc = coef1 * scale1;
        const float g = __shfl_sync(0xffffffffu, gc, k2);
        const float T11 = __shfl_sync(0xffffffffu, tot1, kk);
        const float T12 = __shfl_sync(0xffffffffu, tot1, k2);
        const float T22 = __shfl_sync(0xffffffffu, tot2, k2);
        const float sp2 = fmaf(g, fmaf(g, T11, -2.f * T12), T22);
        const bool pair = two && sp2 >= 0.f && sp2 >= PAIR_GUARD * T22;
        const float p2n = lane == kk ? scale1 * pk1 : (lane > kk ? fmaf(-gc, pk1, pj2) : pj2);
        float tau2 = 0.f, beta2 = 0.f, scale2 = 0.f, dot2 = 0.f;
        if (pair) {
            pair_reflector(__shfl_sync(0xffffffffu, p2n, k2), sp2, tau2, beta2, scale2);
            float X;
            if (lane < kk) X = fmaf(-g, tot1, tot2);
            else if (lane == kk) X = scale1 * fmaf(-g, T11, T12);
            else X = fmaf(g * gc, T11, fmaf(-g, tot1, fmaf(-gc, T12, tot2)));
            dot2 = fmaf(scale2, X, p2n);
        }
        const float coef2 = (pair && lane > k2) ? tau2 * dot2 : 0.f;
        coefw[warp][0][lane] = coef1;
        coefw[warp][1][lane] = coef2;
        if (warp == 0) {
            if (lane < kk) G_s[lane][kk] = dot1;
            if (pair && lane < k2) G_s[lane][k2] = dot2;
            if (lane == 0) {
                tau_s[kk] = tau1;
                if (pair) tau_s[k2] = tau2;
            }
        }
        __syncwarp();
        const float c1k2 = __shfl_sync(0xffffffffu, coef1, k2);        // coefficient of column kk+1
        // branch-free updates of the owned rows: reflector kk, then kk+1
#pragma unroll
        for (int q = 0; q < RPT; q++) {
            const bool below1 = rr[q] > kk, piv1 = rr[q] == kk;
            const float s1 = ak1[q] * scale1;
            const float f1 = below1 ? s1 : (piv1 ? 1.f : 0.f);
            const float nk1 = below1 ? s1 : (piv1 ? beta1 : ak1[q]);
            const float a2 = fmaf(-c1k2, f1, ak2[q]);                  // a(i, kk+1) after reflector kk
            const bool below2 = rr[q] > k2, piv2 = rr[q] == k2;
            const float s2 = a2 * scale2;
            const float f2 = pair ? (below2 ? s2 : (piv2 ? 1.f : 0.f)) : 0.f;
            const float nk2 = below2 ? s2 : (piv2 ? beta2 : a2);
#pragma unroll
            for (int g8 = 0; g8 < NB; g8 += 8) {
                if (g8 + 7 >= kk) {
#pragma unroll
                    for (int c = g8; c < g8 + 8; c++) {
                        float x = fmaf(-coefw[warp][0][c], f1, a[q][c]);
                        x = (c == kk) ? nk1 : x;
                        x = fmaf(-coefw[warp][1][c], f2, x);
                        a[q][c] = (pair && c == k2) ? nk2 : x;
                    }
                }
            }
        }
        kk += pair ? 2 : 1;
    }
    __syncthreads();

    float *Aw = A;
    asm volatile("" : "+l"(Aw));
#pragma unroll
    for (int c = 0; c < NB; c++) {
        if (c < ncols) {
            float *col = Aw + idx2(j0, j0 + c, lda);
#pragma unroll
            for (int q = 0; q < RPT; q++)
                if (rr[q] >= 0) col[rr[q]] = a[q][c];
        }
    }
    if (crank == 0 && warp == 0) {
        if (lane < kpanel) tau[j0 + lane] = tau_s[lane];
        panel_T_from_gram<float, NB, NB + 1>(G_s, tau_s, kpanel, Tw);
    }
    if (timed_out) atomicOr(err, 8);
    if (cs > 1) cluster.sync();
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

// ---------------------------------------------------------------------------
// Row-parallel inner update (within a 128-wide outer block): the trailing
// columns of the outer block are few (<= 96) but the panel is tall, so the
// work is split over row chunks:
//   k_inner_w      P[chunk] = V_chunk^T C_chunk             (32 x nc)
//   k_inner_reduce W = Tw^T sum_chunk P[chunk]
//   k_inner_update C_chunk -= V_chunk W
// V is the unit lower trapezoid stored in the panel columns.
// ---------------------------------------------------------------------------
constexpr int INNER_ROWS = 256;
constexpr int INNER_MAXC = 96;

template <typename T, int NB>
__global__ void __launch_bounds__(256)
k_inner_w(const T *__restrict__ V, int ldv, int kb, int L, const T *__restrict__ C, int ldc, int nc,
          T *__restrict__ P)
{
    __shared__ T Vs[32][NB + 1];
    __shared__ T Cs[32][INNER_MAXC + 1];
    const int tid = threadIdx.x;
    const int r0 = blockIdx.x * INNER_ROWS;
    // thread owns outputs (i, c) with i = tid % NB, c = tid / NB + 256/NB * s
    constexpr int CSTEP = 256 / NB;
    constexpr int NOUT = (INNER_MAXC + CSTEP - 1) / CSTEP;
    T acc[NOUT];
#pragma unroll
    for (int s = 0; s < NOUT; s++) acc[s] = T(0);
    const int i = tid % NB, cb = tid / NB;
    for (int rr = 0; rr < INNER_ROWS; rr += 32) {
        for (int e = tid; e < 32 * NB; e += 256) {
            const int r = e % 32, c = e / 32, gr = r0 + rr + r;
            T v = T(0);
            if (gr < L && c < kb) v = gr > c ? V[idx2(gr, c, ldv)] : (gr == c ? T(1) : T(0));
            Vs[r][c] = v;
        }
        for (int e = tid; e < 32 * nc; e += 256) {
            const int r = e % 32, c = e / 32, gr = r0 + rr + r;
            Cs[r][c] = gr < L ? C[idx2(gr, c, ldc)] : T(0);
        }
        __syncthreads();
#pragma unroll 4
        for (int r = 0; r < 32; r++) {
            const T v = Vs[r][i];
#pragma unroll
            for (int s = 0; s < NOUT; s++) {
                const int c = cb + CSTEP * s;
                if (c < nc) acc[s] = fma(v, Cs[r][c], acc[s]);
            }
        }
        __syncthreads();
    }
    T *Pc = P + (size_t)blockIdx.x * NB * INNER_MAXC;
#pragma unroll
    for (int s = 0; s < NOUT; s++) {
        const int c = cb + CSTEP * s;
        if (c < nc) Pc[i + c * NB] = acc[s];
    }
}

template <typename T, int NB>
__global__ void __launch_bounds__(256)
k_inner_reduce(const T *__restrict__ P, int nchunks, const T *__restrict__ Tw, int nc, int trans,
               T *__restrict__ W)
{
    __shared__ T S[NB][INNER_MAXC + 1];
    __shared__ T X[NB][NB + 1];
    const int tid = threadIdx.x;
    for (int e = tid; e < NB * nc; e += 256) {
        const int i = e % NB, c = e / NB;
        T s = T(0);
        for (int k = 0; k < nchunks; k++) s += P[(size_t)k * NB * INNER_MAXC + i + c * NB];
        S[i][c] = s;
    }
    for (int e = tid; e < NB * NB; e += 256) {
        const int i = e % NB, k = e / NB;
        const T t = Tw[i + k * NB];
        if (trans) X[k][i] = t; else X[i][k] = t;
    }
    __syncthreads();
    for (int e = tid; e < NB * nc; e += 256) {
        const int i = e % NB, c = e / NB;
        T s = T(0);
        for (int k = 0; k < NB; k++) s = fma(X[i][k], S[k][c], s);
        W[i + c * NB] = s;
    }
}

template <typename T, int NB>
__global__ void __launch_bounds__(256)
k_inner_update(const T *__restrict__ V, int ldv, int kb, int L, T *__restrict__ C, int ldc, int nc,
               const T *__restrict__ W)
{
    __shared__ T Ws[NB][INNER_MAXC + 1];
    __shared__ T Vs[32][NB + 1];
    const int tid = threadIdx.x;
    for (int e = tid; e < NB * nc; e += 256) Ws[e % NB][e / NB] = W[e];
    const int r0 = blockIdx.x * INNER_ROWS;
    const int lr = tid & 31, cg0 = tid >> 5;     // 8 column groups
    for (int rr = 0; rr < INNER_ROWS; rr += 32) {
        __syncthreads();
        for (int e = tid; e < 32 * NB; e += 256) {
            const int r = e % 32, c = e / 32, gr = r0 + rr + r;
            T v = T(0);
            if (gr < L && c < kb) v = gr > c ? V[idx2(gr, c, ldv)] : (gr == c ? T(1) : T(0));
            Vs[r][c] = v;
        }
        __syncthreads();
        const int gr = r0 + rr + lr;
        if (gr < L) {
            for (int c = cg0; c < nc; c += 8) {
                T t = T(0);
#pragma unroll 8
                for (int k = 0; k < NB; k++) t = fma(Vs[lr][k], Ws[k][c], t);
                C[idx2(gr, c, ldc)] -= t;
            }
        }
    }
}

// Fused inner update on one thread-block cluster: CTA r owns rows
// [r*chunk, (r+1)*chunk); partial V^T C over its rows, a DSMEM sum over the
// cluster (rank order, identical on every CTA), W = Tw^T S, then
// C -= V W on its rows.  One launch and one cluster barrier per update.
template <int NB>
__global__ void __launch_bounds__(256, 1)
k_inner_cl(const float *__restrict__ V, int ldv, int kb, int L, float *__restrict__ C, int ldc, int nc,
           const float *__restrict__ Tw, int chunk)
{
    __shared__ float Vs[32][NB + 1];
    __shared__ float Cs[32][INNER_MAXC + 1];      // C staging, later the reduced S = V^T C
    __shared__ float pw[NB * INNER_MAXC];         // this CTA's partial, read remotely
    __shared__ float Wt[NB][INNER_MAXC + 1];
    __shared__ float Xs[NB][NB + 1];
    cg::cluster_group cluster = cg::this_cluster();
    const int cs = (int)cluster.num_blocks();
    const int crank = (int)cluster.block_rank();
    const int tid = threadIdx.x;
    const int r0 = crank * chunk, r1 = min(r0 + chunk, L);
    constexpr int CSTEP = 256 / NB;
    constexpr int NOUT = (INNER_MAXC + CSTEP - 1) / CSTEP;
    const int i = tid % NB, cb = tid / NB;
    float acc[NOUT];
#pragma unroll
    for (int q = 0; q < NOUT; q++) acc[q] = 0.f;
    for (int rr = r0; rr < r1; rr += 32) {
        for (int e = tid; e < 32 * NB; e += 256) {
            const int r = e % 32, c = e / 32, gr = rr + r;
            float v = 0.f;
            if (gr < r1 && c < kb) v = gr > c ? V[idx2(gr, c, ldv)] : (gr == c ? 1.f : 0.f);
            Vs[r][c] = v;
        }
        for (int e = tid; e < 32 * nc; e += 256) {
            const int r = e % 32, c = e / 32, gr = rr + r;
            Cs[r][c] = gr < r1 ? C[idx2(gr, c, ldc)] : 0.f;
        }
        __syncthreads();
#pragma unroll 4
        for (int r = 0; r < 32; r++) {
            const float v = Vs[r][i];
#pragma unroll
            for (int q = 0; q < NOUT; q++) {
                const int c = cb + CSTEP * q;
                if (c < nc) acc[q] = fmaf(v, Cs[r][c], acc[q]);
            }
        }
        __syncthreads();
    }
#pragma unroll
    for (int q = 0; q < NOUT; q++) {
        const int c = cb + CSTEP * q;
        if (c < nc) pw[i + c * NB] = acc[q];
    }
    for (int e = tid; e < NB * NB; e += 256) {
        const int a = e % NB, k = e / NB;
        Xs[k][a] = Tw[a + k * NB];                // X = Tw^T
    }
    cluster.sync();
    for (int e = tid; e < NB * nc; e += 256) {
        float sum = 0.f;
        for (int r = 0; r < cs; r++) sum += *cluster.map_shared_rank(&pw[e], r);
        Cs[e % NB][e / NB] = sum;
    }
    __syncthreads();
    for (int e = tid; e < NB * nc; e += 256) {
        const int a = e % NB, c = e / NB;
        float sum = 0.f;
#pragma unroll 8
        for (int k = 0; k < NB; k++) sum = fmaf(Xs[a][k], Cs[k][c], sum);
        Wt[a][c] = sum;
    }
    __syncthreads();
    const int lr = tid & 31, cg0 = tid >> 5;
    for (int rr = r0; rr < r1; rr += 32) {
        __syncthreads();
        for (int e = tid; e < 32 * NB; e += 256) {
            const int r = e % 32, c = e / 32, gr = rr + r;
            float v = 0.f;
            if (gr < r1 && c < kb) v = gr > c ? V[idx2(gr, c, ldv)] : (gr == c ? 1.f : 0.f);
            Vs[r][c] = v;
        }
        __syncthreads();
        const int gr = rr + lr;
        if (gr < r1) {
            for (int c = cg0; c < nc; c += 8) {
                float t = 0.f;
#pragma unroll 8
                for (int k = 0; k < NB; k++) t = fmaf(Vs[lr][k], Wt[k][c], t);
                C[idx2(gr, c, ldc)] -= t;
            }
        }
    }
    cluster.sync();   // pw must outlive the remote reads
}

// ---------------------------------------------------------------------------
// Outer (128-reflector) blocks, FP32 storage.
//
// Nearest TF32 value (the tensor cores read only a TF32 operand's top 19 bits;
// rounding the low part of a hi/lo split, instead of letting the hardware
// truncate it, halves the split's representation error to 2^-22 |a|).
__device__ __forceinline__ float tf32_rn(float x)
{
    uint32_t u;
    asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(u) : "f"(x));
    return __uint_as_float(u);
}

// k_prep_v: the unit lower trapezoid V of an outer block (rows j0.., columns
// j0..j0+nr) in the layouts the tensor-core GEMMs read:
//   V, Vlo   L x 128 column-major (ld ldv)  -- A operand of W = V^T C
//   Vt, Vtlo 128 x L column-major (ld 128)  -- A operand of C -= V W
// with V = Vhi + Vlo, Vhi = TF32(V) when split (TF32X3), else V raw.
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(256)
k_prep_v(const float *__restrict__ X, int ldx, int L, int nr, float *__restrict__ Vh, float *__restrict__ Vl,
         int ldv, float *__restrict__ Vth, float *__restrict__ Vtl, int split)
{
    pdl_wait();
    pdl_trigger();
    __shared__ float tile[32][OUTER_NB + 1];
    const int r0 = blockIdx.x * 32;
    const int tid = threadIdx.x;
    for (int e = tid; e < 32 * OUTER_NB; e += 256) {
        const int r = e % 32, c = e / 32, gr = r0 + r;
        float v = 0.f;
        if (gr < L && c < nr) v = gr > c ? X[idx2(gr, c, ldx)] : (gr == c ? 1.f : 0.f);
        tile[r][c] = v;
    }
    __syncthreads();
    // V / Vlo: column-major, coalesced along rows
    for (int e = tid; e < 32 * OUTER_NB; e += 256) {
        const int r = e % 32, c = e / 32, gr = r0 + r;
        if (gr < ldv) {
            const float v = tile[r][c];
            float h = v;
            if (split) { uint32_t u; asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(u) : "f"(v)); h = __uint_as_float(u); }
            Vh[idx2(gr, c, ldv)] = h;
            if (split) Vl[idx2(gr, c, ldv)] = tf32_rn(v - h);
        }
    }
    // Vt / Vtlo: 128 x L, coalesced along the 128 columns of V
    for (int e = tid; e < 32 * OUTER_NB; e += 256) {
        const int c = e % OUTER_NB, r = e / OUTER_NB, gr = r0 + r;
        if (gr < ldv) {
            const float v = tile[r][c];
            float h = v;
            if (split) { uint32_t u; asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(u) : "f"(v)); h = __uint_as_float(u); }
            Vth[idx2(c, gr, OUTER_NB)] = h;
            if (split) Vtl[idx2(c, gr, OUTER_NB)] = tf32_rn(v - h);
        }
    }
}

// W = op(Tb) * sum_z P[z] (128 x nc), op = Tb^T (trans), Tb, or identity
// (Tb == NULL); optionally split into W = Wh + Wl.  One block per 16 columns.
template <int RW_COLS>
__global__ void __launch_bounds__(256)
k_reduce_w(const float *__restrict__ P, int nsplit, size_t pstride, int ldp, const float *__restrict__ Tb,
           int trans, int nc, float *__restrict__ Wh, float *__restrict__ Wl, int ldw, int split)
{
    pdl_wait();
    pdl_trigger();
    extern __shared__ float sm[];
    constexpr int LDX = OUTER_NB + 1;                // odd stride: the transposed stores hit 32 banks
    float *S = sm;                                   // 128 x RW_COLS, column-major
    float *Xs = sm + RW_COLS * OUTER_NB;             // 128 x 128 (x(i,k) at i + LDX k)
    const int tid = threadIdx.x;
    const int c0 = blockIdx.x * RW_COLS;
    if (Tb) {
        for (int e = tid; e < OUTER_NB * OUTER_NB; e += 256) {
            const int i = e % OUTER_NB, k = e / OUTER_NB;
            const float t = Tb[i + k * OUTER_NB];
            if (trans) Xs[k + i * LDX] = t; else Xs[i + k * LDX] = t;
        }
    }
    for (int e = tid; e < RW_COLS * OUTER_NB; e += 256) {
        const int i = e % OUTER_NB, c = e / OUTER_NB;
        float s = 0.f;
        if (c0 + c < nc) {
            const float *pp = P + (size_t)(c0 + c) * ldp + i;
            int z = 0;
            for (; z + 8 <= nsplit; z += 8) {
                float a[8];
#pragma unroll
                for (int u = 0; u < 8; u++) a[u] = pp[(size_t)(z + u) * pstride];
#pragma unroll
                for (int u = 0; u < 8; u++) s += a[u];
            }
            for (; z < nsplit; z++) s += pp[(size_t)z * pstride];
        }
        S[i + c * OUTER_NB] = s;
    }
    __syncthreads();
    for (int e = tid; e < RW_COLS * OUTER_NB; e += 256) {
        const int i = e % OUTER_NB, c = e / OUTER_NB;
        if (c0 + c >= nc) continue;
        float w;
        if (Tb) {
            float s0 = 0.f, s1 = 0.f, s2 = 0.f, s3 = 0.f;
#pragma unroll 8
            for (int k = 0; k < OUTER_NB; k += 4) {
                s0 = fmaf(Xs[i + k * LDX], S[k + c * OUTER_NB], s0);
                s1 = fmaf(Xs[i + (k + 1) * LDX], S[k + 1 + c * OUTER_NB], s1);
                s2 = fmaf(Xs[i + (k + 2) * LDX], S[k + 2 + c * OUTER_NB], s2);
                s3 = fmaf(Xs[i + (k + 3) * LDX], S[k + 3 + c * OUTER_NB], s3);
            }
            w = (s0 + s1) + (s2 + s3);
        } else {
            w = S[i + c * OUTER_NB];
        }
        float h = w;
        if (split) { uint32_t u; asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(u) : "f"(w)); h = __uint_as_float(u); }
        Wh[(size_t)(c0 + c) * ldw + i] = h;
        if (split) Wl[(size_t)(c0 + c) * ldw + i] = tf32_rn(w - h);
    }
}

// W = op(Tb) sum_z P[z] (or the plain sum when Tb is null) over nc columns:
// 16 columns per CTA, 4 when that would leave the grid small.
static void reduce_w(const float *P, int nsplit, size_t pstride, const float *Tb, int trans, int nc, float *Wh,
                     float *Wl, int ldw, int split, cudaStream_t s)
{
    if (nc >= 16 * 64) {
        const size_t smem = ((size_t)16 * OUTER_NB + (size_t)(OUTER_NB + 1) * OUTER_NB) * 4;
        static PerDeviceOnce once;
        once([&] { cudaFuncSetAttribute(k_reduce_w<16>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem); });
        pdl_launch(k_reduce_w<16>, dim3(ceil_div(nc, 16)), dim3(256), smem, s, P, nsplit, pstride, (int)OUTER_NB, Tb, trans,
                   nc, Wh, Wl, ldw, split);
    } else {
        const size_t smem = ((size_t)4 * OUTER_NB + (size_t)(OUTER_NB + 1) * OUTER_NB) * 4;
        static PerDeviceOnce once;
        once([&] { cudaFuncSetAttribute(k_reduce_w<4>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem); });
        pdl_launch(k_reduce_w<4>, dim3(ceil_div(nc, 4)), dim3(256), smem, s, P, nsplit, pstride, (int)OUTER_NB, Tb, trans,
                   nc, Wh, Wl, ldw, split);
    }
}

// out[e] = sum_z P[z * pstride + e] in split order, one element per thread.
__global__ void __launch_bounds__(256)
k_sum_splits(const float *__restrict__ P, int nsplit, size_t pstride, int n, float *__restrict__ out)
{
    pdl_wait();
    pdl_trigger();
    const int e = blockIdx.x * 256 + threadIdx.x;
    if (e >= n) return;
    float v[8];
    float sum = 0.f;
    int z = 0;
    for (; z + 8 <= nsplit; z += 8) {
#pragma unroll
        for (int u = 0; u < 8; u++) v[u] = P[(size_t)(z + u) * pstride + e];
#pragma unroll
        for (int u = 0; u < 8; u++) sum += v[u];
    }
    for (; z < nsplit; z++) sum += P[(size_t)z * pstride + e];
    out[e] = sum;
}

// Compact-WY factor of an outer block from its four 32-wide inner factors
// and the Gram matrix G = V^T V (Tw^{-1} = triu(G, 1) + diag(1/tau)):
//   T(0:32j, 32j:32j+32) = -T(0:32j, 0:32j) G(0:32j, 32j:32j+32) T_j.
__global__ void __launch_bounds__(256, 1)
k_outer_T(const float *__restrict__ Tw32, const float *__restrict__ G, int nr, float *__restrict__ Tb)
{
    pdl_wait();
    pdl_trigger();
    extern __shared__ float sm[];
    float *Ts = sm;                                  // 128 x 128 column-major
    float *Pm = sm + OUTER_NB * OUTER_NB;            // 96 x 32 scratch
    float *Gs = Pm + 96 * 32;                        // G staged, 128 x 128
    const int tid = threadIdx.x;
    for (int e = tid; e < OUTER_NB * OUTER_NB; e += 256) { Ts[e] = 0.f; Gs[e] = G[e]; }
    __syncthreads();
    const int nblk = ceil_div(nr, 32);
    for (int b = 0; b < nblk; b++)
        for (int e = tid; e < 32 * 32; e += 256) {
            const int ii = e & 31, k = e >> 5;
            Ts[(32 * b + ii) + (32 * b + k) * OUTER_NB] = Tw32[(size_t)b * 1024 + ii + k * 32];
        }
    __syncthreads();
    // thread (row i = tid % 128, 16-column half ch = tid / 128): 16
    // independent accumulators per product, no index division
    const int i = tid & (OUTER_NB - 1), ch = tid >> 7;
    for (int j = 1; j < nblk; j++) {
        const int h = 32 * j;
        // Pm = G(0:h, h:h+32) * T_j
        if (i < h) {
            float acc[16];
#pragma unroll
            for (int c = 0; c < 16; c++) acc[c] = 0.f;
#pragma unroll 4
            for (int k = 0; k < 32; k++) {
                const float g = Gs[i + (h + k) * OUTER_NB];
#pragma unroll
                for (int c = 0; c < 16; c++)
                    acc[c] = fmaf(g, Ts[(h + k) + (h + 16 * ch + c) * OUTER_NB], acc[c]);
            }
#pragma unroll
            for (int c = 0; c < 16; c++) Pm[i + (16 * ch + c) * 96] = acc[c];
        }
        __syncthreads();
        // T(0:h, h:h+32) = -T(0:h, 0:h) * Pm   (T upper triangular)
        if (i < h) {
            float acc[16];
#pragma unroll
            for (int c = 0; c < 16; c++) acc[c] = 0.f;
#pragma unroll 4
            for (int k = i; k < h; k++) {
                const float t = Ts[i + k * OUTER_NB];
#pragma unroll
                for (int c = 0; c < 16; c++) acc[c] = fmaf(t, Pm[k + (16 * ch + c) * 96], acc[c]);
            }
#pragma unroll
            for (int c = 0; c < 16; c++) Ts[i + (h + 16 * ch + c) * OUTER_NB] = -acc[c];
        }
        __syncthreads();
    }
    for (int e = tid; e < OUTER_NB * OUTER_NB; e += 256) Tb[e] = Ts[e];
}

// ------------------------------------------------------------------ host --

template <typename T, int NT, int RPT>
static int launch_panel_shape(T *A, int lda, int M, int j0, int ncols, T *tau, T *Tw, int *err, cudaStream_t s)
{
    constexpr int NB = panel_nb<T>();
    const int L = M - j0;
    int cs = ceil_div(L, NT * RPT);
    if (cs < 1) cs = 1;
    if (cs > PANEL_MAX_CLUSTER) return MPIR_UNSUP();
    const int chunk = ceil_div(L, cs);
    auto kern = k_panel_qr<T, NB, NT, RPT>;
    static PerDeviceOnce once;
    once([&] { cudaFuncSetAttribute(kern, cudaFuncAttributeNonPortableClusterSizeAllowed, 1); });
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(cs, 1, 1);
    cfg.blockDim = dim3(NT, 1, 1);
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
    cudaError_t e = cudaLaunchKernelEx(&cfg, kern, A, lda, M, j0, ncols, chunk, tau, Tw, err);
    return e == cudaSuccess ? 0 : MPIR_CUDA_ERROR;
}

template <int NT, int RPT>
static int launch_panel_pair(float *A, int lda, int M, int j0, int ncols, float *tau, float *Tw, int *err,
                             cudaStream_t s)
{
    const int L = M - j0;
    int cs = ceil_div(L, NT * RPT);
    if (cs < 1) cs = 1;
    if (cs > PANEL_MAX_CLUSTER) return MPIR_UNSUP();
    const int chunk = ceil_div(L, cs);
    auto kern = k_panel_qr_pair<NT, RPT>;
    static PerDeviceOnce once;
    once([&] { cudaFuncSetAttribute(kern, cudaFuncAttributeNonPortableClusterSizeAllowed, 1); });
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(cs, 1, 1);
    cfg.blockDim = dim3(NT, 1, 1);
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
    cudaError_t e = cudaLaunchKernelEx(&cfg, kern, A, lda, M, j0, ncols, chunk, tau, Tw, err);
    return e == cudaSuccess ? 0 : MPIR_CUDA_ERROR;
}

template <typename T, int NT, int RPT>
static int launch_panel_grid(T *A, int lda, int M, int j0, int ncols, T *tau, T *Tw, int *err, const PanelGrid &pg,
                             cudaStream_t s)
{
    constexpr int NB = panel_nb<T>();
    int L = M - j0;
    int G = ceil_div(L, NT * RPT);
    if (G < 1) G = 1;
    if (!pg.gx || !pg.bar || G > PANEL_GRID_MAX) return MPIR_UNSUP();
    auto kern = k_panel_qr_grid<T, NB, NT, RPT>;
    int per_sm = 0, dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, NT, 0) != cudaSuccess) {
        cudaGetLastError();
        return MPIR_UNSUP();
    }
    if (per_sm * sms < G) return MPIR_UNSUP();      // every CTA must be resident (grid barrier)
    int chunk = ceil_div(L, G);
    GridBarrier gb{pg.bar, err};
    T *gx = reinterpret_cast<T *>(pg.gx);
    void *args[] = {&A, &lda, &M, &j0, &ncols, &chunk, &tau, &Tw, &err, &gx, &gb};
    ProfScope ps(K_PANEL, s);
    cudaError_t e = cudaLaunchCooperativeKernel((const void *)kern, dim3(G), dim3(NT), args, 0, s);
    return e == cudaSuccess ? 0 : MPIR_CUDA_ERROR;
}

template <int NT>
static int launch_panel2(float *A, int lda, int M, int j0, int ncols, float *tau, float *Tw, int *err, cudaStream_t s)
{
    const int L = M - j0;
    int cs = ceil_div(L, NT / 2);
    if (cs < 1) cs = 1;
    if (cs > PANEL_MAX_CLUSTER) return MPIR_UNSUP();
    const int chunk = ceil_div(L, cs);
    auto kern = k_panel_qr2<NT>;
    static PerDeviceOnce once;
    once([&] { cudaFuncSetAttribute(kern, cudaFuncAttributeNonPortableClusterSizeAllowed, 1); });
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(cs, 1, 1);
    cfg.blockDim = dim3(NT, 1, 1);
    cfg.dynamicSmemBytes = 0;
    cfg.stream = s;
    cudaLaunchAttribute attr[2];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = cs;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    attr[1].id = cudaLaunchAttributeProgrammaticStreamSerialization;   // waits in-kernel
    attr[1].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 2;
    ProfScope ps(K_PANEL, s);
    cudaError_t e = cudaLaunchKernelEx(&cfg, kern, A, lda, M, j0, ncols, chunk, tau, Tw, err);
    return e == cudaSuccess ? 0 : MPIR_CUDA_ERROR;
}

// Rows per CTA as small as the 16-CTA cluster limit allows: the panel's
// column steps are latency and issue bound, so fewer rows per SM (more SMs)
// shorten every step.  FP32 panels of up to 4096 rows hold two threads per
// row.
// Panels beyond what 16 CTAs hold (pg: the exchange buffers of the
// global-memory variant) run on one CTA per 1024 rows with a grid barrier.
template <typename T>
static int launch_panel(T *A, int lda, int M, int j0, int ncols, T *tau, T *Tw, int *err, cudaStream_t s,
                        const PanelGrid *pg = nullptr)
{
    const int L = M - j0;
    if constexpr (sizeof(T) == 4) {
        if (L <= 16 * 64) return launch_panel2<128>(A, lda, M, j0, ncols, tau, Tw, err, s);
        if (L <= 16 * 128) return launch_panel2<256>(A, lda, M, j0, ncols, tau, Tw, err, s);
        if (L <= 16 * 256) return launch_panel2<512>(A, lda, M, j0, ncols, tau, Tw, err, s);
        // taller panels: one message round per column pair
        if (L <= 16 * 512) return launch_panel_pair<512, 1>(A, lda, M, j0, ncols, tau, Tw, err, s);
        if (L <= 16 * 1024 || !pg) return launch_panel_pair<512, 2>(A, lda, M, j0, ncols, tau, Tw, err, s);
        return launch_panel_grid<float, 512, 2>(A, lda, M, j0, ncols, tau, Tw, err, *pg, s);
    }
    if (L <= PANEL_MAX_CLUSTER * PANEL_NT * PANEL_RPT || !pg)
        return launch_panel_shape<T, PANEL_NT, PANEL_RPT>(A, lda, M, j0, ncols, tau, Tw, err, s);
    return launch_panel_grid<T, PANEL_NT, PANEL_RPT>(A, lda, M, j0, ncols, tau, Tw, err, *pg, s);
}

// Inner update with the CTA's whole row chunk of V and of a 32-column group
// of C staged in shared memory: partial S = V^T C, DSMEM sum over the
// cluster, W = Tw^T S, C -= V W in shared memory, one coalesced write-back.
// Column groups are independent (grid y, one cluster each), so an update of
// nc columns spans ceil(nc / 32) clusters.  V is staged row-major (rows of
// 36 floats: 16-byte vectors, distinct banks per quarter warp), C
// column-major with an odd leading dimension rp.  S is register-blocked in
// 4 x 4 tiles over four row groups (one vector load of V and four loads of C
// per 16 FMAs), summed over the groups in shared memory; the update is one
// row per thread with W^T rows read as broadcast vectors.
constexpr int IV_LD = 36;
constexpr int IC = 32;                             // columns per cluster

template <int NB>
__global__ void __launch_bounds__(256, 1)
k_inner_cl_s(const float *__restrict__ V, int ldv, int kb, int L, float *__restrict__ C, int ldc, int nc,
             const float *__restrict__ Tw, int chunk, int rp)
{
    static_assert(NB == 32, "32-wide panels");
    extern __shared__ __align__(16) float sm[];
    float *Vc = sm;                                    // chunk x IV_LD, row-major
    float *Cc = Vc + (size_t)chunk * IV_LD;            // IC x rp, column-major
    __shared__ __align__(16) float pg[4][IC * NB];     // row-group partials, [c][i]
    __shared__ __align__(16) float pw[IC * NB];        // this CTA's partial S, read remotely
    __shared__ __align__(16) float Sx[IC * NB];        // cluster sum
    __shared__ __align__(16) float Wc[IC * IV_LD];     // W^T rows: Wc[c][k] = W(k, c)
    __shared__ float Xs[NB][NB + 1];                   // Xs[a][k] = Tw(k, a)
    cg::cluster_group cluster = cg::this_cluster();
    const int cs = (int)cluster.num_blocks();
    const int crank = (int)cluster.block_rank();
    const int tid = threadIdx.x;
    const int cg0 = blockIdx.y * IC;
    const int ncl = min(IC, nc - cg0);                 // columns of this group
    C += (size_t)cg0 * ldc;
    const int r0 = crank * chunk, r1 = min(r0 + chunk, L), R = max(0, r1 - r0);
    pdl_wait();                                         // previous kernel's results
    pdl_trigger();
    // staging: rows over threads, columns unrolled (no index division)
    for (int r = tid; r < R; r += 256) {
        const int gr = r0 + r;
        float v[NB], cv[IC];
#pragma unroll
        for (int c = 0; c < NB; c++) v[c] = (c < kb && gr > c) ? V[idx2(gr, c, ldv)] : 0.f;
#pragma unroll
        for (int c = 0; c < IC; c++) cv[c] = c < ncl ? C[idx2(gr, c, ldc)] : 0.f;
#pragma unroll
        for (int c = 0; c < NB; c++) Vc[(size_t)r * IV_LD + c] = (c < kb && gr == c) ? 1.f : v[c];
#pragma unroll
        for (int c = 0; c < IC; c++) Cc[r + (size_t)c * rp] = cv[c];
    }
    for (int e = tid; e < NB * NB; e += 256) {
        const int k = e & (NB - 1), a = e / NB;
        Xs[a][k] = Tw[k + a * NB];
    }
    __syncthreads();
    // partial S: thread (rg, ti, tc) owns S(4ti.., 4tc..) over row group rg
    {
        const int rg = tid >> 6, ti = tid & 7, tc = (tid >> 3) & 7;
        const int i0 = 4 * ti, c0 = 4 * tc;
        const int ra = (R * rg) >> 2, rb = (R * (rg + 1)) >> 2;
        float acc[4][4];
#pragma unroll
        for (int a = 0; a < 4; a++)
#pragma unroll
            for (int b = 0; b < 4; b++) acc[a][b] = 0.f;
        const float *cp = Cc + (size_t)c0 * rp;
#pragma unroll 4
        for (int r = ra; r < rb; r++) {
            const float4 v = *reinterpret_cast<const float4 *>(Vc + (size_t)r * IV_LD + i0);
            float cv[4];
#pragma unroll
            for (int b = 0; b < 4; b++) cv[b] = cp[(size_t)b * rp + r];
#pragma unroll
            for (int b = 0; b < 4; b++) {
                acc[0][b] = fmaf(v.x, cv[b], acc[0][b]);
                acc[1][b] = fmaf(v.y, cv[b], acc[1][b]);
                acc[2][b] = fmaf(v.z, cv[b], acc[2][b]);
                acc[3][b] = fmaf(v.w, cv[b], acc[3][b]);
            }
        }
#pragma unroll
        for (int b = 0; b < 4; b++)
            *reinterpret_cast<float4 *>(&pg[rg][(c0 + b) * NB + i0]) =
                make_float4(acc[0][b], acc[1][b], acc[2][b], acc[3][b]);
    }
    __syncthreads();
    for (int e = tid; e < IC * NB; e += 256) pw[e] = (pg[0][e] + pg[1][e]) + (pg[2][e] + pg[3][e]);
    cluster.sync();
    // cluster sum, 16-byte remote loads in rank order (all issued before the
    // first add: cs <= 16)
    {
        const int e = tid;                              // IC * NB / 4 == 256 vectors
        float4 v[16];
#pragma unroll
        for (int q = 0; q < 16; q++)
            v[q] = q < cs ? reinterpret_cast<const float4 *>(cluster.map_shared_rank(pw, q))[e]
                          : make_float4(0.f, 0.f, 0.f, 0.f);
        float4 sum = make_float4(0.f, 0.f, 0.f, 0.f);
#pragma unroll
        for (int q = 0; q < 16; q++) { sum.x += v[q].x; sum.y += v[q].y; sum.z += v[q].z; sum.w += v[q].w; }
        reinterpret_cast<float4 *>(Sx)[e] = sum;
    }
    __syncthreads();
    // W(a, c) = sum_k Tw(k, a) S(k, c)
    for (int e = tid; e < NB * IC; e += 256) {
        const int a = e & (NB - 1), c = e / NB;
        float sum = 0.f;
#pragma unroll 8
        for (int k = 0; k < NB; k++) sum = fmaf(Xs[a][k], Sx[c * NB + k], sum);
        Wc[c * IV_LD + a] = sum;
    }
    __syncthreads();
    // C -= V W, one row per thread (two accumulators per column)
    for (int r = tid; r < R; r += 256) {
        float vr[NB];
#pragma unroll
        for (int q = 0; q < NB / 4; q++) {
            const float4 v = *reinterpret_cast<const float4 *>(Vc + (size_t)r * IV_LD + 4 * q);
            vr[4 * q] = v.x; vr[4 * q + 1] = v.y; vr[4 * q + 2] = v.z; vr[4 * q + 3] = v.w;
        }
#pragma unroll 2
        for (int c = 0; c < ncl; c++) {
            float t0 = 0.f, t1 = 0.f;
#pragma unroll
            for (int q = 0; q < NB / 4; q += 2) {
                const float4 w0 = *reinterpret_cast<const float4 *>(&Wc[c * IV_LD + 4 * q]);
                const float4 w1 = *reinterpret_cast<const float4 *>(&Wc[c * IV_LD + 4 * q + 4]);
                t0 = fmaf(vr[4 * q], w0.x, t0);
                t0 = fmaf(vr[4 * q + 1], w0.y, t0);
                t0 = fmaf(vr[4 * q + 2], w0.z, t0);
                t0 = fmaf(vr[4 * q + 3], w0.w, t0);
                t1 = fmaf(vr[4 * q + 4], w1.x, t1);
                t1 = fmaf(vr[4 * q + 5], w1.y, t1);
                t1 = fmaf(vr[4 * q + 6], w1.z, t1);
                t1 = fmaf(vr[4 * q + 7], w1.w, t1);
            }
            Cc[r + (size_t)c * rp] -= t0 + t1;
        }
    }
    __syncthreads();
    for (int r = tid; r < R; r += 256) {
#pragma unroll 8
        for (int c = 0; c < ncl; c++) C[idx2(r0 + r, c, ldc)] = Cc[r + (size_t)c * rp];
    }
    cluster.sync();   // pw must outlive the remote reads
}

template <typename T>
static int launch_larfb(const T *V, int ldv, const T *Tw, int kb, int L, T *C, int ldc, int Nc,
                        int trans, cudaStream_t s)
{
    constexpr int NB = panel_nb<T>();
    if (Nc <= 0 || L <= 0 || kb <= 0) return 0;
    ProfScope ps(K_LARFB, s);
    k_larfb_left<T, NB><<<ceil_div(Nc, 32), 256, 0, s>>>(V, ldv, Tw, kb, L, C, ldc, Nc, trans);
    return cudaGetLastError() == cudaSuccess ? 0 : MPIR_CUDA_ERROR;
}

// Row-chunked inner update for panels too tall for one cluster's shared
// memory (FP32): the rows are split into IT_ROWS-row chunks and the columns
// into 32-column groups, one CTA per (chunk, group) in each of three
// kernels chained by programmatic dependent launch:
//   k_itall_part   P[g][q] = V_q^T C_{q,g}                     (32 x 32)
//   k_itall_red    W_g = Tw^T sum_q P[g][q]   (fixed summation order)
//   k_itall_apply  C_{q,g} -= V_q W_g
// V is the unit lower trapezoid stored in the panel's columns (kb <= 32).
constexpr int IT_ROWS = 256;

__device__ __forceinline__ float itall_v(const float *__restrict__ V, int ldv, int kb, int gr, int c)
{
    return c < kb ? (gr > c ? V[idx2(gr, c, ldv)] : (gr == c ? 1.f : 0.f)) : 0.f;
}

__global__ void __launch_bounds__(256)
k_itall_part(const float *__restrict__ V, int ldv, int kb, int L, const float *__restrict__ C, int ldc, int nc,
             float *__restrict__ P, int nch)
{
    extern __shared__ __align__(16) float sm[];
    float *Vc = sm;                                    // IT_ROWS x IV_LD, row-major
    float *Cc = Vc + IT_ROWS * IV_LD;                  // IC x (IT_ROWS + 1), column-major
    constexpr int RP = IT_ROWS + 1;
    __shared__ __align__(16) float pg[4][IC * 32];
    const int tid = threadIdx.x;
    const int q = blockIdx.x, g = blockIdx.y;
    const int cg0 = g * IC, ncl = min(IC, nc - cg0);
    const int r0 = q * IT_ROWS, R = min(IT_ROWS, L - r0);
    pdl_wait();
    pdl_trigger();
    for (int r = tid; r < IT_ROWS; r += 256) {
        const int gr = r0 + r;
        const bool in = r < R;
#pragma unroll
        for (int c = 0; c < 32; c++) Vc[r * IV_LD + c] = in ? itall_v(V, ldv, kb, gr, c) : 0.f;
#pragma unroll
        for (int c = 0; c < IC; c++) Cc[r + c * RP] = (in && c < ncl) ? C[idx2(gr, cg0 + c, ldc)] : 0.f;
    }
    __syncthreads();
    const int rg = tid >> 6, ti = tid & 7, tc = (tid >> 3) & 7;
    const int i0 = 4 * ti, c0 = 4 * tc;
    const int ra = rg * (IT_ROWS / 4), rb = ra + IT_ROWS / 4;
    float acc[4][4];
#pragma unroll
    for (int a = 0; a < 4; a++)
#pragma unroll
        for (int b = 0; b < 4; b++) acc[a][b] = 0.f;
    const float *cp = Cc + c0 * RP;
#pragma unroll 4
    for (int r = ra; r < rb; r++) {
        const float4 v = *reinterpret_cast<const float4 *>(Vc + r * IV_LD + i0);
        float cv[4];
#pragma unroll
        for (int b = 0; b < 4; b++) cv[b] = cp[b * RP + r];
#pragma unroll
        for (int b = 0; b < 4; b++) {
            acc[0][b] = fmaf(v.x, cv[b], acc[0][b]);
            acc[1][b] = fmaf(v.y, cv[b], acc[1][b]);
            acc[2][b] = fmaf(v.z, cv[b], acc[2][b]);
            acc[3][b] = fmaf(v.w, cv[b], acc[3][b]);
        }
    }
#pragma unroll
    for (int b = 0; b < 4; b++)
        *reinterpret_cast<float4 *>(&pg[rg][(c0 + b) * 32 + i0]) =
            make_float4(acc[0][b], acc[1][b], acc[2][b], acc[3][b]);
    __syncthreads();
    float *Pq = P + ((size_t)g * nch + q) * (IC * 32);
    for (int e = tid; e < IC * 32; e += 256) Pq[e] = (pg[0][e] + pg[1][e]) + (pg[2][e] + pg[3][e]);
}

__global__ void __launch_bounds__(1024)
k_itall_red(const float *__restrict__ P, int nch, const float *__restrict__ Tw, float *__restrict__ W)
{
    __shared__ float S[IC * 32];                       // S(k, c) at k + 32 c
    __shared__ float X[32][33];                        // X[a][k] = Tw(k, a)
    const int e = threadIdx.x, g = blockIdx.x;
    pdl_wait();
    pdl_trigger();
    X[e >> 5][e & 31] = Tw[(e & 31) + (e >> 5) * 32];
    const float *Pg = P + (size_t)g * nch * (IC * 32) + e;
    float a0 = 0.f, a1 = 0.f, a2 = 0.f, a3 = 0.f;
    int q = 0;
    for (; q + 4 <= nch; q += 4) {
        a0 += Pg[(size_t)q * (IC * 32)];
        a1 += Pg[(size_t)(q + 1) * (IC * 32)];
        a2 += Pg[(size_t)(q + 2) * (IC * 32)];
        a3 += Pg[(size_t)(q + 3) * (IC * 32)];
    }
    for (; q < nch; q++) a0 += Pg[(size_t)q * (IC * 32)];
    S[e] = (a0 + a1) + (a2 + a3);
    __syncthreads();
    const int a = e & 31, c = e >> 5;                  // W(a, c) = sum_k Tw(k, a) S(k, c)
    float t = 0.f;
#pragma unroll 8
    for (int k = 0; k < 32; k++) t = fmaf(X[a][k], S[k + 32 * c], t);
    W[(size_t)g * (IC * 32) + a + 32 * c] = t;
}

__global__ void __launch_bounds__(256)
k_itall_apply(const float *__restrict__ V, int ldv, int kb, int L, float *__restrict__ C, int ldc, int nc,
              const float *__restrict__ W)
{
    __shared__ __align__(16) float Wc[IC * IV_LD];     // Wc[c][k] = W(k, c)
    const int tid = threadIdx.x;
    const int q = blockIdx.x, g = blockIdx.y;
    const int cg0 = g * IC, ncl = min(IC, nc - cg0);
    const int gr = q * IT_ROWS + tid;
    pdl_wait();
    pdl_trigger();
    for (int e = tid; e < IC * 32; e += 256) Wc[(e >> 5) * IV_LD + (e & 31)] = W[(size_t)g * (IC * 32) + e];
    float vr[32];
#pragma unroll
    for (int k = 0; k < 32; k++) vr[k] = gr < L ? itall_v(V, ldv, kb, gr, k) : 0.f;
    __syncthreads();
    if (gr >= L) return;
    float *Cr = C + gr + (size_t)cg0 * ldc;
#pragma unroll 2
    for (int c = 0; c < ncl; c++) {
        float t0 = 0.f, t1 = 0.f;
#pragma unroll
        for (int k = 0; k < 32; k += 8) {
            const float4 w0 = *reinterpret_cast<const float4 *>(&Wc[c * IV_LD + k]);
            const float4 w1 = *reinterpret_cast<const float4 *>(&Wc[c * IV_LD + k + 4]);
            t0 = fmaf(vr[k], w0.x, t0);
            t0 = fmaf(vr[k + 1], w0.y, t0);
            t0 = fmaf(vr[k + 2], w0.z, t0);
            t0 = fmaf(vr[k + 3], w0.w, t0);
            t1 = fmaf(vr[k + 4], w1.x, t1);
            t1 = fmaf(vr[k + 5], w1.y, t1);
            t1 = fmaf(vr[k + 6], w1.z, t1);
            t1 = fmaf(vr[k + 7], w1.w, t1);
        }
        Cr[(size_t)c * ldc] -= t0 + t1;
    }
}

static int inner_update_tall(const float *V, int ldv, const float *Tw, int kb, int L, float *C, int ldc, int nc,
                             float *P, float *W, cudaStream_t s)
{
    const int nch = ceil_div(L, IT_ROWS), ngrp = ceil_div(nc, IC);
    const size_t smem = ((size_t)IT_ROWS * IV_LD + (size_t)(IT_ROWS + 1) * IC) * sizeof(float);
    static PerDeviceOnce once;
    once([&] { cudaFuncSetAttribute(k_itall_part, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem); });
    ProfScope ps(K_LARFB, s);
    cudaError_t e = pdl_launch(k_itall_part, dim3(nch, ngrp), dim3(256), smem, s, V, ldv, kb, L, (const float *)C,
                               ldc, nc, P, nch);
    if (e == cudaSuccess) e = pdl_launch(k_itall_red, dim3(ngrp), dim3(1024), 0, s, (const float *)P, nch, Tw, W);
    if (e == cudaSuccess)
        e = pdl_launch(k_itall_apply, dim3(nch, ngrp), dim3(256), 0, s, V, ldv, kb, L, C, ldc, nc, (const float *)W);
    return e == cudaSuccess ? 0 : MPIR_CUDA_ERROR;
}

// Inner update of nc (<= 96) columns on one cluster (fused kernel).
static int inner_update_cl(const float *V, int ldv, const float *Tw, int kb, int L, float *C, int ldc, int nc,
                           float *P, float *W, cudaStream_t s)
{
    {   // whole chunk in shared memory when it fits (16-CTA cluster)
        auto kern = k_inner_cl_s<32>;
        static PerDeviceOnce once;
        once([&] {
            cudaFuncSetAttribute(kern, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
            cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, 160 * 1024);
        });
        const int want = std::max(1, std::min(16, ceil_div(L, 64)));
        const int chunk0 = ceil_div(L, want);
        const size_t smem0 = ((size_t)chunk0 * IV_LD + (size_t)(chunk0 | 1) * IC) * sizeof(float);
        const int cs = cluster_size_for((const void *)kern, 256, smem0, want);
        const int chunk = ceil_div(L, cs), rp = chunk | 1;
        const size_t smem = ((size_t)chunk * IV_LD + (size_t)rp * IC) * sizeof(float);
        if (smem <= 160 * 1024) {
            cudaLaunchConfig_t cfg = {};
            cfg.gridDim = dim3(cs, ceil_div(nc, IC), 1);
            cfg.blockDim = dim3(256, 1, 1);
            cfg.dynamicSmemBytes = smem;
            cfg.stream = s;
            cudaLaunchAttribute at[2];
            at[0].id = cudaLaunchAttributeClusterDimension;
            at[0].val.clusterDim.x = cs;
            at[0].val.clusterDim.y = 1;
            at[0].val.clusterDim.z = 1;
            at[1].id = cudaLaunchAttributeProgrammaticStreamSerialization;   // waits in-kernel
            at[1].val.programmaticStreamSerializationAllowed = 1;
            cfg.attrs = at;
            cfg.numAttrs = 2;
            ProfScope ps(K_LARFB, s);
            cudaError_t e = cudaLaunchKernelEx(&cfg, kern, V, ldv, kb, L, C, ldc, nc, Tw, chunk, rp);
            return e == cudaSuccess ? 0 : MPIR_CUDA_ERROR;
        }
    }
    if (P && W) return inner_update_tall(V, ldv, Tw, kb, L, C, ldc, nc, P, W, s);
    auto kern = k_inner_cl<32>;
    static PerDeviceOnce once;
    once([&] { cudaFuncSetAttribute(kern, cudaFuncAttributeNonPortableClusterSizeAllowed, 1); });
    int want = ceil_div(L, 256);
    if (want > 16) want = 16;
    const int cs = cluster_size_for((const void *)kern, 256, 0, want);
    const int chunk = ceil_div(L, cs);
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(cs, 1, 1);
    cfg.blockDim = dim3(256, 1, 1);
    cfg.stream = s;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeClusterDimension;
    at[0].val.clusterDim.x = cs;
    at[0].val.clusterDim.y = 1;
    at[0].val.clusterDim.z = 1;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    ProfScope ps(K_LARFB, s);
    cudaError_t e = cudaLaunchKernelEx(&cfg, kern, V, ldv, kb, L, C, ldc, nc, Tw, chunk);
    return e == cudaSuccess ? 0 : MPIR_CUDA_ERROR;
}

// Inner update of nc (<= 96) columns: three row-parallel kernels.
template <typename T>
static int inner_update(const T *V, int ldv, const T *Tw, int kb, int L, T *C, int ldc, int nc, T *P, T *W,
                        cudaStream_t s)
{
    constexpr int NB = panel_nb<T>();
    if (nc <= 0 || L <= 0 || kb <= 0) return 0;
    if (nc > INNER_MAXC) return launch_larfb<T>(V, ldv, Tw, kb, L, C, ldc, nc, 1, s);
    if (sizeof(T) == 4)
        return inner_update_cl((const float *)V, ldv, (const float *)Tw, kb, L, (float *)C, ldc, nc, (float *)P,
                               (float *)W, s);
    const int nch = ceil_div(L, INNER_ROWS);
    ProfScope ps(K_LARFB, s);
    k_inner_w<T, NB><<<nch, 256, 0, s>>>(V, ldv, kb, L, C, ldc, nc, P);
    k_inner_reduce<T, NB><<<1, 256, 0, s>>>(P, nch, Tw, nc, 1, W);
    k_inner_update<T, NB><<<nch, 256, 0, s>>>(V, ldv, kb, L, C, ldc, nc, W);
    return cudaGetLastError() == cudaSuccess ? 0 : MPIR_CUDA_ERROR;
}

// Scratch of the two-level factorization (FP32 path).
struct OuterWs {
    float *V, *Vl, *Vt, *Vtl, *P, *W, *Wl, *G, *GP, *innerP, *innerW;
    int ldv;
    size_t pcap;
    PanelGrid pg;                        // exchange buffers of the tall-panel variant
};
constexpr int GSPLIT = 24;               // split-K of the outer block's Gram matrix
constexpr int SPLIT_MIN_K = 8;           // K steps (of 32) per split of V^T C, at least

static constexpr int PSPLIT_CAP = 320;   // (column tiles x K splits) of W = V^T C

static OuterWs outer_layout(void *base, int M, int N, size_t *bytes)
{
    uintptr_t b = (uintptr_t)base, off = 0;
    auto take = [&](size_t n) { off = (off + 1023) & ~(uintptr_t)1023; float *p = (float *)(b + off); off += n * 4; return p; };
    OuterWs w{};
    w.ldv = rup32(M > 0 ? M : 1);
    const size_t ncp = (size_t)rup32(N > 0 ? N : 1);
    w.V = take((size_t)w.ldv * OUTER_NB);
    w.Vl = take((size_t)w.ldv * OUTER_NB);
    w.Vt = take((size_t)OUTER_NB * w.ldv);
    w.Vtl = take((size_t)OUTER_NB * w.ldv);
    w.pcap = (size_t)OUTER_NB * OUTER_NB * PSPLIT_CAP;
    const size_t ncp128 = (size_t)ceil_div(N > 0 ? N : 1, OUTER_NB) * OUTER_NB;
    if (w.pcap < (size_t)OUTER_NB * ncp128) w.pcap = (size_t)OUTER_NB * ncp128;
    w.P = take(w.pcap);
    w.W = take((size_t)OUTER_NB * ncp);
    w.Wl = take((size_t)OUTER_NB * ncp);
    w.G = take((size_t)OUTER_NB * OUTER_NB);
    w.GP = take((size_t)OUTER_NB * OUTER_NB * GSPLIT);
    w.innerP = take((size_t)ceil_div(M > 0 ? M : 1, INNER_ROWS) * 32 * INNER_MAXC * 2);
    w.innerW = take((size_t)32 * INNER_MAXC * 2);
    w.pg.gx = take((size_t)2 * PANEL_GRID_MAX * 64);       // 2 NB FP32 or NB FP64 values per CTA and parity
    w.pg.bar = reinterpret_cast<unsigned int *>(take(64));
    if (bytes) *bytes = (size_t)((off + 1023) & ~(uintptr_t)1023);
    return w;
}

size_t geqrf_ws_bytes(int M, int N)
{
    size_t b = 0;
    outer_layout(nullptr, M, N, &b);
    return b;
}

// two block-parity copies for the critical path + one for the wide updates
size_t geqrf_la_ws_bytes(int M, int N) { return 3 * geqrf_ws_bytes(M, N); }

static int tc_mode(GemmPrec p)
{
    return p == GemmPrec::FP32 ? TCM_TF32X3 : (p == GemmPrec::BF16 ? TCM_BF16 : TCM_TF32);
}

// Prepares V (and splits) for the outer block whose panel sits at X (ldx),
// height L, nr reflectors.
static void prep_v(const float *X, int ldx, int L, int nr, OuterWs &w, int split, cudaStream_t s)
{
    ProfScope ps(K_LARFB_AUX, s);
    pdl_launch(k_prep_v, dim3(ceil_div(w.ldv, 32)), dim3(256), 0, s, X, ldx, L, nr, w.V, w.Vl, w.ldv, w.Vt, w.Vtl, split);
}

struct OuterPlan {
    int nsplit;
    size_t pstride;
};

// Phase 1 of an outer update: P = V^T C (split-K partials), which does not
// need the block's T factor.
static int outer_apply_p1(OuterWs &w, int L, float *C, int ldc, int Nc, int mode, int *err, cudaStream_t s,
                          OuterPlan *pl)
{
    pl->nsplit = 0;
    if (Nc <= 0 || L <= 0) return 0;
    const int split = mode == TCM_TF32X3;
    CUtensorMap tV, tVl, tC;
    int rc = 0;
    rc |= tmap_colmajor(&tV, w.V, L, OUTER_NB, w.ldv, OUTER_NB);
    rc |= tmap_colmajor(&tVl, split ? w.Vl : w.V, L, OUTER_NB, w.ldv, OUTER_NB);
    rc |= tmap_colmajor(&tC, C, L, Nc, ldc, OUTER_NB);
    if (rc) return MPIR_UNSUP();
    const int ntn = ceil_div(Nc, OUTER_NB);
    const int ksteps = ceil_div(L, 32);
    int nsplit = ceil_div(2 * 152, ntn);
    if (nsplit > PSPLIT_CAP / ntn) nsplit = PSPLIT_CAP / ntn;
    // every split runs at least SPLIT_MIN_K K steps: shorter ones spend
    // their time in pipeline fill and in writing partials the reduction
    // then has to read back
    if (nsplit > ksteps / SPLIT_MIN_K) nsplit = ksteps / SPLIT_MIN_K;
    if (nsplit > ksteps) nsplit = ksteps;
    if (nsplit < 1) nsplit = 1;
    if ((size_t)nsplit * OUTER_NB * ntn * OUTER_NB > w.pcap) nsplit = 1;
    const size_t pstride = (size_t)OUTER_NB * ntn * OUTER_NB;
    // P[z] = V^T C  (M = 128 rows of V^T, N = Nc, K = L)
    rc = gemm_tc(mode, split, TCE_STORE, tV, tVl, tC, tC, 0, 0, 0, 0, OUTER_NB, Nc, L, w.P, OUTER_NB, pstride,
                 nsplit, err, s);
    pl->nsplit = nsplit;
    pl->pstride = pstride;
    return rc;
}

// Phase 2: W = op(Tb) sum P, C -= V W.
static int outer_apply_p2(OuterWs &w, const float *Tb, int trans, int L, float *C, int ldc, int Nc, int mode,
                          const OuterPlan &pl, int *err, cudaStream_t s)
{
    if (Nc <= 0 || L <= 0) return 0;
    const int split = mode == TCM_TF32X3;
    CUtensorMap tVt, tVtl, tW, tWl;
    int rc = 0;
    rc |= tmap_colmajor(&tVt, w.Vt, OUTER_NB, L, OUTER_NB, OUTER_NB);
    rc |= tmap_colmajor(&tVtl, split ? w.Vtl : w.Vt, OUTER_NB, L, OUTER_NB, OUTER_NB);
    rc |= tmap_colmajor(&tW, w.W, OUTER_NB, Nc, OUTER_NB, OUTER_NB);
    rc |= tmap_colmajor(&tWl, split ? w.Wl : w.W, OUTER_NB, Nc, OUTER_NB, OUTER_NB);
    if (rc) return MPIR_UNSUP();
    {
        ProfScope ps(K_LARFB_AUX, s);
        reduce_w(w.P, pl.nsplit, pl.pstride, Tb, trans, Nc, w.W, w.Wl, OUTER_NB, split, s);
    }
    // C -= V W  (M = L, N = Nc, K = 128)
    rc = gemm_tc(mode, 0, TCE_SUB, tVt, tVtl, tW, tWl, 0, 0, 0, 0, L, Nc, OUTER_NB, C, ldc, 0, 1, err, s);
    return rc ? rc : (cudaGetLastError() == cudaSuccess ? 0 : MPIR_CUDA_ERROR);
}

// C (L x Nc, ldc) <- (I - V X V^T) C for the prepared outer block, X = Tb^T
// (trans) or Tb, on the tensor cores:  P = V^T C (split-K),  W = X sum P,
// C -= V W.
static int outer_apply(OuterWs &w, const float *Tb, int trans, int L, float *C, int ldc, int Nc, int mode,
                       int *err, cudaStream_t s)
{
    OuterPlan pl{};
    int rc = outer_apply_p1(w, L, C, ldc, Nc, mode, err, s, &pl);
    if (rc) return rc;
    return outer_apply_p2(w, Tb, trans, L, C, ldc, Nc, mode, pl, err, s);
}

// G = V^T V of the prepared block, then the outer compact-WY factor Tb.
static int outer_T(OuterWs &w, const float *Tw32, int L, int nr, float *Tb, int mode, int *err, cudaStream_t s)
{
    const int split = mode == TCM_TF32X3;
    CUtensorMap tV, tVl;
    int rc = tmap_colmajor(&tV, w.V, L, OUTER_NB, w.ldv, OUTER_NB);
    rc |= tmap_colmajor(&tVl, split ? w.Vl : w.V, L, OUTER_NB, w.ldv, OUTER_NB);
    if (rc) return MPIR_UNSUP();
    const int ksteps = ceil_div(L, 32);
    int nsplit = ksteps < GSPLIT ? ksteps : GSPLIT;
    if (nsplit < 1) nsplit = 1;
    const size_t pstride = (size_t)OUTER_NB * OUTER_NB;
    // G = V^T V with both operands pre-split (w.V holds only the TF32 part);
    // its own partial buffer, so that it can run beside the next columns'
    // V^T C
    rc = gemm_tc(mode, 0, TCE_STORE, tV, tVl, tV, tVl, 0, 0, 0, 0, OUTER_NB, OUTER_NB, L, w.GP, OUTER_NB,
                 pstride, nsplit, err, s);
    if (rc) return rc;
    {
        ProfScope ps(K_LARFB_AUX, s);
        pdl_launch(k_sum_splits, dim3(OUTER_NB * OUTER_NB / 256), dim3(256), 0, s, (const float *)w.GP, nsplit, pstride,
                   (int)(OUTER_NB * OUTER_NB), w.G);
    }
    {
        ProfScope ps(K_LARFB_AUX, s);
        const size_t smem = (size_t)(2 * OUTER_NB * OUTER_NB + 96 * 32) * 4;
        static PerDeviceOnce once;
        once([&] { cudaFuncSetAttribute(k_outer_T, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem); });
        pdl_launch(k_outer_T, dim3(1), dim3(256), smem, s, Tw32, (const float *)w.G, nr, Tb);
    }
    return cudaGetLastError() == cudaSuccess ? 0 : MPIR_CUDA_ERROR;
}

// ---------------------------------------------------------------------------
// Aggregated compact-WY factor of the whole reflector set: Tf (K x K upper
// triangular, column-major, ld ldt) with H_0 ... H_{K-1} = I - V Tf V^T, so
// that a vector application is three matrix-vector products instead of one
// dependent step per block.  Built block column by block column during the
// two-level factorization: with V_1 the reflectors before outer block b
// (columns 0..J0) and V_2 = V_b,
//   (I - V_1 T_1 V_1^T)(I - V_2 T_2 V_2^T)
//       = I - [V_1 V_2] [T_1, -T_1 (V_1^T V_2) T_2; 0, T_2] [V_1 V_2]^T
// (Schreiber and Van Loan's aggregation of WY factors).  V_2 is zero above
// row J0, so V_1^T V_2 only involves rows >= J0, where V_1 is the plain
// stored part A(J0:, 0:J0).  X = (V_1^T V_2) T_2 comes from the tensor-core
// product and the split-K reduction of the trailing update (its transpose,
// 128 x J0, ld 128); T_12 = -T_1 X is the SIMT product below.
// ---------------------------------------------------------------------------
constexpr int TF_TI = 64;                         // rows of T_12 per tile
constexpr int TF_KS = 32;                         // k per shared-memory stage
constexpr int TF_TILE = TF_TI * OUTER_NB;

// part[ti * nkc + kc] (64 x 128, column-major) = T(i0:i0+64, kc chunk) X(kc chunk, :)
__global__ void __launch_bounds__(256)
k_tfull_prod(const float *__restrict__ Tf, int ldt, const float *__restrict__ Xt, int J0, int KC, int nkc,
             float *__restrict__ part)
{
    pdl_wait();
    pdl_trigger();
    const int ti = blockIdx.x, kc = blockIdx.y;
    const int i0 = ti * TF_TI;
    const int k1 = min((kc + 1) * KC, J0);
    if (k1 <= i0) return;                         // T(i, k) = 0 for k < i
    const int k0 = max(kc * KC, i0);
    __shared__ __align__(16) float Ts[TF_KS][TF_TI];       // Ts[kk][r] = T(i0 + r, k + kk)
    __shared__ __align__(16) float Xs[TF_KS][OUTER_NB];    // Xs[kk][c] = X(k + kk, c)
    const int tid = threadIdx.x, ty = tid >> 4, tx = tid & 15;
    float acc[4][8];
#pragma unroll
    for (int r = 0; r < 4; r++)
#pragma unroll
        for (int c = 0; c < 8; c++) acc[r][c] = 0.f;
    for (int k = k0; k < k1; k += TF_KS) {
        for (int e = tid; e < TF_KS * TF_TI / 4; e += 256) {
            const int kk = e / (TF_TI / 4), r4 = e % (TF_TI / 4);
            float4 v = make_float4(0.f, 0.f, 0.f, 0.f);
            if (k + kk < k1) v = *reinterpret_cast<const float4 *>(Tf + (size_t)(k + kk) * ldt + i0 + 4 * r4);
            *reinterpret_cast<float4 *>(&Ts[kk][4 * r4]) = v;
        }
        for (int e = tid; e < TF_KS * OUTER_NB / 4; e += 256) {
            const int kk = e / (OUTER_NB / 4), c4 = e % (OUTER_NB / 4);
            float4 v = make_float4(0.f, 0.f, 0.f, 0.f);
            if (k + kk < k1) v = *reinterpret_cast<const float4 *>(Xt + (size_t)(k + kk) * OUTER_NB + 4 * c4);
            *reinterpret_cast<float4 *>(&Xs[kk][4 * c4]) = v;
        }
        __syncthreads();
#pragma unroll 8
        for (int kk = 0; kk < TF_KS; kk++) {
            const float4 a = *reinterpret_cast<const float4 *>(&Ts[kk][4 * ty]);
            const float4 b0 = *reinterpret_cast<const float4 *>(&Xs[kk][4 * tx]);
            const float4 b1 = *reinterpret_cast<const float4 *>(&Xs[kk][64 + 4 * tx]);
            const float av[4] = {a.x, a.y, a.z, a.w};
            const float bv[8] = {b0.x, b0.y, b0.z, b0.w, b1.x, b1.y, b1.z, b1.w};
#pragma unroll
            for (int r = 0; r < 4; r++)
#pragma unroll
                for (int c = 0; c < 8; c++) acc[r][c] = fmaf(av[r], bv[c], acc[r][c]);
        }
        __syncthreads();
    }
    float *pp = part + ((size_t)ti * nkc + kc) * TF_TILE;
#pragma unroll
    for (int c = 0; c < 8; c++) {
        const int col = c < 4 ? 4 * tx + c : 64 + 4 * tx + (c - 4);
#pragma unroll
        for (int r = 0; r < 4; r++) pp[(size_t)col * TF_TI + 4 * ty + r] = acc[r][c];
    }
}

// Tf(i0 + r, J0 + c) = -sum over the valid chunks (fixed order); the diagonal
// block Tf(J0:J0+nr, J0:J0+nr) = Tb (grid row blockIdx.x == J0 / 64 copies it).
__global__ void __launch_bounds__(256)
k_tfull_reduce(const float *__restrict__ part, int J0, int nr, int KC, int nkc, const float *__restrict__ Tb,
               float *__restrict__ Tf, int ldt)
{
    pdl_wait();
    pdl_trigger();
    const int ti = blockIdx.x, tid = threadIdx.x;
    if (ti * TF_TI >= J0) {
        if (blockIdx.y) return;
        for (int e = tid; e < OUTER_NB * OUTER_NB; e += 256) {
            const int i = e % OUTER_NB, c = e / OUTER_NB;
            if (i < nr && c < nr) Tf[(size_t)(J0 + c) * ldt + J0 + i] = Tb[i + (size_t)c * OUTER_NB];
        }
        return;
    }
    // blockIdx.y: a group of 16 columns; loads batched 8 deep, summed in chunk order
    const int i0 = ti * TF_TI, kc0 = i0 / KC;
    const int e = blockIdx.y * 16 * TF_TI + tid * 4;          // 4 consecutive rows per thread
    const int r = e % TF_TI, c = e / TF_TI;
    if (c >= nr) return;
    const float *pp = part + (size_t)ti * nkc * TF_TILE + (size_t)c * TF_TI + r;
    float4 sum = make_float4(0.f, 0.f, 0.f, 0.f);
    for (int kc = kc0; kc < nkc; kc += 8) {
        float4 v[8];
#pragma unroll
        for (int u = 0; u < 8; u++)
            v[u] = kc + u < nkc ? *reinterpret_cast<const float4 *>(pp + (size_t)(kc + u) * TF_TILE)
                                : make_float4(0.f, 0.f, 0.f, 0.f);
#pragma unroll
        for (int u = 0; u < 8; u++) { sum.x += v[u].x; sum.y += v[u].y; sum.z += v[u].z; sum.w += v[u].w; }
    }
    float *out = Tf + (size_t)(J0 + c) * ldt + i0 + r;
    out[0] = -sum.x; out[1] = -sum.y; out[2] = -sum.z; out[3] = -sum.w;
}

// Block column b of Tf (outer block at J0, nr reflectors, its prepared V in
// w and its factor Tb).  A: the matrix being factored (lda), M rows.  The
// aggregation restarts every WY_SEG reflectors: the block is coupled to the
// earlier blocks of its own segment only (columns S .. J0-1), and its
// column of the segment's factor sits at Tf(S.., S..) with J0 - S in place
// of J0.  That bounds the aggregation's work by K WY_SEG^2 / 3 instead of
// K^3 / 3; the vector application then runs one segment after another.
static int tfull_block(OuterWs &w, const float *A, int lda, int M, int J0in, int nr, const float *Tb, float *Tf,
                       int ldt, int mode, int *err, cudaStream_t s)
{
    const int L = M - J0in;
    const int S = (J0in / WY_SEG) * WY_SEG;
    const int J0 = J0in - S;                  // position within the segment
    A += (size_t)S * lda;                     // columns S .. J0in-1 hold the segment's earlier reflectors
    Tf += (size_t)S * ldt + S;
    int ntile = J0 / TF_TI, KC = 32, nkc = 0;
    if (J0 > 0) {
        const int split = mode == TCM_TF32X3;
        CUtensorMap tV, tVl, tA;
        int rc = tmap_colmajor(&tV, w.V, L, OUTER_NB, w.ldv, OUTER_NB);
        rc |= tmap_colmajor(&tVl, split ? w.Vl : w.V, L, OUTER_NB, w.ldv, OUTER_NB);
        rc |= tmap_colmajor(&tA, A + J0in, L, J0, lda, OUTER_NB);
        if (rc) return MPIR_UNSUP();
        const int ntn = ceil_div(J0, OUTER_NB);
        const int ksteps = ceil_div(L, 32);
        int nsplit = ceil_div(2 * 152, ntn);
        if (nsplit > PSPLIT_CAP / ntn) nsplit = PSPLIT_CAP / ntn;
        if (nsplit > ksteps) nsplit = ksteps;
        if (nsplit < 1) nsplit = 1;
        if ((size_t)nsplit * OUTER_NB * ntn * OUTER_NB > w.pcap) nsplit = 1;
        const size_t pstride = (size_t)OUTER_NB * ntn * OUTER_NB;
        // P[z] = V_b^T A(J0in:, S:J0in)   (128 x J0, split-K)
        rc = gemm_tc(mode, split, TCE_STORE, tV, tVl, tA, tA, 0, 0, 0, 0, OUTER_NB, J0, L, w.P, OUTER_NB, pstride,
                     nsplit, err, s);
        if (rc) return rc;
        {
            ProfScope ps(K_LARFB_AUX, s);
            // W = T_b^T sum P = X^T,  X = (V_1^T V_b) T_b
            reduce_w(w.P, nsplit, pstride, Tb, 1, J0, w.W, w.W, OUTER_NB, 0, s);
        }
        // chunking of k: about four tiles per SM, partials within w.P
        int want = ceil_div(8 * 152, ntile);
        const int cap = (int)(w.pcap / ((size_t)ntile * TF_TILE));
        if (want > cap) want = cap;
        if (want > J0 / TF_KS) want = J0 / TF_KS;
        if (want < 1) want = 1;
        KC = ceil_div(ceil_div(J0, want), TF_KS) * TF_KS;
        nkc = ceil_div(J0, KC);
        if ((size_t)ntile * nkc * TF_TILE > w.pcap) return MPIR_UNSUP();
        ProfScope ps(K_LARFB_AUX, s);
        k_tfull_prod<<<dim3(ntile, nkc), 256, 0, s>>>(Tf, ldt, w.W, J0, KC, nkc, w.P);
    }
    {
        ProfScope ps(K_LARFB_AUX, s);
        k_tfull_reduce<<<dim3(ntile + 1, OUTER_NB / 16), 256, 0, s>>>(w.P, J0, nr, KC, nkc, Tb, Tf, ldt);
    }
    return cudaGetLastError() == cudaSuccess ? 0 : MPIR_CUDA_ERROR;
}

template <typename T>
static int geqrf_simt(T *A, int lda, int M, int N, T *tau, T *Tw, int *err, cudaStream_t s, int kmax, void *ws)
{
    constexpr int NB = panel_nb<T>();
    int k = M < N ? M : N;
    if (kmax >= 0 && kmax < k) k = kmax;
    OuterWs wo{};
    if (ws) {
        wo = outer_layout(ws, M, N, nullptr);
        cudaMemsetAsync(wo.pg.bar, 0, 2 * sizeof(unsigned int), s);
    }
    for (int j0 = 0; j0 < k; j0 += NB) {
        const int ncols = k - j0 < NB ? k - j0 : NB;
        const int L = M - j0;
        T *Twb = Tw + (size_t)(j0 / NB) * NB * NB;
        int rc = launch_panel<T>(A, lda, M, j0, ncols, tau, Twb, err, s, ws ? &wo.pg : nullptr);
        if (rc) return rc;
        const int kb = ncols < L ? ncols : L;
        const int Nc = N - j0 - ncols;
        if (Nc > 0) {
            rc = launch_larfb<T>(A + idx2(j0, j0, lda), lda, Twb, kb, L, A + idx2(j0, j0 + ncols, lda), lda, Nc,
                                 1, s);
            if (rc) return rc;
        }
    }
    return 0;
}

template <>
int geqrf<double>(double *A, int lda, int M, int N, double *tau, double *Tw, double *, GemmPrec, void *ws,
                  int *err, cudaStream_t s, const TfullJob *, int kmax)
{
    return geqrf_simt<double>(A, lda, M, N, tau, Tw, err, s, kmax, ws);
}

// Two-level QR, FP32 storage: 32-wide register panels inside 128-wide
// outer blocks; inner updates row-parallel SIMT, outer trailing updates on
// the tensor cores.  Streams (when tf provides them): panels, inner updates
// and the next block's columns on tf->crit; each block's factor (Gram
// matrix, T) on tf->aux beside the next columns' V^T C; the rest of the
// trailing update on s; the aggregated factor Tf on tf->side.
template <>
int geqrf<float>(float *A, int lda, int M, int N, float *tau, float *Tw, float *Tw128, GemmPrec prec, void *ws,
                 int *err, cudaStream_t s, const TfullJob *tf, int kmax)
{
    constexpr int NB = 32;
    int k = M < N ? M : N;
    if (kmax >= 0 && kmax < k) k = kmax;
    if (lda % 4) return MPIR_UNSUP();
    const int mode = tc_mode(prec);
    // look-ahead: critical path on tf->crit, wide trailing updates on s
    const bool la = tf && tf->crit && tf->crit != s && tf->la_a && tf->la_b;
    const bool ax = la && tf->aux && tf->ax_a && tf->ax_b;
    const size_t one = geqrf_ws_bytes(M, N);
    OuterWs wv[2] = {outer_layout(ws, M, N, nullptr),
                     outer_layout(la ? (char *)ws + one : ws, M, N, nullptr)};
    OuterWs wu = la ? outer_layout((char *)ws + 2 * one, M, N, nullptr) : wv[0];
    cudaStream_t cs = la ? tf->crit : s;
    if (la) { cudaEventRecord(tf->la_a, s); cudaStreamWaitEvent(cs, tf->la_a, 0); }
    // the aggregated factor is built on the side stream when there is one,
    // from its own prepared copy of each finished outer block
    const bool side = tf && tf->side && tf->side != s && tf->side != cs && tf->ws2;
    cudaStream_t ss = side ? tf->side : cs;
    OuterWs w2 = side ? outer_layout(tf->ws2, M, N, nullptr) : wv[0];
    if (tf && tf->Tf) {
        if (tf->ldt < k || tf->ldt % 4 || ((uintptr_t)tf->Tf & 15)) return MPIR_UNSUP();
        if (side) { cudaEventRecord(tf->fork, cs); cudaStreamWaitEvent(ss, tf->fork, 0); }
        cudaMemsetAsync(tf->Tf, 0, (size_t)tf->ldt * k * sizeof(float), ss);
    }
    cudaMemsetAsync(wv[0].pg.bar, 0, 2 * sizeof(unsigned int), cs);
    if (la) cudaMemsetAsync(wv[1].pg.bar, 0, 2 * sizeof(unsigned int), cs);
    bool wide_pending = false;
    for (int J0 = 0, b = 0; J0 < k; J0 += OUTER_NB, b++) {
        OuterWs &w = wv[b & 1];
        const int ncolsO = k - J0 < OUTER_NB ? k - J0 : OUTER_NB;
        const int L = M - J0;
        const int nr = ncolsO < L ? ncolsO : L;
        for (int j0 = J0; j0 < J0 + nr; j0 += NB) {
            const int ncols = J0 + ncolsO - j0 < NB ? J0 + ncolsO - j0 : NB;
            const int Li = M - j0;
            float *Twb = Tw + (size_t)(j0 / NB) * NB * NB;
            int rc = launch_panel<float>(A, lda, M, j0, ncols, tau, Twb, err, cs, &w.pg);
            if (rc) return rc;
            const int kb = ncols < Li ? ncols : Li;
            const int nc = J0 + ncolsO - j0 - ncols;
            if (nc > 0) {
                rc = inner_update<float>(A + idx2(j0, j0, lda), lda, Twb, kb, Li, A + idx2(j0, j0 + ncols, lda), lda,
                                         nc, w.innerP, w.innerW, cs);
                if (rc) return rc;
            }
        }
        const int Nc = N - J0 - ncolsO;
        const int n1 = la ? (Nc < OUTER_NB ? Nc : OUTER_NB) : Nc;    // columns updated on the critical path
        float *Tb = Tw128 + (size_t)(J0 / OUTER_NB) * OUTER_NB * OUTER_NB;
        prep_v(A + idx2(J0, J0, lda), lda, L, nr, w, mode == TCM_TF32X3, cs);
        // the block's factor (Gram matrix and T) on the auxiliary stream while
        // the critical path forms V^T C for the next columns, which needs no T
        int rc = 0;
        OuterPlan pl{};
        cudaStream_t ts = ax ? tf->aux : cs;
        if (ax) { cudaEventRecord(tf->ax_a, cs); cudaStreamWaitEvent(ts, tf->ax_a, 0); }
        rc = outer_T(w, Tw + (size_t)(J0 / NB) * NB * NB, L, nr, Tb, mode, err, ts);
        if (rc) return rc;
        if (ax) cudaEventRecord(tf->ax_b, ts);
        if (Nc > 0) {
            // the next block's columns (after the previous wide update has
            // finished with them)
            if (wide_pending) { cudaStreamWaitEvent(cs, tf->la_b, 0); wide_pending = false; }
            rc = outer_apply_p1(w, L, A + idx2(J0, J0 + ncolsO, lda), lda, n1, mode, err, cs, &pl);
            if (rc) return rc;
        }
        if (ax) cudaStreamWaitEvent(cs, tf->ax_b, 0);                 // T of this block ready
        if (tf && tf->Tf) {
            if (side) {
                cudaEventRecord(tf->fork, cs);
                cudaStreamWaitEvent(ss, tf->fork, 0);
                prep_v(A + idx2(J0, J0, lda), lda, L, nr, w2, mode == TCM_TF32X3, ss);
            }
            rc = tfull_block(side ? w2 : w, A, lda, M, J0, nr, Tb, tf->Tf, tf->ldt, mode, err, ss);
            if (rc) return rc;
        }
        if (Nc > 0) {
            rc = outer_apply_p2(w, Tb, 1, L, A + idx2(J0, J0 + ncolsO, lda), lda, n1, mode, pl, err, cs);
            if (rc) return rc;
            if (la && Nc > n1) {
                cudaEventRecord(tf->la_a, cs);
                cudaStreamWaitEvent(s, tf->la_a, 0);
                OuterWs wt = wu;
                wt.V = w.V; wt.Vl = w.Vl; wt.Vt = w.Vt; wt.Vtl = w.Vtl; wt.ldv = w.ldv;
                rc = outer_apply(wt, Tb, 1, L, A + idx2(J0, J0 + ncolsO + n1, lda), lda, Nc - n1, mode, err, s);
                if (rc) return rc;
                cudaEventRecord(tf->la_b, s);
                wide_pending = true;
            }
        }
    }
    if (la) {
        if (wide_pending) cudaStreamWaitEvent(cs, tf->la_b, 0);
        cudaEventRecord(tf->la_a, cs);
        cudaStreamWaitEvent(s, tf->la_a, 0);
    }
    return 0;
}

template <>
int apply_reflectors_left<double>(const double *V, int ldv, int M, int K, const double *Tw, const double *,
                                  int trans, double *C, int ldc, int Nc, GemmPrec, void *, int *, cudaStream_t s)
{
    constexpr int NB = panel_nb<double>();
    const int nblk = ceil_div(K, NB);
    for (int t = 0; t < nblk; t++) {
        const int b = trans ? t : nblk - 1 - t;
        const int j0 = b * NB;
        const int kb = K - j0 < NB ? K - j0 : NB;
        int rc = launch_larfb<double>(V + idx2(j0, j0, ldv), ldv, Tw + (size_t)b * NB * NB, kb, M - j0, C + j0, ldc,
                                      Nc, trans, s);
        if (rc) return rc;
    }
    return 0;
}

template <>
int apply_reflectors_left<float>(const float *V, int ldv, int M, int K, const float *, const float *Tw128,
                                 int trans, float *C, int ldc, int Nc, GemmPrec prec, void *ws, int *err,
                                 cudaStream_t s)
{
    if (ldc % 4 || ldv % 4) return MPIR_UNSUP();
    OuterWs w = outer_layout(ws, M, Nc, nullptr);
    const int mode = tc_mode(prec);
    const int nblk = ceil_div(K, OUTER_NB);
    for (int t = 0; t < nblk; t++) {
        const int b = trans ? t : nblk - 1 - t;
        const int J0 = b * OUTER_NB;
        const int nr = K - J0 < OUTER_NB ? K - J0 : OUTER_NB;
        const int L = M - J0;
        prep_v(V + idx2(J0, J0, ldv), ldv, L, nr, w, mode == TCM_TF32X3, s);
        int rc = outer_apply(w, Tw128 + (size_t)b * OUTER_NB * OUTER_NB, trans, L, C + J0, ldc, Nc, mode, err, s);
        if (rc) return rc;
    }
    return 0;
}

// One block reflector with an explicit compact-WY factor (K <= 128).
int larfb_tc(const float *V, int ldv, int M, int K, const float *Tb, int trans, float *C, int ldc, int N,
             GemmPrec prec, void *ws, int *err, cudaStream_t s)
{
    if (K > OUTER_NB || K < 0) return MPIR_UNSUP();
    if (ldc % 4 || ((uintptr_t)C & 15)) return MPIR_UNSUP();
    if (K == 0 || M == 0 || N == 0) return 0;
    OuterWs w = outer_layout(ws, M, N, nullptr);
    const int mode = tc_mode(prec);
    prep_v(V, ldv, M, K, w, mode == TCM_TF32X3, s);
    return outer_apply(w, Tb, trans, M, C, ldc, N, mode, err, s);
}

} // namespace mpir
