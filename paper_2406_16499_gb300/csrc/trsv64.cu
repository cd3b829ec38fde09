// trsv64.cu -- the triangular solves of the correction solve (Alg. 3 / 4:
// R, T22 and their transposes) for FP32-stored factors of order <= 8192,
// in 64-row diagonal blocks whose inverses are formed once per
// factorization.
//
// One thread-block cluster; CTA r owns rows [r*slice, (r+1)*slice) of x
// (slice a multiple of 64, at most 512: one row per thread).  Per diagonal
// block (from the bottom for U x = b, from the top for U^T x = b):
//   1. every thread with an unsolved row loads its 64 entries of the block
//      column of U (independent of x, in flight during the rest of the step);
//      the CTA owning the next block loads that block's inverse;
//   2. the owner forms x_blk = op(D) b_blk (two warps, D staged in shared
//      memory one step earlier) and sends x_blk into every CTA's shared
//      memory with st.async (one message slot and one mbarrier per step);
//   3. every CTA waits for that step's message on its own mbarrier;
//   4. every thread subtracts its row's 64-term product.
// No cluster-wide barrier per step: the chain from one block's owner to the
// next is one distributed-shared-memory hop, and no dependent global-memory
// read sits on it.
//
// Packed block columns.  Read in place, a step's entries are 64 strided
// 4-byte columns (U x = b) or one 256-byte column piece per thread, 32
// different lines per warp load (U^T x = b); the cluster's 16 SMs then move
// them at a small fraction of their bandwidth.  Once per factorization
// t64_pack copies every off-diagonal block column into the order the solve
// reads it: block column J (columns 64J .. 64J+63) as [16 quads][rows][4],
// rows 0 .. 64J-1 for U x = b and rows 64(J+1) .. N-1 (entries of U^T) for
// U^T x = b, so a warp's load of one quad for 32 consecutive rows is 512
// contiguous bytes and a CTA's share of a step is 16 contiguous runs.  A
// pack of order N serves the solves with any leading n x n block (n <= N).

#include "common.cuh"
#include "kernels.h"
#include "mpir.h"

namespace mpir {

constexpr int T64_THREADS = 512;
constexpr int T64_MAXN = 16 * T64_THREADS;
constexpr int T64_DS = 64 * 65;                  // one staged inverse, rows padded

bool trsv64_ok(int n, size_t ts_bytes) { return ts_bytes == 4 && n > 0 && n <= T64_MAXN; }

// Float offsets of block column J in the packs of an order-N triangle:
// U x = b pack (rows above the block), then the U^T x = b pack (rows below).
__host__ __device__ __forceinline__ size_t t64_off_n(int J) { return (size_t)2048 * J * (J - 1 > 0 ? J - 1 : 0); }
__host__ __device__ __forceinline__ int t64_rows_t(int N, int J) { const int r = N - 64 * (J + 1); return r > 0 ? r : 0; }
__host__ __device__ __forceinline__ size_t t64_off_t(int N, int J)
{
    // 64 * sum_{J' < J} (N - 64 (J' + 1)), every term positive for J <= nblk - 1
    return (size_t)64 * ((size_t)J * N - (size_t)32 * J * (J + 1));
}

size_t t64_pack_elems(int N)
{
    if (N <= 0 || N > T64_MAXN) return 0;
    const int nb = ceil_div(N, 64);
    return t64_off_n(nb) + t64_off_t(N, nb - 1) + 4;
}

// One thread per packed float4: blockIdx.y = block column J, blockIdx.z = 0
// for the U x = b pack, 1 for the U^T x = b pack.  Entries past column N - 1
// (the partial last block) are zeros.
__global__ void __launch_bounds__(256)
k_t64_pack(const float *__restrict__ U, int ldu, int N, float *__restrict__ pack)
{
    pdl_wait();
    pdl_trigger();
    const int J = blockIdx.y, tr = blockIdx.z;
    const int nb = ceil_div(N, 64);
    const int rows = tr ? t64_rows_t(N, J) : 64 * J;
    const int e = blockIdx.x * 256 + threadIdx.x;          // quad-major: e = q * rows + ii
    if (e >= 16 * rows) return;
    const int q = e / rows, ii = e % rows;
    const int c = 64 * J + 4 * q;
    float4 v = make_float4(0.f, 0.f, 0.f, 0.f);
    if (!tr) {
        if (c < N) v.x = U[idx2(ii, c, ldu)];
        if (c + 1 < N) v.y = U[idx2(ii, c + 1, ldu)];
        if (c + 2 < N) v.z = U[idx2(ii, c + 2, ldu)];
        if (c + 3 < N) v.w = U[idx2(ii, c + 3, ldu)];
    } else {
        // rows of the U^T pack are columns i = 64 (J + 1) + ii of U; the
        // block is full here (J < nb - 1), so c .. c + 3 < N
        v = *reinterpret_cast<const float4 *>(U + (size_t)(64 * (J + 1) + ii) * ldu + c);
    }
    float *dst = pack + (tr ? t64_off_n(nb) + t64_off_t(N, J) : t64_off_n(J));
    reinterpret_cast<float4 *>(dst)[e] = v;
}

int t64_pack(const float *U, int ldu, int N, float *pack, cudaStream_t s)
{
    if (N <= 64 || N > T64_MAXN || !pack) return 0;
    if (ldu % 4 || ((uintptr_t)U & 15) || ((uintptr_t)pack & 15)) return -1;
    const int nb = ceil_div(N, 64);
    const int maxrows = 64 * (nb - 1);                      // the largest pack of either kind
    ProfScope ps(K_TRSV, s);
    cudaError_t e = pdl_launch(k_t64_pack, dim3(ceil_div(16 * maxrows, 256), nb, 2), dim3(256), 0, s, U, ldu, N, pack);
    return e == cudaSuccess ? 0 : MPIR_CUDA_ERROR;
}

size_t dinv_elems(int N)
{
    const size_t a = (size_t)(ceil_div(N > 0 ? N : 1, 32)) * 1024;
    const size_t b = (size_t)(ceil_div(N > 0 ? N : 1, 64)) * 4096;
    return a > b ? a : b;
}

// Inverses of the 64 x 64 diagonal blocks of an upper triangular N x N U
// (one CTA of 64 threads per block, thread j solves column j by back
// substitution in registers; a partial last block is padded with the
// identity).  Zero
// pivot -> bit 1 of *status.  Dinv block b at Dinv + 4096 b, column-major.
template <typename TS, typename T>
__global__ void __launch_bounds__(64)
k_invert_diag64(const TS *__restrict__ U, int ldu, int N, T *__restrict__ Dinv, int *__restrict__ status)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    T *Us = reinterpret_cast<T *>(smem_raw);     // [64][65]
    const int j = threadIdx.x, blk = blockIdx.x, r0 = blk * 64;
    for (int c = 0; c < 64; c++) {
        T v;
        if (r0 + j < N && r0 + c < N) v = j <= c ? (T)U[idx2(r0 + j, r0 + c, ldu)] : T(0);
        else v = j == c ? T(1) : T(0);
        Us[j * 65 + c] = v;
    }
    __syncthreads();
    // column j in registers, recurrence fully unrolled (x[k] = 0 for k > j, so
    // the full-length sums are exact); U entries are warp-broadcast reads
    T xr[64];
    bool zero_pivot = false;
#pragma unroll
    for (int i = 63; i >= 0; i--) {
        T sum = i == j ? T(1) : T(0);
#pragma unroll
        for (int k = i + 1; k < 64; k++) sum = fma(-Us[i * 65 + k], xr[k], sum);
        const T d = Us[i * 65 + i];
        zero_pivot |= d == T(0);
        xr[i] = i <= j ? sum / d : T(0);
    }
    if (zero_pivot && j == 0) atomicOr(status, 2);
#pragma unroll
    for (int i = 0; i < 64; i++) Dinv[(size_t)blk * 4096 + i + 64 * j] = xr[i];
}

template <typename TS, typename T>
void invert_diag64(const TS *U, int ldu, int N, T *Dinv, int *status, cudaStream_t s)
{
    if (N <= 0) return;
    const size_t smem = T64_DS * sizeof(T);
    static PerDeviceOnce once;
    once([&] { cudaFuncSetAttribute(k_invert_diag64<TS, T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem); });
    ProfScope ps(K_TRSV, s);
    k_invert_diag64<TS, T><<<ceil_div(N, 64), 64, smem, s>>>(U, ldu, N, Dinv, status);
}

template <typename T>
__device__ __forceinline__ void t64_load_d(const T *__restrict__ Dinv, int blk, int tid, T (&d)[8])
{
    const T *D = Dinv + (size_t)blk * 4096;
#pragma unroll
    for (int u = 0; u < 8; u++) d[u] = D[tid + u * T64_THREADS];
}

// Stage op(D) row-major (padded): Ds[r * 65 + c] = op(D)(r, c), op = D or D^T.
template <typename T>
__device__ __forceinline__ void t64_store_d(T *Ds, int trans, int tid, const T (&d)[8])
{
#pragma unroll
    for (int u = 0; u < 8; u++) {
        const int e = tid + u * T64_THREADS;     // D(r, c) at r + 64 c
        const int r = e & 63, c = e >> 6;
        if (trans) Ds[c * 65 + r] = d[u]; else Ds[r * 65 + c] = d[u];
    }
}

constexpr uint32_t T64_POLL_LIMIT = 1u << 24;

__device__ __forceinline__ uint32_t t64_smem(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ uint32_t t64_mapa(uint32_t addr, int rank)
{
    uint32_t r;
    asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(r) : "r"(addr), "r"(rank));
    return r;
}

__device__ __forceinline__ void t64_st_async(uint32_t raddr, uint4 v, uint32_t rbar)
{
    asm volatile("st.async.shared::cluster.mbarrier::complete_tx::bytes.v4.b32 [%0], {%1, %2, %3, %4}, [%5];"
                 ::"r"(raddr), "r"(v.x), "r"(v.y), "r"(v.z), "r"(v.w), "r"(rbar) : "memory");
}

// Threads of the owner CTA (warps 0..7) that send a solved block: 16-byte
// pieces, one (destination, piece) pair per thread and round.
constexpr int T64_SENDERS = 256;

// Bounded wait on phase 0 of a step's mbarrier; false on timeout.  try_wait
// parks the warp between polls, so waiting warps do not crowd the shared-
// memory pipe that the owner's products and messages use.
__device__ __forceinline__ bool t64_wait(uint32_t bar)
{
    for (uint32_t it = 0; it < T64_POLL_LIMIT; it++) {
        uint32_t done;
        asm volatile("{\n\t.reg .pred p;\n\t"
                     "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], 0;\n\t"
                     "selp.u32 %0, 1, 0, p;\n\t}"
                     : "=r"(done)
                     : "r"(bar)
                     : "memory");
        if (done) return true;
    }
    return false;
}

// Message passing instead of a cluster barrier per step: the owner of block
// t sends x_t with st.async (16-byte pieces) into slot t of every CTA, which
// signals that CTA's mbarrier t (one slot and one barrier per step, so a fast owner never
// overwrites a slot a slower CTA still reads).  Every CTA waits only for the
// x block it needs next; the chain from one owner to the next is one
// distributed-shared-memory hop.
// TPR threads per row (2 when a CTA owns at most 256 rows): each holds 64 /
// TPR entries of the row's block column and the partial products meet by a
// lane-pair shuffle, so every per-row chain (and the FP64 work of the FP64
// variant) is spread over twice the warps.
template <typename T, int TPR>
__global__ void __launch_bounds__(T64_THREADS, 1)
k_trsv64(const float *__restrict__ U, int ldu, int n, int trans, T *__restrict__ x, int slice,
         const T *__restrict__ Dinv, const float *__restrict__ pack, int npack, int *__restrict__ err)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    __shared__ __align__(16) T xsend[64];
    const int nblk = ceil_div(n, 64);
    unsigned long long *mbar = reinterpret_cast<unsigned long long *>(smem_raw);     // [nblk]
    T *xin = reinterpret_cast<T *>(smem_raw + 8 * ((nblk + 1) & ~1));            // [nblk][64]
    T *Ds = xin + (size_t)nblk * 64;                                             // [2][64 * 65]
    T *xs = Ds + 2 * T64_DS;                                                     // slice
    cg::cluster_group cluster = cg::this_cluster();
    const int cs = (int)cluster.num_blocks();
    const int crank = (int)cluster.block_rank();
    const int tid = threadIdx.x;
    const int s0 = crank * slice;
    const int s1 = min(s0 + slice, n);
    constexpr int CW = 64 / TPR;                             // block-column entries per thread
    const int i = s0 + tid / TPR;                            // this thread's row
    const int c0 = (tid % TPR) * CW;                         // its first column in the block
    for (int t = tid; t < nblk; t += T64_THREADS) {
        const uint32_t b = t64_smem(&mbar[t]);
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(b) : "memory");
        asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(b), "r"((uint32_t)(64 * sizeof(T)))
                     : "memory");
    }
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    cluster.sync();                                          // every barrier armed before any message
    pdl_wait();                                              // x and Dinv come from earlier kernels
    pdl_trigger();
    for (int r = s0 + tid; r < s1; r += T64_THREADS) xs[r - s0] = x[r];
    {
        const int b0 = trans ? 0 : nblk - 1;
        if (crank == (b0 * 64) / slice) {
            T d[8];
            t64_load_d(Dinv, b0, tid, d);
            t64_store_d(Ds, trans, tid, d);
        }
    }
    __syncthreads();
    bool timed_out = false;
    for (int t = 0; t < nblk; t++) {
        const int blk = trans ? t : nblk - 1 - t;
        const int r0 = blk * 64;
        const int bs = min(64, n - r0);
        const int par = t & 1;
        const int owner = r0 / slice;
        T *xt = xin + (size_t)t * 64;
        // 1. this row's entries of the block column (rows still unsolved)
        const int lo = trans ? max(s0, r0 + bs) : s0;
        const int hi = trans ? s1 : min(s1, r0);
        const bool va = i >= lo && i < hi;
        float u[CW];
        if (pack) {
            // packed block column: quad q of row i at [q][row][4]
            const int rows = trans ? t64_rows_t(npack, blk) : r0;
            const int ii = trans ? i - (r0 + 64) : i;
            const float4 *src = reinterpret_cast<const float4 *>(
                pack + (trans ? t64_off_n(ceil_div(npack, 64)) + t64_off_t(npack, blk) : t64_off_n(blk)));
#pragma unroll
            for (int q = 0; q < CW / 4; q++) {
                const float4 v = va ? src[(size_t)(c0 / 4 + q) * rows + ii] : make_float4(0.f, 0.f, 0.f, 0.f);
                u[4 * q] = v.x; u[4 * q + 1] = v.y; u[4 * q + 2] = v.z; u[4 * q + 3] = v.w;
            }
            if (bs < 64) {
                // the partial last block of a leading n x n solve: the pack
                // holds columns past n - 1 (or zeros past N - 1)
#pragma unroll
                for (int c = 0; c < CW; c++)
                    if (c0 + c >= bs) u[c] = 0.f;
            }
        } else if (trans) {
            // U(r0 + c0 + c, i): consecutive entries of column i (16-byte
            // aligned when bs = 64: r0, c0, ldu multiples of 4)
            const float *col = U + (size_t)i * ldu + r0 + c0;
            if (va && bs == 64) {
#pragma unroll
                for (int q = 0; q < CW / 4; q++) {
                    const float4 v = *reinterpret_cast<const float4 *>(col + 4 * q);
                    u[4 * q] = v.x; u[4 * q + 1] = v.y; u[4 * q + 2] = v.z; u[4 * q + 3] = v.w;
                }
            } else {
#pragma unroll
                for (int c = 0; c < CW; c++) u[c] = (va && c0 + c < bs) ? col[c] : 0.f;
            }
        } else {
#pragma unroll
            for (int c = 0; c < CW; c++) u[c] = (va && c0 + c < bs) ? U[idx2(i, r0 + c0 + c, ldu)] : 0.f;
        }
        // next block's inverse, loaded by its owner
        const int nb = t + 1 < nblk ? (trans ? t + 1 : nblk - 2 - t) : -1;
        const bool stage = nb >= 0 && crank == (nb * 64) / slice;
        T dn[8];
        if (stage) t64_load_d(Dinv, nb, tid, dn);
        // 2. the owner forms x_t in a staging buffer, its warps 0..7 meet on
        // a named barrier and send it to every CTA (itself included) in
        // 16-byte pieces
        if (crank == owner) {
            if (tid < 64 * TPR) {
                const int row = tid / TPR, k0 = (tid % TPR) * CW;
                const T *Dr = Ds + par * T64_DS + row * 65 + k0;
                const T *xb = xs + r0 - s0 + k0;
                T acc = T(0);
#pragma unroll 16
                for (int k = 0; k < CW; k++) acc = fma(Dr[k], k0 + k < bs ? xb[k] : T(0), acc);
                if (TPR == 2) acc += __shfl_xor_sync(0xffffffffu, acc, 1);
                if (tid % TPR == 0) xsend[row] = row < bs ? acc : T(0);
            }
            if (tid < T64_SENDERS) {
                asm volatile("bar.sync 1, %0;" ::"n"(T64_SENDERS) : "memory");
                constexpr int NCH = 64 * (int)sizeof(T) / 16;
                const uint32_t dst = t64_smem(xt), bar = t64_smem(&mbar[t]);
                for (int e = tid; e < cs * NCH; e += T64_SENDERS) {
                    const int r = e / NCH, ch = e % NCH;
                    t64_st_async(t64_mapa(dst + 16 * ch, r), reinterpret_cast<const uint4 *>(xsend)[ch],
                                 t64_mapa(bar, r));
                }
            }
        }
        // 3. wait for x_t (after a timeout the remaining steps skip their
        // waits; the error flag reports it)
        if (!timed_out && !t64_wait(t64_smem(&mbar[t]))) timed_out = true;
        // 4. update the unsolved rows (x_t read as 16-byte vectors); the
        // owner stores its block
        {
            T d0 = T(0), d1 = T(0);
            if (va) {
                if constexpr (sizeof(T) == 4) {
#pragma unroll
                    for (int q = 0; q < CW / 4; q++) {
                        const float4 xv = reinterpret_cast<const float4 *>(xt + c0)[q];
                        d0 = fma((T)u[4 * q], (T)xv.x, d0);
                        d1 = fma((T)u[4 * q + 1], (T)xv.y, d1);
                        d0 = fma((T)u[4 * q + 2], (T)xv.z, d0);
                        d1 = fma((T)u[4 * q + 3], (T)xv.w, d1);
                    }
                } else {
#pragma unroll
                    for (int q = 0; q < CW / 2; q++) {
                        const double2 xv = reinterpret_cast<const double2 *>(xt + c0)[q];
                        d0 = fma((T)u[2 * q], (T)xv.x, d0);
                        d1 = fma((T)u[2 * q + 1], (T)xv.y, d1);
                    }
                }
            }
            T dsum = d0 + d1;
            if (TPR == 2) dsum += __shfl_xor_sync(0xffffffffu, dsum, 1);
            if (va && tid % TPR == 0) xs[i - s0] -= dsum;
        }
        if (crank == owner && tid < bs) xs[r0 + tid - s0] = xt[tid];
        if (stage) t64_store_d(Ds + (par ^ 1) * T64_DS, trans, tid, dn);
        __syncthreads();
    }
    for (int r = s0 + tid; r < s1; r += T64_THREADS) x[r] = xs[r - s0];
    if (timed_out && tid == 0) atomicOr(err, 16);
    cluster.sync();   // no CTA leaves while messages to it may be in flight
}

template <typename T>
int trsv64(const float *U, int ldu, int n, int trans, T *x, const T *Dinv, const float *pack, int npack, int *err,
           cudaStream_t s)
{
    if (n <= 0) return 0;
    if (n > T64_MAXN || ldu % 4 || ((uintptr_t)U & 15)) return -1;
    // a pack exists for orders 65 .. T64_MAXN (t64_pack writes none below)
    if (npack < n || npack <= 64 || npack > T64_MAXN || ((uintptr_t)pack & 15)) pack = nullptr;
    const int nblk = ceil_div(n, 64);
    int want = nblk < 16 ? nblk : 16;                      // as many CTAs as the cluster allows
    // barriers, one message slot per step, two staged inverses, the owned rows
    const size_t fixed = 8 * (size_t)((nblk + 1) & ~1) + (size_t)nblk * 64 * sizeof(T) + 2 * T64_DS * sizeof(T);
    static PerDeviceOnce once;
    once([&] {
        for (auto kk : {k_trsv64<T, 1>, k_trsv64<T, 2>}) {
            cudaFuncSetAttribute(kk, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
            cudaFuncSetAttribute(kk, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)(8 * 128 + 128 * 64 * sizeof(T) + 2 * T64_DS * sizeof(T) + T64_THREADS * sizeof(T)));
        }
    });
    int cs = cluster_size_for((const void *)k_trsv64<T, 1>, T64_THREADS,
                              fixed + (size_t)ceil_div(nblk, want) * 64 * sizeof(T), want);
    const int slice = ceil_div(nblk, cs) * 64;
    if (slice > T64_THREADS) return -1;
    cs = ceil_div(n, slice);
    // two threads per row when a CTA owns at most 256 rows (same block size
    // and shared memory, so the cluster size above holds for both)
    auto kern = slice <= T64_THREADS / 2 ? k_trsv64<T, 2> : k_trsv64<T, 1>;
    const size_t smem = fixed + (size_t)slice * sizeof(T);
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(cs, 1, 1);
    cfg.blockDim = dim3(T64_THREADS, 1, 1);
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
    ProfScope ps(K_TRSV, s);
    cudaError_t e = cudaLaunchKernelEx(&cfg, kern, U, ldu, n, trans, x, slice, Dinv, pack, npack, err);
    return e == cudaSuccess ? 0 : MPIR_CUDA_ERROR;
}

template void invert_diag64<float, float>(const float *, int, int, float *, int *, cudaStream_t);
template void invert_diag64<float, double>(const float *, int, int, double *, int *, cudaStream_t);
template int trsv64<float>(const float *, int, int, int, float *, const float *, const float *, int, int *,
                           cudaStream_t);
template int trsv64<double>(const float *, int, int, int, double *, const double *, const float *, int, int *,
                            cudaStream_t);

} // namespace mpir
