// gemm_tc.cu -- tcgen05 (5th-generation tensor core) GEMM used by the
// trailing updates of the blocked Householder factorizations (xLARFB with a
// 128-reflector block):
//     D (M x N) = A (M x K) * B (N x K)^T,   A and B K-major FP32 in global,
// operands staged by TMA into 128-byte-swizzled shared memory, accumulator
// in TMEM, read back with tcgen05.ld for the epilogue.
//
// Precision modes
//   TF32   : one kind::tf32 MMA per K step (inputs truncated to TF32).
//   BF16   : FP32 tiles (two 32-wide K halves per 64-wide stage) rounded to
//            bfloat16 (nearest even) in shared memory by the epilogue warps,
//            written in the same 128-byte-swizzled K-major layout, then four
//            kind::f16 MMAs (BF16 x BF16 -> FP32) per stage.
//   TF32X3 : FP32-class accuracy from three TF32 MMAs per K step,
//            a_hi b_hi + a_hi b_lo + a_lo b_hi, with x = x_hi + x_lo,
//            x_hi = TF32(x) (round to nearest), x_lo = x - x_hi.
//            A is supplied pre-split (two tensor maps); B is either
//            pre-split or split in shared memory by the epilogue warps.
// Epilogues
//   STORE : P[split] = D            (split-K partials of W = V^T C)
//   SUB   : C -= D                  (C <- C - V W)
//
// Warp roles (192 threads): warp 0 = TMA producer, warp 1 = TMEM owner and
// MMA issuer, warps 2..5 = B-split converters and the epilogue warpgroup.
// Every mbarrier wait is bounded; on timeout the CTA records an error flag,
// skips the remaining work, frees its TMEM and returns.
#include <cuda.h>
#include <cudaTypedefs.h>

#include "common.cuh"
#include "gemm_tc.h"
#include "kernels.h"
#include "mpir.h"

namespace mpir {

constexpr int TC_BM = 128;
constexpr int TC_BN = 128;
constexpr int TC_BK = 32;                         // 32 FP32 = one 128-byte swizzle row
constexpr int TC_TILE_A = TC_BM * TC_BK * 4;      // 16 KB
constexpr int TC_TILE_B = TC_BN * TC_BK * 4;      // 16 KB
constexpr int TC_THREADS = 192;
constexpr int TC_BK16 = 64;                       // K per BF16 stage: 64 BF16 = one 128-byte swizzle row
constexpr uint32_t TC_WAIT_LIMIT = 1u << 22;

// ------------------------------------------------------------------ PTX --

__device__ __forceinline__ uint32_t smem_u32(const void *p)
{
    return (uint32_t)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ void mbar_init(uint32_t bar, uint32_t count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count) : "memory");
}

__device__ __forceinline__ void mbar_expect_tx(uint32_t bar, uint32_t bytes)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes) : "memory");
}

__device__ __forceinline__ void mbar_arrive(uint32_t bar)
{
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(bar) : "memory");
}

// Bounded wait for the phase of parity `parity` to complete.
__device__ __forceinline__ bool mbar_wait(uint32_t bar, uint32_t parity)
{
    for (uint32_t it = 0; it < TC_WAIT_LIMIT; it++) {
        uint32_t done;
        asm volatile("{\n\t.reg .pred p;\n\t"
                     "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
                     "selp.u32 %0, 1, 0, p;\n\t}"
                     : "=r"(done)
                     : "r"(bar), "r"(parity)
                     : "memory");
        if (done) return true;
    }
    return false;
}

__device__ __forceinline__ void tma_load_2d(uint32_t dst, const CUtensorMap *tm, int x, int y, uint32_t bar)
{
    asm volatile("cp.async.bulk.tensor.2d.shared::cluster.global.tile.mbarrier::complete_tx::bytes"
                 " [%0], [%1, {%2, %3}], [%4];" ::"r"(dst),
                 "l"((uint64_t)tm), "r"(x), "r"(y), "r"(bar)
                 : "memory");
}

__device__ __forceinline__ void fence_proxy_async_smem()
{
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

// Shared-memory matrix descriptor: K-major operand, 128-byte swizzle,
// 8-row core-matrix groups 1024 bytes apart (SBO), version 1 (tcgen05).
__device__ __forceinline__ uint64_t sdesc_sw128(uint32_t saddr)
{
    uint64_t d = 0;
    d |= (uint64_t)((saddr & 0x3FFFFu) >> 4);
    d |= (uint64_t)(16u >> 4) << 16;       // LBO (not used by swizzled K-major)
    d |= (uint64_t)(1024u >> 4) << 32;     // SBO
    d |= (uint64_t)1 << 46;                // descriptor version for tcgen05
    d |= (uint64_t)2 << 61;                // SWIZZLE_128B
    return d;
}

// Instruction descriptor, kind::tf32: D = F32, A = B = TF32, both K-major.
__host__ __device__ constexpr uint32_t idesc_tf32(int M, int N)
{
    return (1u << 4) | (2u << 7) | (2u << 10) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}

// Instruction descriptor, kind::f16 with BF16 A and B: D = F32, both K-major.
__host__ __device__ constexpr uint32_t idesc_bf16(int M, int N)
{
    return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}

__device__ __forceinline__ void mma_bf16(uint32_t tmem_d, uint64_t ad, uint64_t bd, uint32_t idesc, uint32_t acc)
{
    asm volatile("{\n\t.reg .pred p;\n\t"
                 "setp.ne.b32 p, %4, 0;\n\t"
                 "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(tmem_d),
                 "l"(ad), "l"(bd), "r"(idesc), "r"(acc)
                 : "memory");
}

// Two floats rounded to nearest-even bfloat16, packed with lo at the lower
// address.
__device__ __forceinline__ uint32_t pack_bf16x2(float lo, float hi)
{
    uint32_t r;
    asm("cvt.rn.bf16x2.f32 %0, %1, %2;" : "=r"(r) : "f"(hi), "f"(lo));
    return r;
}

// One FP32 operand tile pair (K halves 0..31, 32..63, 128 rows, 128-byte
// swizzle) -> the BF16 tile (128 rows x 64, 128-byte swizzle).  Thread et of
// the 128 converters handles 16-byte output chunks e = et, et + 128, ...:
// row r = e / 8, chunk j = e % 8 (BF16 k = 8j .. 8j+7), read from FP32 half
// j / 4, chunks 2 (j % 4) and 2 (j % 4) + 1.  In a 128-byte-swizzled tile
// chunk c of row r sits at chunk c ^ (r % 8).
__device__ __forceinline__ void convert_tile_bf16(const unsigned char *src0, const unsigned char *src1,
                                                  unsigned char *dst, int et)
{
#pragma unroll 2
    for (int e = et; e < 128 * 8; e += 128) {
        const int r = e >> 3, j = e & 7, x = r & 7;
        const unsigned char *src = (j < 4 ? src0 : src1) + r * 128;
        const int c0 = 2 * (j & 3);
        const float4 u = *reinterpret_cast<const float4 *>(src + ((c0 ^ x) << 4));
        const float4 v = *reinterpret_cast<const float4 *>(src + (((c0 + 1) ^ x) << 4));
        uint4 o;
        o.x = pack_bf16x2(u.x, u.y);
        o.y = pack_bf16x2(u.z, u.w);
        o.z = pack_bf16x2(v.x, v.y);
        o.w = pack_bf16x2(v.z, v.w);
        *reinterpret_cast<uint4 *>(dst + r * 128 + ((j ^ x) << 4)) = o;
    }
}

__device__ __forceinline__ void mma_tf32(uint32_t tmem_d, uint64_t ad, uint64_t bd, uint32_t idesc, uint32_t acc)
{
    asm volatile("{\n\t.reg .pred p;\n\t"
                 "setp.ne.b32 p, %4, 0;\n\t"
                 "tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n\t}" ::"r"(tmem_d),
                 "l"(ad), "l"(bd), "r"(idesc), "r"(acc)
                 : "memory");
}

__device__ __forceinline__ void mma_commit(uint32_t bar)
{
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(bar)
                 : "memory");
}

__device__ __forceinline__ void tmem_ld32(uint32_t taddr, float (&v)[32])
{
    uint32_t r[32];
    asm volatile("tcgen05.ld.sync.aligned.32x32b.x32.b32 "
                 "{%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, %15, "
                 "%16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, %28, %29, %30, %31}, [%32];"
                 : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
                   "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]),
                   "=r"(r[14]), "=r"(r[15]), "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]),
                   "=r"(r[21]), "=r"(r[22]), "=r"(r[23]), "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]),
                   "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
                 : "r"(taddr));
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
    for (int j = 0; j < 32; j++) v[j] = __uint_as_float(r[j]);
}

__device__ __forceinline__ float tf32_round(float x)
{
    uint32_t r;
    asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
    return __uint_as_float(r);
}

// ---------------------------------------------------------------- kernel --
//
// Grid: (ceil(N / BN), ceil(M / BM), nsplit).  K steps of BK are distributed
// over blockIdx.z: split z handles steps [z*kps, min((z+1)*kps, ksteps)).
// Tensor-map coordinates: A tile (m, k) at (a_x0 + k*BK, a_y0 + m*BM); B tile
// at (b_x0 + k*BK, b_y0 + n*BN).
struct TcArgs {
    int a_x0, a_y0, b_x0, b_y0;
    int M, N;                 // valid extent of D
    int ksteps, kps;          // total K steps, steps per split
    float *out;               // STORE: out + z*split_stride ; SUB: C
    int ldo;
    size_t split_stride;
    int *err;
};

template <int MODE, int BSPLIT, int EPI, int STAGES>
__global__ void __launch_bounds__(TC_THREADS, 1)
k_gemm_tc(const __grid_constant__ CUtensorMap tmA, const __grid_constant__ CUtensorMap tmA2,
          const __grid_constant__ CUtensorMap tmB, const __grid_constant__ CUtensorMap tmB2, TcArgs args)
{
    // A_lo / B_lo buffers exist only for TF32X3; BF16 stages hold two FP32
    // K halves of A and of B plus the BF16 tiles of A and B
    constexpr bool BF = MODE == TCM_BF16;
    constexpr int NA = MODE == TCM_TF32X3 || BF ? 2 : 1;
    constexpr int NBUF = MODE == TCM_TF32X3 || BF ? 2 : 1;
    constexpr int STAGE_BYTES = NA * TC_TILE_A + NBUF * TC_TILE_B + (BF ? TC_TILE_A + TC_TILE_B : 0);
    constexpr int KSTEP = BF ? TC_BK16 : TC_BK;
    constexpr int NCONV = 128;   // converter / epilogue threads

    extern __shared__ __align__(1024) unsigned char smem_dyn[];
    // 1024-byte alignment for the swizzled tiles
    unsigned char *smem = (unsigned char *)(((uintptr_t)smem_dyn + 1023) & ~(uintptr_t)1023);
    __shared__ __align__(8) uint64_t bar_full[STAGES], bar_ready[STAGES], bar_empty[STAGES], bar_accum;
    __shared__ uint32_t tmem_base_s;
    __shared__ int abort_s;

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int n_tile = blockIdx.x, m_tile = blockIdx.y, z = blockIdx.z;
    const int k_begin = z * args.kps;
    const int k_end = min(args.ksteps, k_begin + args.kps);
    const int nk = k_end - k_begin;

    if (threadIdx.x == 0) {
        for (int s = 0; s < STAGES; s++) {
            mbar_init(smem_u32(&bar_full[s]), 1);
            mbar_init(smem_u32(&bar_ready[s]), NCONV);
            mbar_init(smem_u32(&bar_empty[s]), 1);
        }
        mbar_init(smem_u32(&bar_accum), 1);
        abort_s = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    // (no-op under an ordinary launch) the previous kernel's outputs are read
    // only after this wait; no tensor memory is held while waiting
    pdl_wait();
    if (warp == 1) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&tmem_base_s)),
                     "r"((uint32_t)TC_BN)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = tmem_base_s;

    auto tileA = [&](int s) { return smem + (size_t)s * STAGE_BYTES; };
    auto tileA2 = [&](int s) { return smem + (size_t)s * STAGE_BYTES + TC_TILE_A; };
    auto tileB = [&](int s) { return smem + (size_t)s * STAGE_BYTES + NA * TC_TILE_A; };
    auto tileB2 = [&](int s) { return smem + (size_t)s * STAGE_BYTES + NA * TC_TILE_A + TC_TILE_B; };
    auto tileAb = [&](int s) { return smem + (size_t)s * STAGE_BYTES + NA * TC_TILE_A + NBUF * TC_TILE_B; };
    auto tileBb = [&](int s) { return tileAb(s) + TC_TILE_A; };

    int issued = 0;   // TMA stages issued by the producer (lane 0 of warp 0)
    if (warp == 0) {
        // ------------------------------------------------ TMA producer
        if (lane == 0) {
            const bool b_two = (MODE == TCM_TF32X3 && BSPLIT == 0) || BF;
            const uint32_t bytes = (uint32_t)(NA * TC_TILE_A + (b_two ? 2 : 1) * TC_TILE_B);
            for (int i = 0; i < nk; i++) {
                const int s = i % STAGES;
                if (!mbar_wait(smem_u32(&bar_empty[s]), ((i / STAGES) + 1) & 1)) { atomicOr(args.err, 4); abort_s = 1; break; }
                if (*(volatile int *)&abort_s) break;
                const uint32_t fb = smem_u32(&bar_full[s]);
                mbar_expect_tx(fb, bytes);
                const int kx = (k_begin + i) * KSTEP;
                tma_load_2d(smem_u32(tileA(s)), &tmA, args.a_x0 + kx, args.a_y0 + m_tile * TC_BM, fb);
                if (MODE == TCM_TF32X3)
                    tma_load_2d(smem_u32(tileA2(s)), &tmA2, args.a_x0 + kx, args.a_y0 + m_tile * TC_BM, fb);
                if (BF)       // the second K half of A (same map, 32 further along K)
                    tma_load_2d(smem_u32(tileA2(s)), &tmA, args.a_x0 + kx + TC_BK, args.a_y0 + m_tile * TC_BM, fb);
                tma_load_2d(smem_u32(tileB(s)), &tmB, args.b_x0 + kx, args.b_y0 + n_tile * TC_BN, fb);
                if (BF)
                    tma_load_2d(smem_u32(tileB2(s)), &tmB, args.b_x0 + kx + TC_BK, args.b_y0 + n_tile * TC_BN, fb);
                else if (b_two)
                    tma_load_2d(smem_u32(tileB2(s)), &tmB2, args.b_x0 + kx, args.b_y0 + n_tile * TC_BN, fb);
                issued = i + 1;
            }
        }
    } else if (warp == 1) {
        // ------------------------------------------------ MMA issuer
        if (lane == 0) {
            constexpr uint32_t IDESC = BF ? idesc_bf16(TC_BM, TC_BN) : idesc_tf32(TC_BM, TC_BN);
            const bool wait_ready = (MODE == TCM_TF32X3 && BSPLIT == 1) || BF;
            for (int i = 0; i < nk; i++) {
                const int s = i % STAGES;
                const uint32_t par = (i / STAGES) & 1;
                bool ok = mbar_wait(smem_u32(wait_ready ? &bar_ready[s] : &bar_full[s]), par);
                if (!ok || *(volatile int *)&abort_s) { if (!ok) atomicOr(args.err, 4); abort_s = 1; break; }
                tc_fence_after();
                const uint32_t a0 = smem_u32(tileA(s)), b0 = smem_u32(tileB(s));
                const uint32_t a1 = smem_u32(tileA2(s)), b1 = smem_u32(tileB2(s));
                if (BF) {
                    const uint32_t ab = smem_u32(tileAb(s)), bb = smem_u32(tileBb(s));
#pragma unroll
                    for (int ks = 0; ks < TC_BK16 / 16; ks++) {
                        const uint32_t off = ks * 32;    // 16 BF16 = 32 bytes along K
                        mma_bf16(tmem, sdesc_sw128(ab + off), sdesc_sw128(bb + off), IDESC,
                                 (i > 0 || ks > 0) ? 1u : 0u);
                    }
                    mma_commit(smem_u32(&bar_empty[s]));
                    continue;
                }
#pragma unroll
                for (int ks = 0; ks < TC_BK / 8; ks++) {
                    const uint32_t off = ks * 32;    // 8 TF32 = 32 bytes along K
                    const uint32_t acc = (i > 0 || ks > 0) ? 1u : 0u;
                    mma_tf32(tmem, sdesc_sw128(a0 + off), sdesc_sw128(b0 + off), IDESC, acc);
                    if (MODE == TCM_TF32X3) {
                        mma_tf32(tmem, sdesc_sw128(a0 + off), sdesc_sw128(b1 + off), IDESC, 1u);
                        mma_tf32(tmem, sdesc_sw128(a1 + off), sdesc_sw128(b0 + off), IDESC, 1u);
                    }
                }
                mma_commit(smem_u32(&bar_empty[s]));
            }
            mma_commit(smem_u32(&bar_accum));
        }
    } else {
        // ------------------------------------------------ B split + epilogue
        const int et = threadIdx.x - 64;              // 0..127
        if (BF) {
            for (int i = 0; i < nk; i++) {
                const int s = i % STAGES;
                if (!mbar_wait(smem_u32(&bar_full[s]), (i / STAGES) & 1)) { atomicOr(args.err, 4); abort_s = 1; break; }
                convert_tile_bf16(tileA(s), tileA2(s), tileAb(s), et);
                convert_tile_bf16(tileB(s), tileB2(s), tileBb(s), et);
                fence_proxy_async_smem();
                mbar_arrive(smem_u32(&bar_ready[s]));
            }
        }
        if (MODE == TCM_TF32X3 && BSPLIT == 1) {
            for (int i = 0; i < nk; i++) {
                const int s = i % STAGES;
                if (!mbar_wait(smem_u32(&bar_full[s]), (i / STAGES) & 1)) { atomicOr(args.err, 4); abort_s = 1; break; }
                float4 *hi = reinterpret_cast<float4 *>(tileB(s));
                float4 *lo = reinterpret_cast<float4 *>(tileB2(s));
#pragma unroll 4
                for (int e = et; e < TC_TILE_B / 16; e += NCONV) {
                    float4 v = hi[e], h, l;
                    // low parts rounded to nearest TF32 (the MMA would truncate them)
                    h.x = tf32_round(v.x); l.x = tf32_round(v.x - h.x);
                    h.y = tf32_round(v.y); l.y = tf32_round(v.y - h.y);
                    h.z = tf32_round(v.z); l.z = tf32_round(v.z - h.z);
                    h.w = tf32_round(v.w); l.w = tf32_round(v.w - h.w);
                    hi[e] = h;
                    lo[e] = l;
                }
                fence_proxy_async_smem();
                mbar_arrive(smem_u32(&bar_ready[s]));
            }
        }
        // epilogue: warp q = warp % 4 owns TMEM lanes (rows) 32q .. 32q+31
        bool ok = nk > 0 && mbar_wait(smem_u32(&bar_accum), 0);
        ok = __all_sync(0xffffffffu, ok);        // tcgen05.ld below is warp-collective
        if (!ok && nk > 0 && lane == 0) { atomicOr(args.err, 4); abort_s = 1; }
        tc_fence_after();
        const int q = warp & 3;
        const int row = m_tile * TC_BM + 32 * q + lane;
        if (ok) {
#pragma unroll 1
            for (int c0 = 0; c0 < TC_BN; c0 += 32) {
                // SUB: issue the 32 loads of C first (independent, coalesced
                // across the warp), then read the accumulator and store
                float cv[32];
                if (EPI == TCE_SUB) {
#pragma unroll
                    for (int j = 0; j < 32; j++) {
                        const int col = n_tile * TC_BN + c0 + j;
                        cv[j] = (row < args.M && col < args.N) ? args.out[(size_t)col * args.ldo + row] : 0.f;
                    }
                }
                float v[32];
                tmem_ld32(tmem + ((uint32_t)(32 * q) << 16) + (uint32_t)c0, v);
                if (row < args.M) {
#pragma unroll
                    for (int j = 0; j < 32; j++) {
                        const int col = n_tile * TC_BN + c0 + j;
                        if (col < args.N) {
                            if (EPI == TCE_STORE)
                                args.out[(size_t)z * args.split_stride + (size_t)col * args.ldo + row] = v[j];
                            else
                                args.out[(size_t)col * args.ldo + row] = cv[j] - v[j];
                        }
                    }
                }
            }
        } else if (EPI == TCE_STORE && nk <= 0) {
            // an empty split contributes zeros
            if (row < args.M)
                for (int j = 0; j < TC_BN; j++) {
                    const int col = n_tile * TC_BN + j;
                    if (col < args.N) args.out[(size_t)z * args.split_stride + (size_t)col * args.ldo + row] = 0.f;
                }
        }
    }
    tc_fence_before();
    __syncthreads();
    if (warp == 0 && lane == 0 && *(volatile int *)&abort_s) {
        // after an abort, wait (bounded) for TMA copies still landing in the
        // stages that were issued but never consumed
        for (int i = issued > STAGES ? issued - STAGES : 0; i < issued; i++)
            mbar_wait(smem_u32(&bar_full[i % STAGES]), (i / STAGES) & 1);
    }
    if (warp == 1) {
        tc_fence_after();
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"((uint32_t)TC_BN)
                     : "memory");
    }
}

// ------------------------------------------------------------------ host --

static PFN_cuTensorMapEncodeTiled_v12000 encode_fn()
{
    static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
    if (!fn) {
        cudaDriverEntryPointQueryResult q;
        void *p = nullptr;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = (PFN_cuTensorMapEncodeTiled_v12000)p;
    }
    return fn;
}

// Tensor map of a column-major FP32 matrix (rows contiguous, ld in elements)
// with a box of 32 rows x box_cols columns and 128-byte swizzle.
int tmap_colmajor(CUtensorMap *tm, const float *base, long rows, long cols, long ld, int box_cols)
{
    auto fn = encode_fn();
    if (!fn) return MPIR_CUDA_ERROR;
    if (((uintptr_t)base & 15) || (ld * 4) % 16) return MPIR_UNSUP();
    cuuint64_t gdim[2] = {(cuuint64_t)rows, (cuuint64_t)cols};
    cuuint64_t gstr[1] = {(cuuint64_t)ld * 4};
    cuuint32_t box[2] = {(cuuint32_t)TC_BK, (cuuint32_t)box_cols};
    cuuint32_t estr[2] = {1, 1};
    CUresult r = fn(tm, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, (void *)base, gdim, gstr, box, estr,
                    CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                    CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    return r == CUDA_SUCCESS ? 0 : MPIR_UNSUPPORTED;
}

template <int MODE, int BSPLIT, int EPI>
static int launch_tc(const CUtensorMap &A, const CUtensorMap &A2, const CUtensorMap &B, const CUtensorMap &B2,
                     const TcArgs &args, int ntn, int ntm, int nsplit, cudaStream_t s)
{
    constexpr bool BF = MODE == TCM_BF16;
    // C -= D (K = 128: four K steps) keeps one or two stages, so that two CTAs
    // share an SM and one's C read / write epilogue overlaps the other's
    // loads and MMAs; the split-K products keep a deep pipeline
    constexpr int STAGES = EPI == TCE_SUB ? (MODE == TCM_TF32 ? 2 : 1) : (MODE == TCM_TF32X3 ? 3 : (BF ? 2 : 5));
    constexpr int NA = MODE == TCM_TF32X3 || BF ? 2 : 1;
    constexpr int NBUF = MODE == TCM_TF32X3 || BF ? 2 : 1;
    const size_t smem =
        (size_t)STAGES * (NA * TC_TILE_A + NBUF * TC_TILE_B + (BF ? TC_TILE_A + TC_TILE_B : 0)) + 1024;
    auto kern = k_gemm_tc<MODE, BSPLIT, EPI, STAGES>;
    static PerDeviceOnce once;
    once([&] { cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem); });
    ProfScope ps(K_LARFB_TC, s);
    // ordinary launch: a waiting grid of this size would hold every SM
    kern<<<dim3(ntn, ntm, nsplit), TC_THREADS, smem, s>>>(A, A2, B, B2, args);
    return cudaGetLastError() == cudaSuccess ? 0 : MPIR_CUDA_ERROR;
}

// D = A B^T over K (A: M x K via tmA[/tmA2], B: N x K via tmB[/tmB2]).
int gemm_tc(int mode, int bsplit, int epi, const CUtensorMap &A, const CUtensorMap &A2, const CUtensorMap &B,
            const CUtensorMap &B2, int a_x0, int a_y0, int b_x0, int b_y0, int M, int N, int K, float *out,
            int ldo, size_t split_stride, int nsplit, int *err, cudaStream_t s)
{
    if (M <= 0 || N <= 0) return 0;
    TcArgs a;
    a.a_x0 = a_x0; a.a_y0 = a_y0; a.b_x0 = b_x0; a.b_y0 = b_y0;
    a.M = M; a.N = N;
    a.ksteps = ceil_div(K, mode == TCM_BF16 ? TC_BK16 : TC_BK);
    if (nsplit < 1) nsplit = 1;
    if (nsplit > a.ksteps) nsplit = a.ksteps > 0 ? a.ksteps : 1;
    a.kps = ceil_div(a.ksteps, nsplit);
    a.out = out; a.ldo = ldo; a.split_stride = split_stride; a.err = err;
    const int ntn = ceil_div(N, TC_BN), ntm = ceil_div(M, TC_BM);
    if (mode == TCM_TF32X3) {
        if (epi == TCE_STORE)
            return bsplit ? launch_tc<TCM_TF32X3, 1, TCE_STORE>(A, A2, B, B2, a, ntn, ntm, nsplit, s)
                          : launch_tc<TCM_TF32X3, 0, TCE_STORE>(A, A2, B, B2, a, ntn, ntm, nsplit, s);
        return bsplit ? launch_tc<TCM_TF32X3, 1, TCE_SUB>(A, A2, B, B2, a, ntn, ntm, nsplit, s)
                      : launch_tc<TCM_TF32X3, 0, TCE_SUB>(A, A2, B, B2, a, ntn, ntm, nsplit, s);
    }
    if (mode == TCM_BF16) {
        if (epi == TCE_STORE) return launch_tc<TCM_BF16, 0, TCE_STORE>(A, A2, B, B2, a, ntn, ntm, nsplit, s);
        return launch_tc<TCM_BF16, 0, TCE_SUB>(A, A2, B, B2, a, ntn, ntm, nsplit, s);
    }
    if (epi == TCE_STORE) return launch_tc<TCM_TF32, 0, TCE_STORE>(A, A2, B, B2, a, ntn, ntm, nsplit, s);
    return launch_tc<TCM_TF32, 0, TCE_SUB>(A, A2, B, B2, a, ntn, ntm, nsplit, s);
}

} // namespace mpir
