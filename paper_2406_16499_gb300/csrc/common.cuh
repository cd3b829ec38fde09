// common.cuh -- device helpers shared by the libmpir kernels (sm_103a).
#pragma once

#include <cuda_runtime.h>
#include <cooperative_groups.h>
#include <atomic>
#include <cstdint>
#include <cstddef>
#include <mutex>
#include <utility>
#include <vector>

namespace mpir {

namespace cg = cooperative_groups;

// Where the last MPIR_UNSUPPORTED of this host thread came from (a launch
// shape or size limit of a kernel's host code); the public entry points put
// it into the handle's message when nothing more specific was recorded.
inline const char *&unsupported_where()
{
    static thread_local const char *where = nullptr;
    return where;
}
#define MPIR_STR2(x) #x
#define MPIR_STR(x) MPIR_STR2(x)
#define MPIR_UNSUP() (::mpir::unsupported_where() = __FILE__ ":" MPIR_STR(__LINE__), MPIR_UNSUPPORTED)

// Function attributes (dynamic shared-memory limit, non-portable cluster
// size) belong to the device that is current when they are set.  A launcher
// keeps one of these per kernel and passes it the set-up: it runs the first
// time each device (0..63; every time on higher ordinals) launches, from any
// host thread; running it twice is harmless.
class PerDeviceOnce {
  public:
    template <typename F>
    void operator()(F &&fn)
    {
        int dev = 0;
        if (cudaGetDevice(&dev) != cudaSuccess) { cudaGetLastError(); dev = 0; }
        if (dev < 0 || dev >= 64) { fn(); return; }
        const unsigned long long bit = 1ull << dev;
        if (done_.load(std::memory_order_acquire) & bit) return;
        fn();
        done_.fetch_or(bit, std::memory_order_acq_rel);
    }

  private:
    std::atomic<unsigned long long> done_{0};
};

// Device-side error word (bit flags) written by kernels that give up a
// bounded wait; the host reads it after synchronising.
enum : int { DEV_ERR_BARRIER_TIMEOUT = 1 };

// Grid-wide barrier for a grid whose blocks are all co-resident (launched
// with cudaLaunchCooperativeKernel).  Sense via a generation counter.
// Every wait is bounded: after ~2^22 polls (about a second) the block sets
// DEV_ERR_BARRIER_TIMEOUT in *err and returns false; callers then return.
struct GridBarrier {
    unsigned int *state;   // [0] arrivals, [1] generation
    int *err;
};

__device__ __forceinline__ unsigned ld_acquire_u32(const unsigned *p)
{
    unsigned v;
    asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

__device__ __forceinline__ bool grid_sync(const GridBarrier &b, unsigned nblocks)
{
    __shared__ int s_ok;
    __syncthreads();
    if (threadIdx.x == 0) {
        int ok = 1;
        unsigned gen = ld_acquire_u32(&b.state[1]);
        __threadfence();
        unsigned arrived = atomicAdd(&b.state[0], 1u) + 1u;
        if (arrived == nblocks) {
            atomicExch(&b.state[0], 0u);
            __threadfence();
            atomicAdd(&b.state[1], 1u);
        } else {
            unsigned spins = 0;
            while (ld_acquire_u32(&b.state[1]) == gen) {
                if (++spins > (1u << 22)) { atomicOr(b.err, DEV_ERR_BARRIER_TIMEOUT); ok = 0; break; }
                __nanosleep(64);
            }
        }
        __threadfence();
        s_ok = ok;
    }
    __syncthreads();
    return s_ok != 0;
}

// ---------------------------------------------------------------- warps --

template <typename T>
__device__ __forceinline__ T warp_sum(T v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// Sum V per-lane values (V a power of two <= 32) over the warp.  On return
// every lane l holds in v[0] the warp total of slot (l % V).  Uses
// (V - 1) + log2(32 / V) shuffles (recursive halving exchange).
template <typename T, int V>
__device__ __forceinline__ T warp_transpose_reduce(T (&v)[V])
{
    const int lane = threadIdx.x & 31;
#pragma unroll
    for (int s = V / 2; s >= 1; s >>= 1) {
        const bool upper = (lane & s) != 0;
#pragma unroll
        for (int i = 0; i < s; i++) {
            T send = upper ? v[i] : v[i + s];
            T keep = upper ? v[i + s] : v[i];
            T recv = __shfl_xor_sync(0xffffffffu, send, s);
            v[i] = keep + recv;
        }
    }
    T r = v[0];
#pragma unroll
    for (int o = V; o < 32; o <<= 1) r += __shfl_xor_sync(0xffffffffu, r, o);
    return r;
}

// -------------------------------------------- programmatic dependent launch --
// A kernel launched with pdl_launch (or the ProgrammaticStreamSerialization
// attribute) may start while the previous kernel on its stream is still
// running: it must call pdl_wait() before touching anything that kernel
// writes (pdl_wait returns once the previous grid has completed and its
// memory is visible).  pdl_trigger() lets the next such kernel begin
// launching; both are no-ops for a kernel launched the ordinary way.
__device__ __forceinline__ void pdl_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }
__device__ __forceinline__ void pdl_trigger() { asm volatile("griddepcontrol.launch_dependents;" ::: "memory"); }

template <typename... KArgs, typename... Args>
inline cudaError_t pdl_launch(void (*kern)(KArgs...), dim3 grid, dim3 block, size_t smem, cudaStream_t s,
                              Args &&...args)
{
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = grid;
    cfg.blockDim = block;
    cfg.dynamicSmemBytes = smem;
    cfg.stream = s;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    at[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, kern, std::forward<Args>(args)...);
}

// ------------------------------------------------------------- helpers --

__host__ __device__ __forceinline__ int ceil_div(int a, int b) { return (a + b - 1) / b; }
__host__ __device__ __forceinline__ size_t idx2(int i, int j, int ld)
{
    return (size_t)j * (size_t)ld + (size_t)i;
}

// Largest power-of-two cluster size <= want that the device can schedule for
// `kern` with this block size and dynamic shared memory.
// The occupancy query costs far more host time than a launch, so its answer
// is cached per (kernel, block size, shared memory, wanted size, device).
struct ClusterKey {
    const void *kern;
    int threads, want, device;
    size_t smem;
};

inline int cluster_size_query(const void *kern, int threads, size_t smem, int want);

inline int cluster_size_for(const void *kern, int threads, size_t smem, int want)
{
    if (want <= 1) return 1;
    static std::mutex mu;
    static std::vector<std::pair<ClusterKey, int>> cache;
    int dev = 0;
    cudaGetDevice(&dev);
    {
        std::lock_guard<std::mutex> lk(mu);
        for (const auto &e : cache)
            if (e.first.kern == kern && e.first.threads == threads && e.first.want == want &&
                e.first.device == dev && e.first.smem == smem)
                return e.second;
    }
    const int c = cluster_size_query(kern, threads, smem, want);
    std::lock_guard<std::mutex> lk(mu);
    if (cache.size() < 4096) cache.push_back({ClusterKey{kern, threads, want, dev, smem}, c});
    return c;
}

inline int cluster_size_query(const void *kern, int threads, size_t smem, int want)
{
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(want, 1, 1);
    cfg.blockDim = dim3(threads, 1, 1);
    cfg.dynamicSmemBytes = smem;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = want;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    int maxc = 0;
    if (cudaOccupancyMaxPotentialClusterSize(&maxc, kern, &cfg) != cudaSuccess) { cudaGetLastError(); maxc = 8; }
    int c = 1;
    while (c * 2 <= want && c * 2 <= maxc) c *= 2;
    return c;
}

template <typename T> struct Lim;
template <> struct Lim<float> { static constexpr float eps = 5.9604645e-08f; };
template <> struct Lim<double> { static constexpr double eps = 1.1102230246251565e-16; };

} // namespace mpir
