// noalloc.cu -- an entry point of the GLS residual that never allocates.
//
// mpir_gls_residual needs scratch for the partial sums of its two dual
// gemvs; it takes that scratch from its handle, which grows it with
// cudaMalloc.  Some callers cannot call cudaMalloc at all: plug-ins of
// frameworks that own every device allocation through their own pool and
// forbid others after start-up, and real-time loops that must not block in
// the driver's allocator.  For them this file keeps the
// scratch in a fixed file-scope __device__ array that exists as soon as the
// library is loaded on a device, and mpir_gls_residual_noalloc uses only
// that array, the caller's buffers and the caller's stream.
#include <atomic>
#include <cstdio>

#include "common.cuh"
#include "kernels.h"
#include "mpir.h"

namespace mpir {

// Partial sums of W x, W^T z, V y, V^T z plus the norm partials.  Every
// device that loads the library holds these 4 MiB until the process exits.
constexpr size_t NOALLOC_SCRATCH_DOUBLES = (size_t)1 << 19;
static __device__ __align__(256) double g_noalloc_scratch[NOALLOC_SCRATCH_DOUBLES];

// Device address of g_noalloc_scratch, looked up once per device (with that
// device current).  Host threads may race on a device's first call: each
// looks the same address up and stores it atomically, so every reader sees
// either nothing (and looks it up itself) or the address.
constexpr int NOALLOC_MAX_DEVICES = 64;
static std::atomic<double *> g_scratch_ptr[NOALLOC_MAX_DEVICES];

static int noalloc_scratch(double **out)
{
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= NOALLOC_MAX_DEVICES) return MPIR_CUDA_ERROR;
    double *cached = g_scratch_ptr[dev].load(std::memory_order_acquire);
    if (!cached) {
        void *p = nullptr;
        if (cudaGetSymbolAddress(&p, g_noalloc_scratch) != cudaSuccess || !p) {
            cudaGetLastError();
            return MPIR_CUDA_ERROR;
        }
        cached = (double *)p;
        g_scratch_ptr[dev].store(cached, std::memory_order_release);
    }
    *out = cached;
    return 0;
}

} // namespace mpir

using namespace mpir;

extern "C" int mpir_gls_residual_noalloc(int n, int m, int p, const double *W, int ldw, const double *V, int ldv,
                                         const double *d, const double *x, const double *y, const double *z,
                                         double *f1, double *f2, double *f3, double *norms2, void *stream)
{
    if (n < 1) return -1;
    if (m < 0 || m > n) return -2;
    if (p < 0 || n > m + p) return -3;
    if ((m > 0 && !W) || ldw < n) return -5;
    if ((p > 0 && !V) || ldv < n) return -7;
    if (!d || (m > 0 && !x) || (p > 0 && !y) || !z) return -8;
    if ((p > 0 && !f1) || !f2 || (m > 0 && !f3)) return -12;
    cudaStream_t s = (cudaStream_t)stream;
    const DualGemvPlan pw = dual_gemv_plan(n, m), pv = dual_gemv_plan(n, p);
    const size_t need = (size_t)pw.ncb * n + (size_t)pw.nrb * m + (size_t)pv.ncb * n + (size_t)pv.nrb * p +
                        304 * 6 + 8;
    if (need > NOALLOC_SCRATCH_DOUBLES) return MPIR_UNSUP();
    double *base = nullptr;
    if (noalloc_scratch(&base)) return MPIR_CUDA_ERROR;
    double *pWx = base;
    double *pWtz = pWx + (size_t)pw.ncb * n;
    double *pVy = pWtz + (size_t)pw.nrb * m;
    double *pVtz = pVy + (size_t)pv.ncb * n;
    double *normpart = pVtz + (size_t)pv.nrb * p;
    double *nrm = normpart + 304 * 6;
    // every partial the finalize step reads is written by the gemvs of this
    // call, so nothing has to be cleared first; each launch's own status is
    // checked, so an error left pending by the caller's earlier work is not
    // reported as this call's
    if (dual_gemv(W, ldw, n, m, x, z, pWx, pWtz, s) != cudaSuccess ||
        dual_gemv(V, ldv, n, p, y, z, pVy, pVtz, s) != cudaSuccess ||
        gls_resid_finalize(n, m, p, d, x, y, z, pWx, pw.ncb, pWtz, pw.nrb, pVy, pv.ncb, pVtz, pv.nrb, f1, f2, f3,
                           normpart, nrm, s) != cudaSuccess)
        return MPIR_CUDA_ERROR;
    if (norms2 && cudaMemcpyAsync(norms2, nrm, 6 * sizeof(double), cudaMemcpyDeviceToDevice, s) != cudaSuccess)
        return MPIR_CUDA_ERROR;
    return 0;
}
