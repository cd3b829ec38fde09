// batched.cu -- host side of the batched LSE / GLS solver: dispatch over the
// compiled launch shapes and the sizing helpers (device code in
// batched_kernel.cuh, one translation unit per launch shape).
#include <algorithm>

#include "batched_kernel.cuh"

namespace mpir {

int batched_launch_f32_g512(const BInst *, const int *, int, int *, BResult *, void *, size_t, size_t, int,
                          const BParams &, cudaStream_t);
int batched_occupancy_f32_g512(size_t);
int batched_launch_f32_g256(const BInst *, const int *, int, int *, BResult *, void *, size_t, size_t, int,
                          const BParams &, cudaStream_t);
int batched_occupancy_f32_g256(size_t);
int batched_launch_f32_g128(const BInst *, const int *, int, int *, BResult *, void *, size_t, size_t, int,
                          const BParams &, cudaStream_t);
int batched_occupancy_f32_g128(size_t);
int batched_launch_f32_g64(const BInst *, const int *, int, int *, BResult *, void *, size_t, size_t, int,
                          const BParams &, cudaStream_t);
int batched_occupancy_f32_g64(size_t);
int batched_launch_f64_g512(const BInst *, const int *, int, int *, BResult *, void *, size_t, size_t, int,
                          const BParams &, cudaStream_t);
int batched_occupancy_f64_g512(size_t);
int batched_launch_f64_g128(const BInst *, const int *, int, int *, BResult *, void *, size_t, size_t, int,
                          const BParams &, cudaStream_t);
int batched_occupancy_f64_g128(size_t);

int batched_ctas_per_sm(const BConfig &c, bool fp64)
{
    if (fp64) {
        switch (c.group) {
        case 512: return batched_occupancy_f64_g512(c.smem);
        case 128: return batched_occupancy_f64_g128(c.smem);
        default: return 0;
        }
    }
    switch (c.group) {
    case 512: return batched_occupancy_f32_g512(c.smem);
    case 256: return batched_occupancy_f32_g256(c.smem);
    case 128: return batched_occupancy_f32_g128(c.smem);
    case 64: return batched_occupancy_f32_g64(c.smem);
    default: return 0;
    }
}

int batched_launch(const BConfig &c, bool fp64, const BInst *tab, const int *order, int count, int *next,
                   BResult *res, void *gscr, size_t gstride, int grid, const BParams &prm, cudaStream_t s)
{
    if (count <= 0) return 0;
    if (fp64) {
        switch (c.group) {
        case 512: return batched_launch_f64_g512(tab, order, count, next, res, gscr, gstride, c.smem, grid, prm, s);
        case 128: return batched_launch_f64_g128(tab, order, count, next, res, gscr, gstride, c.smem, grid, prm, s);
        default: return MPIR_UNSUP();
        }
    }
    switch (c.group) {
    case 512: return batched_launch_f32_g512(tab, order, count, next, res, gscr, gstride, c.smem, grid, prm, s);
    case 256: return batched_launch_f32_g256(tab, order, count, next, res, gscr, gstride, c.smem, grid, prm, s);
    case 128: return batched_launch_f32_g128(tab, order, count, next, res, gscr, gstride, c.smem, grid, prm, s);
    case 64: return batched_launch_f32_g64(tab, order, count, next, res, gscr, gstride, c.smem, grid, prm, s);
    default: return MPIR_UNSUP();
    }
}

static BPlan plan_of(int kind, int m, int n, int p)
{
    return kind == BKIND_GLS ? gplan(m, n, p) : bplan(m, n, p);
}

size_t batched_big_words(int kind, int m, int n, int p)
{
    return plan_of(kind, m, n, p).fac_big;
}

size_t batched_smem_min(int kind, int m, int n, int p, bool fp64)
{
    const BPlan P = plan_of(kind, m, n, p);
    return fp64 ? bsmem_need<double>(P, 0) : bsmem_need<float>(P, 0);
}

size_t batched_smem_full(int kind, int m, int n, int p, bool fp64)
{
    const BPlan P = plan_of(kind, m, n, p);
    return fp64 ? bsmem_need<double>(P, 2) : bsmem_need<float>(P, 2);
}

double batched_work(int kind, int m, int n, int p)
{
    if (kind == BKIND_GLS) {
        // GQR flops (QR of n x m with Q^T applied to the p columns of V, QR
        // of the p x n C~) plus one residual
        const double kC = std::min(n, p);
        double f = 2.0 * n * m * m - 2.0 * (double)m * m * m / 3.0;
        f += 4.0 * (double)n * m * p - 2.0 * (double)m * m * p;
        f += 2.0 * (double)p * n * kC - 2.0 * kC * kC * kC / 3.0;
        return f + 8.0 * ((double)n * m + (double)n * p);
    }
    // GRQ flops (QR of n x p, apply to m x n from the right, QR of m x n)
    const double kA = std::min(m, n);
    double f = 2.0 * n * p * p - 2.0 * p * p * p / 3.0;
    f += 4.0 * (double)m * n * p;
    f += 2.0 * m * n * kA - 2.0 * kA * kA * kA / 3.0;
    return f + 8.0 * ((double)m * n + (double)p * n);
}

} // namespace mpir
