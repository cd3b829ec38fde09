// batched_f32_g128.cu -- one launch shape of the batched LSE kernel
// (float factors, groups of 128 threads), compiled on its own.
#include "batched_kernel.cuh"

namespace mpir {

int batched_launch_f32_g128(const BInst *tab, const int *order, int count, int *next, BResult *res, void *gscr,
                          size_t gstride, size_t smem, int grid, const BParams &prm, cudaStream_t s)
{
    return launch_cfg<128, float>(tab, order, count, next, res, (float *)gscr, gstride, smem, grid, prm, s);
}

int batched_occupancy_f32_g128(size_t smem) { return occupancy_of<128, float>(smem); }

} // namespace mpir
