// complex.cu -- the real 2 x 2 block embedding of complex LSE / GLS problems.
//
// The paper states both problems over C (Sec. 1).  A complex matrix
// Z = X + iY (rows x cols) acts on z = u + iw as the real matrix
//     E(Z) = [X, -Y; Y, X]   (2 rows x 2 cols)   on   e(z) = [u; w],
// an isometry of C^k onto R^2k that maps products to products, Z^H to E(Z)^T
// and keeps every singular value (each twice).  So min ||b - A x|| subject
// to B x = d over C is the real LSE of (E(A), E(B), e(b), e(d)) with
// solution e(x), residual e(r) and multiplier e(v); a GLS likewise.  The
// complex solves of the library run the real factorizations, refinement
// and kernels on that embedding.  These kernels form it and read the
// solution back.  Complex arrays are interleaved (re, im) doubles,
// column-major with leading dimensions counted in complex elements.
#include "common.cuh"
#include "kernels.h"
#include "mpir.h"

namespace mpir {

// out (2 rows x 2 cols, leading dimension ldo) = E(Z)
__global__ void __launch_bounds__(256)
k_zembed_mat(const double2 *__restrict__ Z, int rows, int cols, int ldz, double *__restrict__ out, int ldo)
{
    const size_t total = (size_t)rows * cols;
    for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < total; e += (size_t)gridDim.x * blockDim.x) {
        const int i = (int)(e % rows), j = (int)(e / rows);
        const double2 z = Z[i + (size_t)j * ldz];
        out[i + (size_t)j * ldo] = z.x;
        out[i + rows + (size_t)j * ldo] = z.y;
        out[i + (size_t)(j + cols) * ldo] = -z.y;
        out[i + rows + (size_t)(j + cols) * ldo] = z.x;
    }
}

// out (2n) = e(z)
__global__ void __launch_bounds__(256)
k_zembed_vec(const double2 *__restrict__ z, int n, double *__restrict__ out)
{
    for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < n; k += gridDim.x * blockDim.x) {
        const double2 v = z[k];
        out[k] = v.x;
        out[n + k] = v.y;
    }
}

// z = e^-1(in): z_k = in[k] + i in[n + k]
__global__ void __launch_bounds__(256)
k_zunembed_vec(const double *__restrict__ in, int n, double2 *__restrict__ z)
{
    for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < n; k += gridDim.x * blockDim.x)
        z[k] = make_double2(in[k], in[n + k]);
}

static int grid_for(size_t n) { return (int)std::min<size_t>(std::max<size_t>((n + 255) / 256, 1), 4096); }

int zembed_mat(const double *Z, int rows, int cols, int ldz, double *out, int ldo, cudaStream_t s)
{
    if (rows <= 0 || cols <= 0) return 0;
    ProfScope ps(K_CONVERT, s);
    k_zembed_mat<<<grid_for((size_t)rows * cols), 256, 0, s>>>(reinterpret_cast<const double2 *>(Z), rows, cols,
                                                               ldz, out, ldo);
    return cudaGetLastError() == cudaSuccess ? 0 : MPIR_CUDA_ERROR;
}

int zembed_vec(const double *z, int n, double *out, cudaStream_t s)
{
    if (n <= 0) return 0;
    ProfScope ps(K_CONVERT, s);
    k_zembed_vec<<<grid_for(n), 256, 0, s>>>(reinterpret_cast<const double2 *>(z), n, out);
    return cudaGetLastError() == cudaSuccess ? 0 : MPIR_CUDA_ERROR;
}

int zunembed_vec(const double *in, int n, double *z, cudaStream_t s)
{
    if (n <= 0) return 0;
    ProfScope ps(K_CONVERT, s);
    k_zunembed_vec<<<grid_for(n), 256, 0, s>>>(in, n, reinterpret_cast<double2 *>(z));
    return cudaGetLastError() == cudaSuccess ? 0 : MPIR_CUDA_ERROR;
}

} // namespace mpir

namespace mpir {

// Batched embedding: one CTA per job (a matrix: E(Z) into a 2 rows x 2 cols
// block; a vector (vec != 0): e(z) = [Re z; Im z]); jobs of uneven size.
__global__ void __launch_bounds__(256)
k_zembed_batch(const ZEmbedJob *__restrict__ jobs, int njobs)
{
    const int jb = blockIdx.x;
    if (jb >= njobs) return;
    const ZEmbedJob J = jobs[jb];
    const double2 *Z = reinterpret_cast<const double2 *>(J.src);
    const size_t total = (size_t)J.rows * J.cols;
    for (size_t e = threadIdx.x; e < total; e += blockDim.x) {
        const int i = (int)(e % J.rows), j = (int)(e / J.rows);
        const double2 z = Z[i + (size_t)j * J.lds];
        J.dst[i + (size_t)j * J.ldd] = z.x;
        J.dst[i + J.rows + (size_t)j * J.ldd] = z.y;
        if (!J.vec) {
            J.dst[i + (size_t)(j + J.cols) * J.ldd] = -z.y;
            J.dst[i + J.rows + (size_t)(j + J.cols) * J.ldd] = z.x;
        }
    }
}

// Batched read-back: z = e^-1(src), src = [Re; Im] of length 2 rows.
__global__ void __launch_bounds__(256)
k_zunembed_batch(const ZEmbedJob *__restrict__ jobs, int njobs)
{
    const int jb = blockIdx.x;
    if (jb >= njobs) return;
    const ZEmbedJob J = jobs[jb];
    double2 *z = reinterpret_cast<double2 *>(const_cast<double *>(J.src));
    for (int k = threadIdx.x; k < J.rows; k += blockDim.x) z[k] = make_double2(J.dst[k], J.dst[J.rows + k]);
}

int zembed_batch(const ZEmbedJob *jobs_dev, int njobs, int unembed, cudaStream_t s)
{
    if (njobs <= 0) return 0;
    ProfScope ps(K_CONVERT, s);
    if (unembed) k_zunembed_batch<<<njobs, 256, 0, s>>>(jobs_dev, njobs);
    else k_zembed_batch<<<njobs, 256, 0, s>>>(jobs_dev, njobs);
    return cudaGetLastError() == cudaSuccess ? 0 : MPIR_CUDA_ERROR;
}

} // namespace mpir
