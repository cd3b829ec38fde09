// kernels.h -- host-side launchers of the libmpir device kernels.
#pragma once

#include <cuda_runtime.h>
#include <cstddef>

namespace mpir {

// Kernel kinds for the launch counter and the optional per-kind timers.
enum KernelKind {
    K_PANEL = 0, K_LARFB, K_VEC_APPLY, K_TRSV, K_GEMV, K_DUAL_GEMV, K_FINALIZE, K_CONVERT, K_NORM,
    K_ELEMWISE, K_LARFB_TC, K_LARFB_AUX, K_GMRES, K_BATCHED, K_SELECTOR, K_NKINDS
};
// Called around every kernel launch: counts the launch and, when timing is
// enabled (mpir_profile), records a CUDA event pair on the launch stream.
void prof_begin(int kind, cudaStream_t s);
void prof_end(int kind, cudaStream_t s);
void prof_count(int kind);   // count only (launches inside a stream capture)
struct ProfScope {
    int k; cudaStream_t s;
    ProfScope(int kind, cudaStream_t st) : k(kind), s(st) { prof_begin(k, s); }
    ~ProfScope() { prof_end(k, s); }
};

// Larfb (trailing update / block-reflector application) operand precision.
enum class GemmPrec { FP32 = 0, TF32 = 1, BF16 = 2, FP64 = 3 };

template <typename T> constexpr int panel_nb() { return sizeof(T) == 4 ? 32 : 16; }
constexpr int OUTER_NB = 128;            // reflectors per outer (tensor-core) block
__host__ __device__ inline int rup32(int x) { return (x + 31) & ~31; }

struct DevScratch {          // small device scratch owned by the handle
    unsigned int *barrier;   // 2 words, zero between launches
    int *err;                // device error flags
    int *status;             // solver status word (singular diagonals)
    void *part;              // reduction partials
    size_t part_bytes;
};

// ---- factorization (qr.cu) ------------------------------------------
// Blocked Householder QR of the M x N column-major matrix A (lda):
// A = Z T with Z = H_0 ... H_{k-1}, k = min(M, N).  Reflector vectors below
// the diagonal, tau[k], and the compact-WY factor of every panel of
// panel_nb<T>() reflectors in Tw (NB x NB column-major per panel, upper
// triangular; H_j0 ... H_j0+nb-1 = I - V Tw V^T).  For FP32 storage the
// factorization is two-level: 128-reflector outer blocks whose compact-WY
// factors go to Tw128 (128 x 128 per block) and whose trailing updates run
// on the tensor cores (gemm_tc.cu) at `prec`.  lda must be a multiple of 4
// (16-byte rows for TMA).  ws: geqrf_ws_bytes() of scratch.
// tf (optional, FP32 storage only): also form the aggregated compact-WY
// factor of all k reflectors, tf->Tf (k x k upper triangular, column-major,
// ld tf->ldt >= k, a multiple of 4, 16-byte aligned):
// H_0 ... H_{k-1} = I - V Tf V^T.  With tf->side set, that work runs on the
// side stream (forked from s by tf->fork after each outer block, scratch
// tf->ws2 of geqrf_ws_bytes(M, N)): the caller makes s wait for the side
// stream before it reads Tf or reuses the scratch.
// Returns 0, or MPIR_UNSUPPORTED / MPIR_CUDA_ERROR.
//
// Look-ahead (FP32 storage, tf->crit set and ws of geqrf_la_ws_bytes): the
// panels, the inner updates and the update of the next outer block's
// columns run on tf->crit (a high-priority stream forked from s); the rest
// of each trailing update runs on s, overlapped with the next block's
// panels (events tf->la_a / tf->la_b order the two).  geqrf returns with s
// joined to tf->crit.
struct TfullJob {
    float *Tf;
    int ldt;
    cudaStream_t side;
    cudaEvent_t fork, join;
    void *ws2;
    cudaStream_t crit;
    cudaEvent_t la_a, la_b;
    cudaStream_t aux;            // outer-block factor, beside the next columns' V^T C
    cudaEvent_t ax_a, ax_b;
};
size_t geqrf_la_ws_bytes(int M, int N);
size_t geqrf_ws_bytes(int M, int N);
// kmax >= 0 stops after min(M, N, kmax) reflectors; the remaining columns
// are still updated (so [W | V] with kmax = m leaves R over Q^T V).
template <typename T>
int geqrf(T *A, int lda, int M, int N, T *tau, T *Tw, T *Tw128, GemmPrec prec, void *ws, int *err,
          cudaStream_t s, const TfullJob *tf = nullptr, int kmax = -1);

// C (M x Nc, ldc) <- Z^T C (trans = 1) or Z C (trans = 0) for the reflector
// set left in (V, ldv, K reflectors, Tw, Tw128) by geqrf on an M-row matrix.
template <typename T>
int apply_reflectors_left(const T *V, int ldv, int M, int K, const T *Tw, const T *Tw128, int trans,
                          T *C, int ldc, int Nc, GemmPrec prec, void *ws, int *err, cudaStream_t s);

// C (M x N, ldc) <- (I - V X V^T) C, X = Tb^T (trans) or Tb (K x K upper
// triangular, ld 128), V = unit lower trapezoid of the M x K panel V (ldv),
// K <= 128, on the tensor cores.  ws: geqrf_ws_bytes(M, N).
int larfb_tc(const float *V, int ldv, int M, int K, const float *Tb, int trans, float *C, int ldc, int N,
             GemmPrec prec, void *ws, int *err, cudaStream_t s);

// ---- vectors (vec.cu) -------------------------------------------------
// x (length M) <- Z^T x (trans = 1) or Z x (trans = 0), cooperative launch.
template <typename T>
int apply_reflectors_vec(const T *V, int ldv, int M, int K, const T *Tw, int trans, T *x,
                         const DevScratch &sc, cudaStream_t s);

// Same as apply_reflectors_vec with blocks of nbv reflectors whose
// compact-WY factors are in Tw (nbv x nbv each, ld nbv): one thread-block
// cluster, one cluster barrier per block (nbv in {16, 32, 128}).
template <typename TS, typename T>
int apply_reflectors_vec_blk(const TS *V, int ldv, int M, int K, const TS *Tw, int nbv, int trans, T *x,
                             cudaStream_t s);
// x (length M) <- (I - V op(Tf) V^T) x with the aggregated factor Tf of all
// K reflectors (geqrf's Tf, ld ldt): op = Tf^T (trans = 1, Z^T x) or Tf
// (Z x).  Four or five full-GPU launches, no dependent per-block steps.
// ws: wy_apply_ws_bytes(M, K) bytes (device, 256-byte aligned).
size_t wy_apply_ws_bytes(int M, int K);
// Reflectors per segment of the aggregated compact-WY factor: the
// factorization forms one aggregated factor per segment, the vector
// application runs the segments in turn.
constexpr int WY_SEG = 2048;
template <typename TS, typename T>
int wy_apply_vec(const TS *V, int ldv, int M, int K, const TS *Tf, int ldt, int trans, T *x, void *ws,
                 cudaStream_t s);
// Triangular solves of FP32-stored factors of order n <= 8192 in 64-row
// blocks (trsv64.cu): trsv64_ok(n, sizeof(storage)) says whether they apply;
// invert_diag64 forms the inverses of the 64 x 64 diagonal blocks (4096
// entries per block, column-major; zero pivot -> bit 1 of *status) that
// trsv64 reads.  trsv64 returns -1 when it cannot run (the caller then uses
// the 32-row solve by substitution).  dinv_elems(N): entries of an inverse
// array for either block size.  t64_pack copies the off-diagonal block
// columns of an order-N triangle into the order the solves read them
// (t64_pack_elems(N) floats, 16-byte aligned; once per factorization); a
// solve of any leading n x n block (n <= npack) may pass that pack, or
// nullptr to read U in place.
bool trsv64_ok(int n, size_t ts_bytes);
size_t dinv_elems(int N);
size_t t64_pack_elems(int N);
int t64_pack(const float *U, int ldu, int N, float *pack, cudaStream_t s);
template <typename TS, typename T>
void invert_diag64(const TS *U, int ldu, int N, T *Dinv, int *status, cudaStream_t s);
template <typename T>
int trsv64(const float *U, int ldu, int n, int trans, T *x, const T *Dinv, const float *pack, int npack, int *err,
           cudaStream_t s);
// Mixed precision (factors stored as TS, arithmetic and vectors in T).
template <typename TS, typename T>
int trsv_upper_mixed(const TS *U, int ldu, int n, int trans, T *x, const DevScratch &sc, cudaStream_t s,
                     const T *Dinv = nullptr);
template <typename TS, typename T>
void invert_diag32_mixed(const TS *U, int ldu, int N, T *Dinv, int *status, cudaStream_t s);
template <typename TS, typename T>
int gemv_mixed(const TS *M, int ld, int rows, int cols, int trans, T alpha, const T *x, T beta, T *y,
               int upper_mask, int diag_off, cudaStream_t s);

// Solve U x = b (trans = 0) or U^T x = b (trans = 1) in place, U upper
// triangular n x n (ldu).  Zero diagonal -> bit 1 of *sc.status.
// Dinv (optional): inverses of the 32 x 32 diagonal blocks of U from
// invert_diag32 (the solve then forms each block by a 32-wide product).
template <typename T>
int trsv_upper(const T *U, int ldu, int n, int trans, T *x, const DevScratch &sc, cudaStream_t s,
               const T *Dinv = nullptr);
template <typename T>
void invert_diag32(const T *U, int ldu, int N, T *Dinv, int *status, cudaStream_t s);

// y <- beta y + alpha op(M) x, M rows x cols (ld); op = M (trans = 0) or M^T.
// If upper_mask, entries M(i, j) with i > j + diag_off are treated as zero.
template <typename T>
int gemv(const T *M, int ld, int rows, int cols, int trans, T alpha, const T *x, T beta, T *y,
         int upper_mask, int diag_off, cudaStream_t s);

// Elementwise helpers.
// dst[i] = (T)(scale * g * src[rev ? n-1-i : i]), g = *dscale (device
// scalar) when dscale != NULL, else 1.
template <typename Ts, typename Td>
void vcopy(const Ts *src, Td *dst, int n, double scale, int rev, cudaStream_t s,
           const double *dscale = nullptr);
// Power-of-two normalization of right-hand sides before down-conversion:
// g = 2^-e with max(|a1 * u|, |a2 * w|) * g in [0.5, 1) (1 if the max is 0 or
// not finite); out[0] = g, out[1] = 1 / g.  Device only (no host sync).
void pow2_normalizer(const double *u, int nu, double a1, const double *w, int nw, double a2, double *out,
                     cudaStream_t s);
// dst[i] += scale * g * src[rev ? n-1-i : i]   (FP64 destination; g = *dscale
// when dscale != NULL, else 1)
template <typename Ts>
void vaxpy(const Ts *src, double *dst, int n, double scale, int rev, cudaStream_t s,
           const double *dscale = nullptr);
void vzero(void *dst, size_t bytes, cudaStream_t s);

// Real 2 x 2 block embedding of complex arrays (complex.cu): interleaved
// (re, im) input, leading dimensions in complex elements.
int zembed_mat(const double *Z, int rows, int cols, int ldz, double *out, int ldo, cudaStream_t s);
int zembed_vec(const double *z, int n, double *out, cudaStream_t s);
int zunembed_vec(const double *in, int n, double *z, cudaStream_t s);
// One embedding job of a batch: src complex (interleaved; lds in complex
// elements), dst real (ldd); vec: e(z) = [Re z; Im z] of a rows-vector (cols
// = 1) instead of the 2 x 2 block matrix.  For the read-back (unembed = 1)
// dst is the embedded vector (2 rows) and src the complex output.
struct ZEmbedJob {
    const double *src;
    double *dst;
    int rows, cols, lds, ldd, vec;
};
int zembed_batch(const ZEmbedJob *jobs_dev, int njobs, int unembed, cudaStream_t s);

// Matrix conversion with optional transpose and index reversal:
//   dst(i, j) = (Td)(scale * src(ri, ci)),  i < rows_d, j < cols_d,
// transpose = 0: (ri, ci) = (i', j');  transpose = 1: (ri, ci) = (j', i'),
// where i' = rev_r ? rows_d-1-i : i and j' = rev_c ? cols_d-1-j : j.
// With rs != NULL every destination row is further multiplied by
// rs[rs_rev ? rows_d-1-i : i] (a per-row power-of-two scale).
template <typename Ts, typename Td>
void mconvert(const Ts *src, int lds, Td *dst, int ldd, int rows_d, int cols_d, int transpose,
              int rev_r, int rev_c, double scale, cudaStream_t s, const double *rs = nullptr,
              int rs_rev = 0);

// v[i] *= D[rev ? n-1-i : i]  (D: device FP64 vector of powers of two).
template <typename T>
void vdiag(T *v, const double *D, int n, int rev, cudaStream_t s);

// Per-column power-of-two scaling of the stacked [a1 A; a2 B] (A rows_a x n,
// B rows_b x n, column-major): D[j] = 2^-e with
// max(a1 max_i |A(i,j)|, a2 max_i |B(i,j)|) * D[j] in [0.5, 1) (1 for a zero
// column).  One warp per column.
void colscale_pow2(const double *A, int lda, int rows_a, const double *B, int ldb, int rows_b, int n, double a1,
                   double a2, double *D, cudaStream_t s);

// max |A(i,j)| and sum A(i,j)^2 (FP64) into out[0], out[1] (device).
void absmax_sumsq(const double *A, int lda, int rows, int cols, double *part, double *out,
                  cudaStream_t s);

// ---- residuals (resid.cu) ------------------------------------------------
// For an FP64 matrix A (rows x cols, lda): partial sums of A x (per column
// block) and A^T r (per row block) -- one read of A.
struct DualGemvPlan {
    int rows, cols, nrb, ncb;   // row / column blocks of 256
};
DualGemvPlan dual_gemv_plan(int rows, int cols);
cudaError_t dual_gemv(const double *A, int lda, int rows, int cols, const double *x, const double *r,
                      double *part_Ax, double *part_Atr, cudaStream_t s);

// LSE residual from partials: f1 = b - r - sum(Ax), f2 = d - sum(Bx),
// f3 = -sum(A^T r) + sum(B^T v); norms2[0..5] = squares of ||f1||, ||f2||,
// ||f3||, ||x||, ||r||, ||v|| (device).
cudaError_t lse_resid_finalize(int m, int n, int p, const double *b, const double *d,
                        const double *x, const double *r, const double *v,
                        const double *pAx, int ncbA, const double *pAtr, int nrbA,
                        const double *pBx, int ncbB, const double *pBtv, int nrbB,
                        double *f1, double *f2, double *f3, double *normpart, double *norms2,
                        cudaStream_t s);
// GLS: f1 = -y + sum(V^T z), f2 = d - sum(Wx) - sum(Vy), f3 = sum(W^T z);
// norms2 = squares of ||f1||, ||f2||, ||f3||, ||x||, ||y||, ||z||.
cudaError_t gls_resid_finalize(int n, int m, int p, const double *d, const double *x,
                        const double *y, const double *z,
                        const double *pWx, int ncbW, const double *pWtz, int nrbW,
                        const double *pVy, int ncbV, const double *pVtz, int nrbV,
                        double *f1, double *f2, double *f3, double *normpart, double *norms2,
                        cudaStream_t s);

// Double-double variants (u_r = u^2): the same residual blocks and norms
// as the finalize routines above, every product sum carried as an
// unevaluated pair.  scr: 2 (m + p + 2 n) doubles (LSE), 2 (2 n + m + p) (GLS).
cudaError_t lse_resid_dd(int m, int n, int p, const double *A, int lda, const double *B, int ldb, const double *b,
                         const double *d, const double *x, const double *r, const double *v, double *scr,
                         double *f1, double *f2, double *f3, double *norms2, cudaStream_t s);
cudaError_t gls_resid_dd(int n, int m, int p, const double *W, int ldw, const double *V, int ldv, const double *d,
                         const double *x, const double *y, const double *z, double *scr, double *f1, double *f2,
                         double *f3, double *norms2, cudaStream_t s);
// out[0] = (accumulate ? out[0] : 0) + ||a - b||^2
cudaError_t diff_norm2(const double *a, const double *b, int n, double *out, int accumulate, cudaStream_t s);

} // namespace mpir
