// selector.h -- launchers of the selector kernels (features, MLP).
#pragma once

#include <cuda_runtime.h>
#include <cstddef>

namespace mpir {

constexpr int MLP_PARAMS = 5638;   // 64*16 + 64 + 64*64 + 64 + 6*64 + 6
constexpr int NCLASS = 6;          // {BF16, FP32, FP64} x {classical, GMRES}
constexpr int NFEAT = 16;

size_t features_ws_doubles(int R, int C);
// kind 0: LSE (A m x n, B p x n, s length n); kind 1: GLS (W n x m as A,
// V n x p as B, s length m + p).  bv/dv: right-hand sides whose norms are
// features (LSE b, d; GLS d and none).  out: 16 floats (device).
int features_launch(int kind, int m, int n, int p, const double *A, int lda, const double *B, int ldb,
                    const double *s, const double *bv, int nbv, const double *dv, int ndv, int k, double *ws,
                    float *out, cudaStream_t st);

size_t mlp_ws_floats(int count);
int mlp_forward(const float *P, const float *X, int count, float *prob, cudaStream_t s);
int mlp_train_step(float *P, float *M, float *V, int t, float lr, const float *X, const int *y, int count,
                   float *ws, float *grad_out, float *loss_out, cudaStream_t s);

} // namespace mpir
