// batched.h -- persistent batched LSE / GLS solver (many small problems, one launch).
#pragma once

#include <cuda_runtime.h>
#include <cstddef>
#include <vector>

namespace mpir {

// One problem of the batch (device table entry; pointers are device memory).
// kind 0: LSE (A m x n, B p x n, b, d -> x).  kind 1: GLS in the xGGGLM
// convention with W = A (n x m, lda), V = B (n x p, ldb), d -> x (m), y (p);
// the fields keep the GLS names m (columns of W), n (rows), p (columns of V).
struct BInst {
    const double *A, *B, *b, *d;
    double *x, *y;
    int m, n, p, lda, ldb, kind;
};
enum { BKIND_LSE = 0, BKIND_GLS = 1 };

// Per-problem result written by the kernel.
struct BResult {
    int status, iters;
    double ratio[3];
};

struct BParams {
    double tol;
    int maxit;
    int refine;        // MPIR_CLASSICAL or MPIR_DIRECT
    int scale;         // power-of-two scaling of A, B (Sec. 6.1)
};

// Launch shape: 512 threads per CTA split into groups of `group` threads
// (512, 256, 128 or 64), each solving its own problem; `smem` dynamic shared
// memory per CTA, split evenly between the groups.
struct BConfig {
    int group;
    size_t smem;
};

// Device-side state a handle keeps for batched solves.
struct BatchArena {
    BInst *tab = nullptr;
    int *order = nullptr;
    BResult *res = nullptr;
    int *next = nullptr;
    void *gscr = nullptr;
    size_t cap = 0, gscr_bytes = 0;
    BInst *htab = nullptr;          // pinned staging
    BResult *hres = nullptr;
    int *horder = nullptr;
    size_t hcap = 0;
    // launch cache: autotuned configuration and captured graph
    struct Tuned { unsigned long long sig; bool fp64; BConfig cfg; };
    std::vector<Tuned> tuned;
    cudaGraphExec_t graph = nullptr;
    unsigned long long graph_key = 0;
    int force_group = 0;            // 0: autotune; else the group size every bucket uses
    BConfig last[2] = {};           // shapes of the last call (per size bucket)
    int last_count[2] = {0, 0};
};

int batched_ctas_per_sm(const BConfig &cfg, bool fp64);
int batched_launch(const BConfig &cfg, bool fp64, const BInst *tab, const int *order, int count, int *next,
                   BResult *res, void *gscr, size_t gstride_words, int grid, const BParams &prm, cudaStream_t s);
// Sizes of one problem (kind: BKIND_LSE with (m, n, p) of lse_solve, or
// BKIND_GLS with (m, n, p) = columns of W, rows, columns of V).
size_t batched_big_words(int kind, int m, int n, int p);           // factor words kept in smem or global scratch
size_t batched_smem_min(int kind, int m, int n, int p, bool fp64);  // smem with the factors in global scratch
size_t batched_smem_full(int kind, int m, int n, int p, bool fp64); // smem with everything resident
double batched_work(int kind, int m, int n, int p);                // factorization + residual flops

} // namespace mpir
