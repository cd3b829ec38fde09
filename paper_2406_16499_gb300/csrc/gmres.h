// gmres.h -- restarted FP64 GMRES engine used by GMRES-IR (Sec. 5).
#pragma once

#include <cuda_runtime.h>
#include <cstddef>

namespace mpir {

constexpr int GMRES_MAX_RESTART = 64;

// A linear operator on device FP64 vectors of length N, enqueued on the
// solver's stream.  Returns 0 or an MPIR_* code.
struct LinOp {
    virtual int apply(const double *in, double *out) = 0;
    virtual ~LinOp() = default;
};

// Device workspace of one GMRES(R) solve of order N.
struct GmresWs {
    int N, R;
    size_t ldv;        // leading dimension of the basis (N rounded up to 32)
    double *Vb;        // basis, R + 1 columns
    double *H;         // (R + 1) x R Hessenberg, rotated in place
    double *cs, *sn;   // Givens rotations
    double *g;         // rotated right-hand side of the least-squares problem
    double *est;       // [0]: |g(j+1)|; [2..3]: norm scratch
    double *part;      // norm partials
    double *r, *tmp;   // cycle residual, operator output
};
size_t gmres_ws_bytes(int N, int R);
GmresWs gmres_layout(void *base, int N, int R);

// Restarted GMRES(R) from x0 = 0 on op t = rhs: stops when the residual
// estimate or the true residual at the end of a cycle drops to tol ||rhs||,
// or after maxit inner iterations.  hbuf: pinned host buffer (>= 2 doubles)
// for the scalars the host reads.  iters: inner iterations taken; rel: the
// true relative residual at the last cycle end.
int gmres_solve(LinOp &op, const double *rhs, double *x, GmresWs &w, double tol, int maxit, double *hbuf,
                cudaStream_t s, int *iters, double *rel);

// out[i] = c0 base[i] + c1 sum_k P1[k st1 + i] + c2 sum_k P2[k st2 + i]
// (partials of dual_gemv; base, P1, P2 may be NULL).
void combine_parts(double *out, int n, double c0, const double *base, double c1, const double *P1, int k1,
                   int st1, double c2, const double *P2, int k2, int st2, cudaStream_t s);

} // namespace mpir
