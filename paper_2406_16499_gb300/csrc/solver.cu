// solver.cu -- the C ABI of libmpir.so (include/mpir.h): handle, workspace,
// the generalized factorizations, the initial solutions, the correction
// solves and the refinement loops of the paper (Alg. 1-4).
//
// Representation of the generalized factorizations
// -------------------------------------------------
// Every factorization is a column-major Householder QR (qr.cu).  An RQ
// factorization C = T Z (rows annihilated from the right) is obtained as the
// QR factorization of the reversed transpose  C~ = P C^T P = Z~ T~  with
//     Z = P Z~^T P,   T = P T~^T P,
// P the reversal permutation of matching size.  Hence
//   LSE (GRQ, Lemma 4.5):  B~ = P_n B^T P_p = Q~ [R~; 0]  (Q = P_n Q~^T P_n,
//        R = P_p R~^T P_p);  X = Q~^T (P_n A^T) = P_n (A Q^T)^T;
//        A Q^T = Z T by QR of X^T P_n.
//   GLS (GQR, Lemma 4.6):  W = Q [R; 0] by QR;  C = Q^T V;
//        C~ = P_p C^T P_n = Z~ T~  (Z = P_p Z~^T P_p, T = P_n T~^T P_p).
// The algorithms below are Alg. 1 / Alg. 3 rewritten in these reversed
// coordinates; every step names the paper's step it implements.
//
// Scaling (Sec. 6.1, "appropriate scaling" before down-conversion): A, B
// (resp. W, V) are multiplied by powers of two sA, sB (sW, sV) so that their
// largest entry lies in [0.5, 1); the corresponding exact rescalings of the
// right-hand sides and solutions are applied around every solve.  The
// right-hand side of each correction solve is further normalized by a power
// of two (gamma) so that it uses the whole low-precision exponent range.
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <cmath>
#include <atomic>
#include <string>
#include <vector>
#include <algorithm>

#include "batched.h"
#include "common.cuh"
#include "gmres.h"
#include "kernels.h"
#include "mpir.h"
#include "selector.h"

using namespace mpir;

// ----------------------------------------------------- launch profiling --
// Process-wide: a launch counter per kernel kind (atomic: launches may come
// from several host threads), and (when enabled, single-threaded use) a pool
// of CUDA event pairs recorded around every launch on its own stream.
namespace mpir {
static std::atomic<long long> g_launches[K_NKINDS];
static bool g_prof = false;
static std::vector<cudaEvent_t> g_ev;
static std::vector<int> g_kind;
static size_t g_nrec = 0;
static bool g_open = false;
constexpr size_t PROF_CAP = 1 << 14;

void prof_begin(int kind, cudaStream_t s)
{
    g_launches[kind].fetch_add(1, std::memory_order_relaxed);
    // the event pool is created by mpir_profile(1); launches beyond it are
    // counted but not timed (no resource is created on the launch path)
    if (!g_prof || 2 * (g_nrec + 1) > g_ev.size()) return;
    cudaEventRecord(g_ev[2 * g_nrec], s);
    g_open = true;
}

void prof_count(int kind) { g_launches[kind].fetch_add(1, std::memory_order_relaxed); }

// Launch counts of the library's own kernels replayed from a captured graph:
// the capture counted them once; every replay adds them again.
static void prof_add(const long long *per_kind, long long times)
{
    for (int k = 0; k < K_NKINDS; k++)
        if (per_kind[k]) g_launches[k].fetch_add(per_kind[k] * times, std::memory_order_relaxed);
}
static void prof_snapshot(long long *out)
{
    for (int k = 0; k < K_NKINDS; k++) out[k] = g_launches[k].load(std::memory_order_relaxed);
}

void prof_end(int kind, cudaStream_t s)
{
    if (!g_prof || !g_open) return;
    cudaEventRecord(g_ev[2 * g_nrec + 1], s);
    g_kind[g_nrec] = kind;
    g_nrec++;
    g_open = false;
}
} // namespace mpir

static const char *g_kind_names[K_NKINDS] = {"panel_qr", "larfb", "vec_apply", "trsv", "gemv",
                                             "dual_gemv_fp64", "resid_finalize", "convert", "norm",
                                             "elementwise", "larfb_tc", "larfb_aux", "gmres",
                                             "batched", "selector"};

#define MPIR_VERSION_STRING "libmpir 0.1 (sm_103a)"

// ------------------------------------------------------------------ ctx --

namespace {
// Makes `dev` the current device for the scope and gives the caller's
// current device back at its end (creation and destruction only: every other
// call on a handle is made with the handle's device current).
struct DeviceScope {
    int prev = -1;
    bool ok = true;
    explicit DeviceScope(int dev)
    {
        if (cudaGetDevice(&prev) != cudaSuccess) { cudaGetLastError(); prev = -1; }
        if (dev >= 0 && dev != prev && cudaSetDevice(dev) != cudaSuccess) { cudaGetLastError(); ok = false; }
    }
    ~DeviceScope()
    {
        int cur = -1;
        if (prev >= 0 && cudaGetDevice(&cur) == cudaSuccess && cur != prev) cudaSetDevice(prev);
    }
    DeviceScope(const DeviceScope &) = delete;
    DeviceScope &operator=(const DeviceScope &) = delete;
};
} // namespace

namespace {

enum class Kind { NONE, LSE, GLS };

struct Carver {
    uintptr_t base, off = 0;
    explicit Carver(void *b) : base((uintptr_t)b) {}
    template <typename U> U *take(size_t count)
    {
        off = (off + 255) & ~(uintptr_t)255;
        U *p = reinterpret_cast<U *>(base + off);
        off += count * sizeof(U) + 0;
        return p;
    }
    size_t used() const { return (size_t)((off + 255) & ~(uintptr_t)255); }
};

// Device-side state of the classical refinement loop (doubles): the loop's
// control kernel reads the squared residual norms, applies the stop test and
// the stagnation rule, and leaves the power-of-two scales of the next
// correction for the correction's kernels.
enum {
    IRD_BEST = 0, IRD_SINCE = 1, IRD_IT = 2, IRD_STATUS = 3, IRD_RATIO = 4,   // ratio: 3 words
    IRD_C = 8,        // c1, c2, c3: scales of the correction's right-hand side blocks
    IRD_I = 11,       // i1, i2, i3: scales of the correction's outputs
    IRD_S1 = 14, IRD_S2 = 15, IRD_F1 = 16, IRD_F2 = 17,   // sA, sB (sW, sV); ||A||_F, ||B||_F
    IRD_N1 = 18,      // absmax, sum of squares of b (LSE) / d (GLS)
    IRD_N2 = 20,      // absmax, sum of squares of d (LSE)
    IRD_WORDS = 24
};

template <typename T> struct LseWs {
    int m, n, p, q, kA;
    int ldBt, ldX, ldAt;                 // padded to 32 (TMA rows of 128 bytes)
    T *Bt, *tauB, *TwB, *X, *At, *tauA, *TwA, *Tw128B, *Tw128A, *DinvB, *DinvA;
    T *TfB, *TfA;                        // aggregated compact-WY factors (FP32 storage only)
    int ldtB, ldtA;
    float *PkB, *PkA;                    // packed block columns of R~ (p) and T (kA) for trsv64
    void *gws;                           // scratch of the two-level factorization
    void *wy;                            // scratch of the aggregated vector applications
    void *gws2;                          // side-stream scratch of the aggregated factors
    T *tu, *tw, *ty, *tq, *tb, *tt, *tt2;
    double *f1, *f2, *f3, *r, *v, *pAx, *pAtr, *pBx, *pBtv, *normpart, *norms2, *scal, *part;
    double *D;                           // column scaling (n), BF16 / TF32 factors
    double *ird;                         // state of the device-side refinement loop (IRD_WORDS)
    DualGemvPlan pa, pb;
};

template <typename T> struct GlsWs {
    int n, m, p, L, o, kC;
    int ldW, ldC, ldCt;                  // padded to 32 (TMA rows of 128 bytes)
    T *Wf, *tauW, *TwW, *Cf, *Ct, *tauC, *TwC, *Tw128W, *Tw128C, *DinvW, *DinvC;
    T *TfW, *TfC;                        // aggregated compact-WY factors (FP32 storage only)
    int ldtW, ldtC;
    float *PkW, *PkC;                    // packed block columns of R (m) and T~ (kC) for trsv64
    void *gws;                           // scratch of the two-level factorization
    void *wy;                            // scratch of the aggregated vector applications
    void *gws2;                          // side-stream scratch of the aggregated factors
    T *tu, *tw, *th, *tg, *tt, *tt2;
    double *f1, *f2, *f3, *z, *pWx, *pWtz, *pVy, *pVtz, *normpart, *norms2, *scal, *part;
    double *ird;                         // state of the device-side refinement loop (IRD_WORDS)
    DualGemvPlan pw, pv;
};

template <typename T> LseWs<T> lse_layout(void *base, int m, int n, int p, size_t *bytes)
{
    constexpr int NB = panel_nb<T>();
    Carver c(base);
    LseWs<T> w{};
    w.m = m; w.n = n; w.p = p; w.q = n - p; w.kA = std::min(m, n);
    const int mx = std::max(std::max(m, n), std::max(p, 1));
    w.ldBt = rup32(std::max(n, 1)); w.ldX = rup32(std::max(n, 1)); w.ldAt = rup32(std::max(m, 1));
    // B~ and X side by side: one factorization call leaves R~ over Q~^T X
    w.Bt = c.take<T>((size_t)w.ldBt * std::max(p + m, 1));
    w.X = w.Bt + (size_t)w.ldBt * p;
    w.tauB = c.take<T>(std::max(p, 1));
    w.TwB = c.take<T>((size_t)std::max(ceil_div(p, NB), 1) * NB * NB);
    w.Tw128B = c.take<T>((size_t)std::max(ceil_div(p, OUTER_NB), 1) * OUTER_NB * OUTER_NB);
    w.At = c.take<T>((size_t)w.ldAt * n);
    w.tauA = c.take<T>(std::max(w.kA, 1));
    w.TwA = c.take<T>((size_t)std::max(ceil_div(w.kA, NB), 1) * NB * NB);
    w.Tw128A = c.take<T>((size_t)std::max(ceil_div(w.kA, OUTER_NB), 1) * OUTER_NB * OUTER_NB);
    w.DinvB = c.take<T>(dinv_elems(p));
    w.DinvA = c.take<T>(dinv_elems(w.kA));
    if (sizeof(T) == 4)   // look-ahead factorizations of [B~ X] and A Q^T
        w.gws = c.take<unsigned char>(std::max(geqrf_la_ws_bytes(n, p + m), geqrf_la_ws_bytes(m, n)));
    else
        w.gws = c.take<unsigned char>(std::max(geqrf_ws_bytes(n, p + m), geqrf_ws_bytes(m, n)));
    w.ldtB = rup32(std::max(p, 1)); w.ldtA = rup32(std::max(w.kA, 1));
    if (sizeof(T) == 4) {
        w.TfB = c.take<T>((size_t)w.ldtB * std::max(p, 1));
        w.TfA = c.take<T>((size_t)w.ldtA * std::max(w.kA, 1));
        w.wy = c.take<unsigned char>(std::max(wy_apply_ws_bytes(n, p), wy_apply_ws_bytes(m, w.kA)));
        w.gws2 = c.take<unsigned char>(std::max(geqrf_ws_bytes(n, p + m), geqrf_ws_bytes(m, n)));
        w.PkB = c.take<float>(t64_pack_elems(p));
        w.PkA = c.take<float>(t64_pack_elems(w.kA));
    }
    w.tu = c.take<T>(mx); w.tw = c.take<T>(mx); w.ty = c.take<T>(mx); w.tq = c.take<T>(mx);
    w.tb = c.take<T>(mx); w.tt = c.take<T>(mx); w.tt2 = c.take<T>(mx);
    w.pa = dual_gemv_plan(m, n);
    w.pb = dual_gemv_plan(p, n);
    w.f1 = c.take<double>(mx); w.f2 = c.take<double>(mx); w.f3 = c.take<double>(mx);
    w.r = c.take<double>(mx); w.v = c.take<double>(mx);
    w.pAx = c.take<double>((size_t)std::max(w.pa.ncb, 1) * std::max(m, 1));
    w.pAtr = c.take<double>((size_t)std::max(w.pa.nrb, 1) * n);
    w.pBx = c.take<double>((size_t)std::max(w.pb.ncb, 1) * std::max(p, 1));
    w.pBtv = c.take<double>((size_t)std::max(w.pb.nrb, 1) * n);
    w.normpart = c.take<double>(304 * 6);
    w.norms2 = c.take<double>(8);
    w.scal = c.take<double>(16);
    w.part = c.take<double>(4096);
    w.D = c.take<double>(std::max(n, 1));
    w.ird = c.take<double>(IRD_WORDS);
    if (bytes) *bytes = c.used();
    return w;
}

template <typename T> GlsWs<T> gls_layout(void *base, int n, int m, int p, size_t *bytes)
{
    constexpr int NB = panel_nb<T>();
    Carver c(base);
    GlsWs<T> w{};
    w.n = n; w.m = m; w.p = p; w.L = n - m; w.o = p - n + m; w.kC = std::min(n, p);
    const int mx = std::max(std::max(m, n), std::max(p, 1));
    w.ldW = rup32(n); w.ldC = rup32(n); w.ldCt = rup32(std::max(p, 1));
    // W and C side by side: one factorization call leaves R over Q^T V
    w.Wf = c.take<T>((size_t)w.ldW * std::max(m + p, 1));
    w.Cf = w.Wf + (size_t)w.ldW * m;
    w.tauW = c.take<T>(std::max(m, 1));
    w.TwW = c.take<T>((size_t)std::max(ceil_div(m, NB), 1) * NB * NB);
    w.Tw128W = c.take<T>((size_t)std::max(ceil_div(m, OUTER_NB), 1) * OUTER_NB * OUTER_NB);
    w.Ct = c.take<T>((size_t)w.ldCt * n);
    w.tauC = c.take<T>(std::max(w.kC, 1));
    w.TwC = c.take<T>((size_t)std::max(ceil_div(w.kC, NB), 1) * NB * NB);
    w.Tw128C = c.take<T>((size_t)std::max(ceil_div(w.kC, OUTER_NB), 1) * OUTER_NB * OUTER_NB);
    w.DinvW = c.take<T>(dinv_elems(m));
    w.DinvC = c.take<T>(dinv_elems(w.kC));
    if (sizeof(T) == 4)   // look-ahead factorizations of [W V] and C~
        w.gws = c.take<unsigned char>(std::max(geqrf_la_ws_bytes(n, m + p), geqrf_la_ws_bytes(p, n)));
    else
        w.gws = c.take<unsigned char>(std::max(geqrf_ws_bytes(n, m + p), geqrf_ws_bytes(p, n)));
    w.ldtW = rup32(std::max(m, 1)); w.ldtC = rup32(std::max(w.kC, 1));
    if (sizeof(T) == 4) {
        w.TfW = c.take<T>((size_t)w.ldtW * std::max(m, 1));
        w.TfC = c.take<T>((size_t)w.ldtC * std::max(w.kC, 1));
        w.wy = c.take<unsigned char>(std::max(wy_apply_ws_bytes(n, m), wy_apply_ws_bytes(p, w.kC)));
        w.gws2 = c.take<unsigned char>(std::max(geqrf_ws_bytes(n, m + p), geqrf_ws_bytes(p, n)));
        w.PkW = c.take<float>(t64_pack_elems(m));
        w.PkC = c.take<float>(t64_pack_elems(w.kC));
    }
    w.tu = c.take<T>(mx); w.tw = c.take<T>(mx); w.th = c.take<T>(mx); w.tg = c.take<T>(mx);
    w.tt = c.take<T>(mx); w.tt2 = c.take<T>(mx);
    w.pw = dual_gemv_plan(n, m);
    w.pv = dual_gemv_plan(n, p);
    w.f1 = c.take<double>(mx); w.f2 = c.take<double>(mx); w.f3 = c.take<double>(mx);
    w.z = c.take<double>(mx);
    w.pWx = c.take<double>((size_t)std::max(w.pw.ncb, 1) * n);
    w.pWtz = c.take<double>((size_t)std::max(w.pw.nrb, 1) * std::max(m, 1));
    w.pVy = c.take<double>((size_t)std::max(w.pv.ncb, 1) * n);
    w.pVtz = c.take<double>((size_t)std::max(w.pv.nrb, 1) * p);
    w.normpart = c.take<double>(304 * 6);
    w.norms2 = c.take<double>(8);
    w.scal = c.take<double>(16);
    w.part = c.take<double>(4096);
    w.ird = c.take<double>(IRD_WORDS);
    if (bytes) *bytes = c.used();
    return w;
}

// Factor state held by the handle between step-level calls.
struct FactorState {
    Kind kind = Kind::NONE;
    int fact = MPIR_FP32;
    int m = 0, n = 0, p = 0;            // LSE (m, n, p) or GLS (n, m, p) as in the API
    double s1 = 1, s2 = 1;              // LSE: sA, sB ; GLS: sW, sV
    double fro1 = 0, fro2 = 0;          // ||A||_F, ||B||_F  /  ||W||_F, ||V||_F
    bool colscale = false;              // LSE factors of (sA A D, sB B D), x = D y
};

} // namespace

struct mpir_ctx {
    int device = 0;
    cudaStream_t stream = nullptr;
    void *ws = nullptr;
    size_t ws_bytes = 0;
    bool ws_owned = false;
    DevScratch sc{};
    void *scratch_base = nullptr;
    double *hbuf = nullptr;      // pinned host staging (64 doubles)
    std::string err;
    FactorState fs;
    cudaEvent_t ev[8];
    cudaEvent_t sw_ev = nullptr;         // orders a stream switch after queued work
    void *rws = nullptr;         // scratch of the standalone residual entry points
    size_t rws_bytes = 0;
    double *zbuf = nullptr;      // real embedding of a complex problem (zlse_solve / zgls_solve)
    size_t zbuf_bytes = 0;
    BatchArena ba;               // batched solves: tables, results, tuned shapes, graph
    cudaStream_t cap_stream = nullptr;   // private stream for graph capture
    // device-side classical refinement loop: the captured graph (a CUDA-graph
    // while loop) of the last shape / buffer set, and whether capture works
    cudaGraphExec_t irg = nullptr;
    unsigned long long irg_key = 0;
    bool irg_off = false;
    long long irg_pre[K_NKINDS] = {}, irg_body[K_NKINDS] = {};   // launches per part of the graph
    cudaStream_t side = nullptr;         // aggregated compact-WY factors, built beside the factorization
    cudaEvent_t side_fork = nullptr, side_join = nullptr;
    cudaStream_t crit = nullptr;         // high-priority stream of the factorization's critical path
    cudaEvent_t la_a = nullptr, la_b = nullptr;
    cudaStream_t aux = nullptr;          // outer-block factors beside the critical path
    cudaEvent_t ax_a = nullptr, ax_b = nullptr;
    TfullJob tfj{};
    // learned selector: parameters and feature standardization (device), scratch
    float *sel = nullptr;        // params[MLP_PARAMS], X[16], prob[6], feat[16]
    float sel_mean[16], sel_scale[16];
    double *sel_s = nullptr;     // start vector of the condition sketch
    size_t sel_s_len = 0;
    cudaStream_t sel_stream = nullptr;   // features + MLP, beside the speculative FP32 factorization
    cudaEvent_t sel_ev = nullptr;
    float *sel_host = nullptr;   // pinned: features (16) and class probabilities (8)
};

namespace {

int set_err(mpir_ctx *h, int code, const char *msg)
{
    if (h) h->err = msg ? msg : "";
    unsupported_where() = nullptr;
    return code;
}

// Job description for geqrf's aggregated factor (FP32 storage only); the
// side stream and its events are created on first use.
template <typename T>
const TfullJob *tfjob(mpir_ctx *h, T *Tf, int ldt, void *ws2)
{
    if (sizeof(T) != 4 || !Tf) return nullptr;
    if (!h->side) {
        if (cudaStreamCreateWithFlags(&h->side, cudaStreamNonBlocking) != cudaSuccess ||
            cudaEventCreateWithFlags(&h->side_fork, cudaEventDisableTiming) != cudaSuccess ||
            cudaEventCreateWithFlags(&h->side_join, cudaEventDisableTiming) != cudaSuccess) {
            cudaGetLastError();
            h->side = nullptr;
        }
    }
    if (!h->crit) {
        int lo = 0, hi = 0;
        cudaDeviceGetStreamPriorityRange(&lo, &hi);
        if (cudaStreamCreateWithPriority(&h->crit, cudaStreamNonBlocking, hi) != cudaSuccess ||
            cudaEventCreateWithFlags(&h->la_a, cudaEventDisableTiming) != cudaSuccess ||
            cudaEventCreateWithFlags(&h->la_b, cudaEventDisableTiming) != cudaSuccess) {
            cudaGetLastError();
            h->crit = nullptr;
        }
        if (h->crit &&
            (cudaStreamCreateWithPriority(&h->aux, cudaStreamNonBlocking, hi) != cudaSuccess ||
             cudaEventCreateWithFlags(&h->ax_a, cudaEventDisableTiming) != cudaSuccess ||
             cudaEventCreateWithFlags(&h->ax_b, cudaEventDisableTiming) != cudaSuccess)) {
            cudaGetLastError();
            h->aux = nullptr;
        }
    }
    h->tfj.Tf = reinterpret_cast<float *>(Tf);
    h->tfj.ldt = ldt;
    h->tfj.side = h->side;
    h->tfj.fork = h->side_fork;
    h->tfj.join = h->side_join;
    h->tfj.ws2 = ws2;
    h->tfj.crit = h->crit;
    h->tfj.la_a = h->la_a;
    h->tfj.la_b = h->la_b;
    h->tfj.aux = h->aux;
    h->tfj.ax_a = h->ax_a;
    h->tfj.ax_b = h->ax_b;
    return &h->tfj;
}

// The stream waits for everything queued on the side and critical-path
// streams so far.
void join_side(mpir_ctx *h, cudaStream_t s)
{
    if (h->side) {
        cudaEventRecord(h->side_join, h->side);
        cudaStreamWaitEvent(s, h->side_join, 0);
    }
    if (h->crit) {
        cudaEventRecord(h->la_a, h->crit);
        cudaStreamWaitEvent(s, h->la_a, 0);
    }
    if (h->aux) {
        cudaEventRecord(h->ax_a, h->aux);
        cudaStreamWaitEvent(s, h->ax_a, 0);
    }
}

int cuda_check(mpir_ctx *h, const char *where)
{
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) {
        if (h) h->err = std::string(where) + ": " + cudaGetErrorString(e);
        return MPIR_CUDA_ERROR;
    }
    return 0;
}

int ensure_ws(mpir_ctx *h, size_t bytes)
{
    if (h->ws_bytes >= bytes) return 0;
    if (h->ws && !h->ws_owned) return set_err(h, MPIR_UNSUPPORTED, "caller workspace too small");
    if (h->ws) {
        cudaStreamSynchronize(h->stream);
        if (h->side) cudaStreamSynchronize(h->side);
        if (h->crit) cudaStreamSynchronize(h->crit);
        if (h->aux) cudaStreamSynchronize(h->aux);
        cudaFree(h->ws); h->ws = nullptr; h->ws_bytes = 0;
    }
    h->fs.kind = Kind::NONE;             // factors held in the old buffer are gone
    if (cudaMalloc(&h->ws, bytes) != cudaSuccess) { cudaGetLastError(); return set_err(h, MPIR_CUDA_ERROR, "workspace cudaMalloc failed"); }
    h->ws_bytes = bytes;
    h->ws_owned = true;
    return 0;
}

int ensure_zbuf(mpir_ctx *h, size_t bytes)
{
    if (h->zbuf_bytes >= bytes) return 0;
    if (h->zbuf) {
        cudaStreamSynchronize(h->stream);
        cudaFree(h->zbuf);
        h->zbuf = nullptr;
        h->zbuf_bytes = 0;
    }
    if (cudaMalloc(&h->zbuf, bytes) != cudaSuccess) {
        cudaGetLastError();
        return set_err(h, MPIR_CUDA_ERROR, "complex embedding cudaMalloc failed");
    }
    h->zbuf_bytes = bytes;
    return 0;
}

int ensure_rws(mpir_ctx *h, size_t bytes)
{
    if (h->rws_bytes >= bytes) return 0;
    if (h->rws) {
        cudaStreamSynchronize(h->stream);
        if (h->sel_stream) cudaStreamSynchronize(h->sel_stream);    // the selector's features use it too
        cudaFree(h->rws);
        h->rws = nullptr;
        h->rws_bytes = 0;
    }
    if (cudaMalloc(&h->rws, bytes) != cudaSuccess) { cudaGetLastError(); return set_err(h, MPIR_CUDA_ERROR, "residual scratch cudaMalloc failed"); }
    h->rws_bytes = bytes;
    return 0;
}

// Scratch of a standalone residual: partials of the two dual gemvs.
struct ResWs {
    DualGemvPlan pa, pb;
    double *pA1, *pA2, *pB1, *pB2, *normpart, *norms2, *scal, *part;
};
ResWs res_layout(void *base, int ra, int ca, int rb, int cb, size_t *bytes)
{
    Carver c(base);
    ResWs w{};
    w.pa = dual_gemv_plan(ra, ca);
    w.pb = dual_gemv_plan(rb, cb);
    w.pA1 = c.take<double>((size_t)std::max(w.pa.ncb, 1) * std::max(ra, 1));
    w.pA2 = c.take<double>((size_t)std::max(w.pa.nrb, 1) * std::max(ca, 1));
    w.pB1 = c.take<double>((size_t)std::max(w.pb.ncb, 1) * std::max(rb, 1));
    w.pB2 = c.take<double>((size_t)std::max(w.pb.nrb, 1) * std::max(cb, 1));
    w.normpart = c.take<double>(304 * 6);
    w.norms2 = c.take<double>(8);
    w.scal = c.take<double>(16);
    w.part = c.take<double>(4096);
    if (bytes) *bytes = c.used();
    return w;
}

double pow2_scale(double amax)
{
    if (!(amax > 0) || !std::isfinite(amax)) return 1.0;
    int e = std::ilogb(amax) + 1;       // amax * 2^-e in [0.5, 1)
    return std::ldexp(1.0, -e);
}

double pow2_norm(double nrm)
{   // gamma with nrm * gamma in [0.5, 1)
    return pow2_scale(nrm);
}

// read `count` doubles from device to the pinned staging buffer (synchronous)
int read_back(mpir_ctx *h, const double *dptr, int count)
{
    cudaMemcpyAsync(h->hbuf, dptr, sizeof(double) * count, cudaMemcpyDeviceToHost, h->stream);
    if (cudaStreamSynchronize(h->stream) != cudaSuccess) return cuda_check(h, "sync");
    return 0;
}

int check_dev_flags(mpir_ctx *h)
{
    int flags[2] = {0, 0};
    cudaMemcpyAsync(&flags[0], h->sc.err, sizeof(int), cudaMemcpyDeviceToHost, h->stream);
    cudaMemcpyAsync(&flags[1], h->sc.status, sizeof(int), cudaMemcpyDeviceToHost, h->stream);
    if (cudaStreamSynchronize(h->stream) != cudaSuccess) return cuda_check(h, "sync");
    if (flags[0] & DEV_ERR_BARRIER_TIMEOUT) return set_err(h, MPIR_DEVICE_TIMEOUT, "device barrier timed out");
    if (flags[0] & 4) return set_err(h, MPIR_DEVICE_TIMEOUT, "tensor-core pipeline wait timed out");
    if (flags[0] & 8) return set_err(h, MPIR_DEVICE_TIMEOUT, "panel message wait timed out");
    if (flags[0] & 16) return set_err(h, MPIR_DEVICE_TIMEOUT, "triangular solve message wait timed out");
    if (flags[1] & 1) return set_err(h, MPIR_SINGULAR_R, "R has a zero diagonal entry");
    if (flags[1] & 2) return set_err(h, MPIR_SINGULAR_T, "triangular factor has a zero diagonal entry");
    return 0;
}

void clear_dev_flags(mpir_ctx *h)
{
    cudaMemsetAsync(h->sc.err, 0, sizeof(int), h->stream);
    cudaMemsetAsync(h->sc.status, 0, sizeof(int), h->stream);
}

GemmPrec gemm_prec(int fact)
{
    switch (fact) {
    case MPIR_BF16: return GemmPrec::BF16;
    case MPIR_TF32: return GemmPrec::TF32;
    case MPIR_FP64: return GemmPrec::FP64;
    default: return GemmPrec::FP32;
    }
}

#define RC(x) do { int _rc = (x); if (_rc) return _rc; } while (0)

// Triangular solve with FP32 or FP64 factors: FP32 factors of order <= 8192
// use 64-row diagonal blocks (inverses from inv_diag), others 32-row blocks.
// pk: the packed block columns of the order-npk triangle whose leading
// n x n block is solved (FP32 factors; nullptr reads U in place).
template <typename T>
int tsolve(const T *U, int ldu, int n, int trans, T *x, const DevScratch &sc, cudaStream_t s, const T *Dinv,
           const float *pk = nullptr, int npk = 0)
{
    if constexpr (sizeof(T) == 4) {
        if (trsv64_ok(n, sizeof(T))) {
            const int rc = trsv64<T>(U, ldu, n, trans, x, Dinv, pk, npk, sc.err, s);
            if (rc >= 0) return rc;
            return trsv_upper<T>(U, ldu, n, trans, x, sc, s, nullptr);
        }
    }
    return trsv_upper<T>(U, ldu, n, trans, x, sc, s, Dinv);
}
template <typename T>
void inv_diag(const T *U, int ldu, int N, T *Dinv, int *status, cudaStream_t s)
{
    if constexpr (sizeof(T) == 4) {
        if (trsv64_ok(N, sizeof(T))) { invert_diag64<T, T>(U, ldu, N, Dinv, status, s); return; }
    }
    invert_diag32<T>(U, ldu, N, Dinv, status, s);
}

// Reflector-set application to one vector with the widest compact-WY
// blocks the factorization kept: 128 (two-level FP32) or 16 (FP64).
template <typename T>
int vapply(const T *V, int ldv, int M, int K, const T *Tw, const T *Tw128, const T *Tf, int ldt, void *wy, int trans,
           T *x, const DevScratch &, cudaStream_t s)
{
    if (sizeof(T) == 4 && Tf) return wy_apply_vec<T, T>(V, ldv, M, K, Tf, ldt, trans, x, wy, s);
    if (sizeof(T) == 4) return apply_reflectors_vec_blk<T, T>(V, ldv, M, K, Tw128, OUTER_NB, trans, x, s);
    return apply_reflectors_vec_blk<T, T>(V, ldv, M, K, Tw, panel_nb<T>(), trans, x, s);
}

// T-vector combine: out[i] = alpha * a[ra ? n-1-i : i] + beta * b[rb ? n-1-i : i]
template <typename T>
__global__ void k_vcomb(T *out, int n, const T *a, int ra, T alpha, const T *b, int rb, T beta)
{
    pdl_wait();
    pdl_trigger();
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) {
        T v = alpha * a[ra ? n - 1 - i : i];
        if (b) v += beta * b[rb ? n - 1 - i : i];
        out[i] = v;
    }
}
template <typename T>
void vcomb(T *out, int n, const T *a, int ra, T alpha, const T *b, int rb, T beta, cudaStream_t s)
{
    if (n <= 0) return;
    ProfScope ps(K_ELEMWISE, s);
    pdl_launch(k_vcomb<T>, dim3(ceil_div(n, 256)), dim3(256), 0, s, out, n, a, ra, alpha, b, rb, beta);
}

__global__ void k_mask_lower(double *M, int ld, int rows, int cols, int off)
{
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    int j = blockIdx.y;
    if (i < rows && j < cols && i > j + off) M[idx2(i, j, ld)] = 0.0;
}

// ================================================================= GLS ==

template <typename T>
int gls_factor_impl(mpir_ctx *h, int n, int m, int p, const double *W, int ldw, const double *V, int ldv,
                    int fact)
{
    size_t bytes = 0;
    gls_layout<T>(nullptr, n, m, p, &bytes);
    RC(ensure_ws(h, bytes));
    GlsWs<T> w = gls_layout<T>(h->ws, n, m, p, nullptr);
    cudaStream_t s = h->stream;
    join_side(h, s);
    clear_dev_flags(h);
    absmax_sumsq(W, ldw, n, m, w.part, w.scal + 0, s);
    absmax_sumsq(V, ldv, n, p, w.part, w.scal + 2, s);
    RC(read_back(h, w.scal, 4));
    const double sW = pow2_scale(h->hbuf[0]), sV = pow2_scale(h->hbuf[2]);
    if (!std::isfinite(h->hbuf[1]) || !std::isfinite(h->hbuf[3]))
        return set_err(h, MPIR_NONFINITE, "non-finite entry in W or V");
    h->fs.kind = Kind::GLS;
    h->fs.fact = fact;
    h->fs.m = m; h->fs.n = n; h->fs.p = p;
    h->fs.s1 = sW; h->fs.s2 = sV;
    h->fs.fro1 = std::sqrt(h->hbuf[1]);
    h->fs.fro2 = std::sqrt(h->hbuf[3]);
    const GemmPrec gp = gemm_prec(fact);
    // QR of W (Lemma 4.6, first factorization) with C = Q^T V formed by the
    // same trailing updates: [W V] factored through its first m columns
    mconvert<double, T>(W, ldw, w.Wf, w.ldW, n, m, 0, 0, 0, sW, s);
    mconvert<double, T>(V, ldv, w.Cf, w.ldC, n, p, 0, 0, 0, sV, s);
    // as for LSE: the QR of W and the application of its Q to V stay
    // FP32-class; the dominant RQ of Q^T V runs at the class's precision
    const GemmPrec gp1 = gp == GemmPrec::FP64 ? gp : GemmPrec::FP32;
    RC(geqrf<T>(w.Wf, w.ldW, n, m + p, w.tauW, w.TwW, w.Tw128W, gp1, w.gws, h->sc.err, s,
                tfjob(h, w.TfW, w.ldtW, w.gws2), m));
    // RQ of C as QR of C~ = P_p C^T P_n
    mconvert<T, T>(w.Cf, w.ldC, w.Ct, w.ldCt, p, n, 1, 1, 1, 1.0, s);
    RC(geqrf<T>(w.Ct, w.ldCt, p, n, w.tauC, w.TwC, w.Tw128C, gp, w.gws, h->sc.err, s, tfjob(h, w.TfC, w.ldtC, w.gws2)));
    // inverses of the 32 x 32 diagonal blocks of R and T~ for the solves
    inv_diag<T>(w.Wf, w.ldW, m, w.DinvW, h->sc.status, s);
    inv_diag<T>(w.Ct, w.ldCt, w.L, w.DinvC, h->sc.status, s);   // T~_L, the block that is solved
    if constexpr (sizeof(T) == 4) {
        // block columns of R and of the whole T~ (the preconditioners solve
        // with its leading min(n, p) block) in the solves' read order
        RC(t64_pack(w.Wf, w.ldW, m, w.PkW, s));
        RC(t64_pack(w.Ct, w.ldCt, w.kC, w.PkC, s));
    }
    if (sizeof(T) == 4) join_side(h, s);
    return cuda_check(h, "gls_factor");
}

// Paige's method (Sec. 2.2) in reversed coordinates.  x, y FP64 outputs.
template <typename T>
int gls_initial_impl(mpir_ctx *h, const double *d, double *x, double *y)
{
    const FactorState &fs = h->fs;
    GlsWs<T> w = gls_layout<T>(h->ws, fs.n, fs.m, fs.p, nullptr);
    const int n = w.n, m = w.m, p = w.p, L = w.L;
    cudaStream_t s = h->stream;
    // c = Q^T (g d), g a power-of-two normalizer; x, y = result / g
    double *g = w.scal + 8;
    pow2_normalizer(d, n, 1.0, nullptr, 0, 0.0, g, s);
    vcopy<double, T>(d, w.tu, n, 1.0, 0, s, g);
    RC(vapply<T>(w.Wf, w.ldW, n, m, w.TwW, w.Tw128W, w.TfW, w.ldtW, w.wy, 1, w.tu, h->sc, s));
    // T22 s2 = c2  <=>  T~_L^T s~2 = P_L c2   (s~2 in tg[0:L], tg[L:p] = 0)
    vzero(w.tg, sizeof(T) * p, s);
    vcomb<T>(w.tg, L, w.tu + m, 1, T(1), nullptr, 0, T(0), s);
    RC(tsolve<T>(w.Ct, w.ldCt, L, 1, w.tg, h->sc, s, w.DinvC, w.PkC, w.kC));
    // R x = c1 - T12 s2,  P_m (T12 s2) = T~_12^T s~2
    RC(gemv<T>(w.Ct + idx2(0, L, w.ldCt), w.ldCt, L, m, 1, T(1), w.tg, T(0), w.tt, 0, 0, s));
    vcomb<T>(w.tt2, m, w.tu, 0, T(1), w.tt, 1, T(-1), s);
    RC(tsolve<T>(w.Wf, w.ldW, m, 0, w.tt2, h->sc, s, w.DinvW, w.PkW, w.m));
    vcopy<T, double>(w.tt2, x, m, fs.s1, 0, s, g + 1);
    // y = Z^T [0; s2] = P_p Z~ [s~2; 0]
    RC(vapply<T>(w.Ct, w.ldCt, p, w.kC, w.TwC, w.Tw128C, w.TfC, w.ldtC, w.wy, 0, w.tg, h->sc, s));
    vcopy<T, double>(w.tg, y, p, fs.s2, 1, s, g + 1);
    return cuda_check(h, "gls_initial");
}

// z0 = Q [0; h], T22^T h = (Z y)(p-n+m+1:p)  (Sec. 3.2, with Q in front).
template <typename T>
int gls_multipliers_impl(mpir_ctx *h, const double *y, double *z)
{
    const FactorState &fs = h->fs;
    GlsWs<T> w = gls_layout<T>(h->ws, fs.n, fs.m, fs.p, nullptr);
    const int n = w.n, m = w.m, p = w.p, L = w.L;
    cudaStream_t s = h->stream;
    // y' = y / sV ; w~ = Z~^T (P_p g y'), g a power-of-two normalizer
    double *g = w.scal + 8;
    pow2_normalizer(y, p, 1.0 / fs.s2, nullptr, 0, 0.0, g, s);
    vcopy<double, T>(y, w.tw, p, 1.0 / fs.s2, 1, s, g);
    RC(vapply<T>(w.Ct, w.ldCt, p, w.kC, w.TwC, w.Tw128C, w.TfC, w.ldtC, w.wy, 1, w.tw, h->sc, s));
    // T~_L h~2 = w~[0:L]
    vcomb<T>(w.th, L, w.tw, 0, T(1), nullptr, 0, T(0), s);
    RC(tsolve<T>(w.Ct, w.ldCt, L, 0, w.th, h->sc, s, w.DinvC, w.PkC, w.kC));
    // z' = Q [0_m; P_L h~2]
    vzero(w.tt, sizeof(T) * n, s);
    vcomb<T>(w.tt + m, L, w.th, 1, T(1), nullptr, 0, T(0), s);
    RC(vapply<T>(w.Wf, w.ldW, n, m, w.TwW, w.Tw128W, w.TfW, w.ldtW, w.wy, 0, w.tt, h->sc, s));
    vcopy<T, double>(w.tt, z, n, fs.s2 * fs.s2, 0, s, g + 1);
    return cuda_check(h, "gls_multipliers");
}

// Alg. 3 in reversed coordinates; the results are ADDED (scaled) to
// (dy, dz, dx).  gamma normalizes the right-hand side.
template <typename T>
int gls_correction_impl(mpir_ctx *h, const double *f1, const double *f2, const double *f3, double gamma,
                        double *dy, double *dz, double *dx, const double *dsc = nullptr)
{
    const FactorState &fs = h->fs;
    GlsWs<T> w = gls_layout<T>(h->ws, fs.n, fs.m, fs.p, nullptr);
    const int n = w.n, m = w.m, p = w.p, L = w.L, o = w.o;
    const double sW = fs.s1, sV = fs.s2;
    // host scales, or the device scalars (c1, c2, c3, i1, i2, i3) of the
    // device-side loop: i1 for dy, i2 for dz, i3 for dx
    const double c1 = dsc ? 1.0 : gamma, c2 = dsc ? 1.0 : gamma * sV, c3 = dsc ? 1.0 : gamma * sW / sV;
    const double i1 = dsc ? 1.0 : 1.0 / gamma, i2 = dsc ? 1.0 : -sV / gamma, i3 = dsc ? 1.0 : sW / sV / gamma;
    const double *d1 = dsc, *d2 = dsc ? dsc + 1 : nullptr, *d3 = dsc ? dsc + 2 : nullptr;
    const double *e1 = dsc ? dsc + 3 : nullptr, *e2 = dsc ? dsc + 4 : nullptr, *e3 = dsc ? dsc + 5 : nullptr;
    cudaStream_t s = h->stream;
    // step 1: u = Q^T f2'
    vcopy<double, T>(f2, w.tu, n, c2, 0, s, d2);
    RC(vapply<T>(w.Wf, w.ldW, n, m, w.TwW, w.Tw128W, w.TfW, w.ldtW, w.wy, 1, w.tu, h->sc, s));
    // step 2: w~ = Z~^T (P_p f1') = P_p (Z f1')
    vcopy<double, T>(f1, w.tw, p, c1, 1, s, d1);
    RC(vapply<T>(w.Ct, w.ldCt, p, w.kC, w.TwC, w.Tw128C, w.TfC, w.ldtC, w.wy, 1, w.tw, h->sc, s));
    // step 3: R^T h1 = f3'   (th[0:m] = h1)
    vcopy<double, T>(f3, w.th, m, c3, 0, s, d3);
    RC(tsolve<T>(w.Wf, w.ldW, m, 1, w.th, h->sc, s, w.DinvW, w.PkW, w.m));
    // h~1 = P_m h1 (tt)
    vcomb<T>(w.tt, m, w.th, 1, T(1), nullptr, 0, T(0), s);
    // step 4: T22 g2 = u2  <=>  T~_L^T g~2 = P_L u2   (tg[0:L] = g~2)
    vcomb<T>(w.tg, L, w.tu + m, 1, T(1), nullptr, 0, T(0), s);
    RC(tsolve<T>(w.Ct, w.ldCt, L, 1, w.tg, h->sc, s, w.DinvC, w.PkC, w.kC));
    // step 5: T22^T h2 = w2 - g2 - T12^T h1  <=>  T~_L h~2 = w~2 - g~2 - T~_12 h~1
    RC(gemv<T>(w.Ct + idx2(0, L, w.ldCt), w.ldCt, L, m, 0, T(1), w.tt, T(0), w.tt2, 0, 0, s));
    vcomb<T>(w.th + m, L, w.tw, 0, T(1), w.tg, 0, T(-1), s);
    vcomb<T>(w.th + m, L, w.th + m, 0, T(1), w.tt2, 0, T(-1), s);
    RC(tsolve<T>(w.Ct, w.ldCt, L, 0, w.th + m, h->sc, s, w.DinvC, w.PkC, w.kC));
    // step 6: g1 = w1 - T11^T h1  <=>  g~1 = w~1 - T~_22 h~1   (tg[L:p])
    if (o > 0) {
        vcomb<T>(w.tg + L, o, w.tw + L, 0, T(1), nullptr, 0, T(0), s);
        RC(gemv<T>(w.Ct + idx2(L, L, w.ldCt), w.ldCt, o, m, 0, T(-1), w.tt, T(1), w.tg + L, 1, 0, s));
    }
    // step 8 (before the in-place apply of step 7):
    // R dx = u1 - T11 g1 - T12 g2,  P_m(T11 g1 + T12 g2) = T~_22^T g~1 + T~_12^T g~2
    RC(gemv<T>(w.Ct + idx2(0, L, w.ldCt), w.ldCt, L, m, 1, T(1), w.tg, T(0), w.tt2, 0, 0, s));
    if (o > 0) RC(gemv<T>(w.Ct + idx2(L, L, w.ldCt), w.ldCt, o, m, 1, T(1), w.tg + L, T(1), w.tt2, 1, 0, s));
    vcomb<T>(w.tt, m, w.tu, 0, T(1), w.tt2, 1, T(-1), s);
    RC(tsolve<T>(w.Wf, w.ldW, m, 0, w.tt, h->sc, s, w.DinvW, w.PkW, w.m));
    vaxpy<T>(w.tt, dx, m, i3, 0, s, e3);
    // step 7: dy = Z^T g = P_p Z~ g~
    RC(vapply<T>(w.Ct, w.ldCt, p, w.kC, w.TwC, w.Tw128C, w.TfC, w.ldtC, w.wy, 0, w.tg, h->sc, s));
    vaxpy<T>(w.tg, dy, p, i1, 1, s, e1);
    //         dz = -Q h,  h = [h1; P_L h~2]
    vcomb<T>(w.tt2, L, w.th + m, 1, T(1), nullptr, 0, T(0), s);
    cudaMemcpyAsync(w.th + m, w.tt2, sizeof(T) * L, cudaMemcpyDeviceToDevice, s);
    RC(vapply<T>(w.Wf, w.ldW, n, m, w.TwW, w.Tw128W, w.TfW, w.ldtW, w.wy, 0, w.th, h->sc, s));
    vaxpy<T>(w.th, dz, n, i2, 0, s, e2);
    return cuda_check(h, "gls_correction");
}

// FP64 residual of eq. aug-GLS + squared norms into w.norms2 (device).
template <typename T>
void gls_residual_dev(mpir_ctx *h, GlsWs<T> &w, const double *W, int ldw, const double *V, int ldv,
                      const double *d, const double *x, const double *y, const double *z)
{
    cudaStream_t s = h->stream;
    const int n = w.n, m = w.m, p = w.p;
    dual_gemv(W, ldw, n, m, x, z, w.pWx, w.pWtz, s);
    dual_gemv(V, ldv, n, p, y, z, w.pVy, w.pVtz, s);
    gls_resid_finalize(n, m, p, d, x, y, z, w.pWx, w.pw.ncb, w.pWtz, w.pw.nrb, w.pVy, w.pv.ncb, w.pVtz,
                       w.pv.nrb, w.f1, w.f2, w.f3, w.normpart, w.norms2, s);
}

double dnorm_host(mpir_ctx *h, const double *dvec, int n, double *scratch);

// ----------------------------------------------- device-side refinement loop --
// The classical loop (Alg. 2 / Alg. 4) without a host decision per step: a
// one-thread control kernel after each residual applies eq. lse-stop /
// gls-stop and the stagnation rule to the squared norms on the device,
// records the step count, status and ratios, leaves the power-of-two scales
// of the next correction (gamma normalizes the scaled right-hand side) and
// sets the condition of a CUDA-graph while node: the graph is
//     reset, ||b||, ||d||, residual, control; while (cond) { correction,
//     residual, control }
// and the host reads the final state once.
__global__ void k_ir_reset(double *__restrict__ ird)
{
    if (threadIdx.x != 0) return;
    ird[IRD_BEST] = INFINITY;
    ird[IRD_SINCE] = 0.0;
    ird[IRD_IT] = 0.0;
    ird[IRD_STATUS] = -1.0;
    for (int k = 0; k < 4; k++) ird[IRD_N1 + k] = 0.0;
}

__device__ __forceinline__ double ir_pow2(double v)
{   // 2^-e with v 2^-e in [0.5, 1); 1 for 0 or non-finite v
    if (!(v > 0.0) || !isfinite(v)) return 1.0;
    return ldexp(1.0, -(ilogb(v) + 1));
}

// kind 0: LSE, norms2 = squares of ||f1||, ||f2||, ||f3||, ||x||, ||r||, ||v||;
// kind 1: GLS, ||f1||, ||f2||, ||f3||, ||x||, ||y||, ||z||.
__global__ void k_ir_control(const double *__restrict__ norms2, double *__restrict__ ird, int kind, double tol,
                             int maxit, cudaGraphConditionalHandle hc, int use_hc)
{
    if (threadIdx.x != 0) return;
    double nr[6];
    for (int k = 0; k < 6; k++) nr[k] = sqrt(norms2[k]);
    const double s1 = ird[IRD_S1], s2 = ird[IRD_S2], f1 = ird[IRD_F1], f2 = ird[IRD_F2];
    double den[3];
    if (kind == 0) {
        const double nb = sqrt(ird[IRD_N1 + 1]), nd = sqrt(ird[IRD_N2 + 1]);
        den[0] = nb + nr[4] + f1 * nr[3];
        den[1] = nd + f2 * nr[3];
        den[2] = f1 * nr[4] + f2 * nr[5];
    } else {
        const double nd = sqrt(ird[IRD_N1 + 1]);
        den[0] = nr[4] + f2 * nr[5];
        den[1] = nd + f1 * nr[3] + f2 * nr[4];
        den[2] = f1 * nr[5];
    }
    bool ok = true, fin = true;
    for (int k = 0; k < 3; k++) {
        const double rt = den[k] > 0 ? nr[k] / den[k] : (nr[k] > 0 ? INFINITY : 0.0);
        ird[IRD_RATIO + k] = rt;
        if (!(nr[k] <= tol * den[k])) ok = false;
        if (!isfinite(nr[k])) fin = false;
    }
    const int it = (int)ird[IRD_IT];
    int status = -1;
    if (!fin) status = MPIR_NONFINITE;
    else if (ok) status = MPIR_OK;
    else {
        const double eta = fmax(ird[IRD_RATIO], fmax(ird[IRD_RATIO + 1], ird[IRD_RATIO + 2]));
        double best = ird[IRD_BEST];
        int since = (int)ird[IRD_SINCE];
        if (eta < 0.5 * best) { best = eta; since = 0; }
        else if (++since >= 3) status = best <= 1e-14 ? MPIR_OK : MPIR_NOT_CONVERGED;
        ird[IRD_BEST] = best;
        ird[IRD_SINCE] = since;
        if (status < 0 && it >= maxit) status = MPIR_NOT_CONVERGED;
    }
    ird[IRD_STATUS] = status;
    if (status < 0) {
        double g;
        if (kind == 0) {       // scaled system (f1, sB/sA f2, sA f3)
            g = ir_pow2(fmax(nr[0], fmax(nr[1] * s2 / s1, nr[2] * s1)));
            ird[IRD_C] = g; ird[IRD_C + 1] = g * s2 / s1; ird[IRD_C + 2] = g * s1;
            ird[IRD_I] = 1.0 / g; ird[IRD_I + 1] = s2 / s1 / g; ird[IRD_I + 2] = s1 / g;
        } else {               // scaled system (f1, sV f2, sW/sV f3)
            g = ir_pow2(fmax(nr[0], fmax(nr[1] * s2, nr[2] * s1 / s2)));
            ird[IRD_C] = g; ird[IRD_C + 1] = g * s2; ird[IRD_C + 2] = g * s1 / s2;
            ird[IRD_I] = 1.0 / g; ird[IRD_I + 1] = -s2 / g; ird[IRD_I + 2] = s1 / s2 / g;
        }
        ird[IRD_IT] = it + 1;
    }
    if (use_hc) cudaGraphSetConditional(hc, status < 0 ? 1u : 0u);
}

static unsigned long long ir_mix(unsigned long long h, unsigned long long v)
{
    h ^= v + 0x9e3779b97f4a7c15ULL + (h << 6) + (h >> 2);
    return h;
}

// Runs the device-side loop: (re)captures the graph when the key changes,
// stages the per-solve scalars (s1, s2, ||.||_F of both matrices), launches
// on the handle's stream and reads the final state back (the one host
// synchronization of the loop).  pre(hc) / body(hc) enqueue the two parts on
// h->stream (the capture stream while capturing).  Returns 0, or a positive
// code when the graph could not be built (the caller then runs the host loop).
template <typename Pre, typename Body>
static int ir_graph_run(mpir_ctx *h, double *ird, unsigned long long key, Pre pre, Body body, int *it_out,
                        int *st_out, double ratio[3])
{
    if (!h->cap_stream && cudaStreamCreateWithFlags(&h->cap_stream, cudaStreamNonBlocking) != cudaSuccess) {
        cudaGetLastError();
        return 1;
    }
    if (!h->irg || h->irg_key != key) {
        if (h->irg) { cudaGraphExecDestroy(h->irg); h->irg = nullptr; }
        cudaStream_t user = h->stream, cs = h->cap_stream;
        cudaGraph_t g = nullptr;
        cudaGraphConditionalHandle hc{};
        bool okc = cudaGraphCreate(&g, 0) == cudaSuccess && cudaGraphConditionalHandleCreate(&hc, g, 0, 0) == cudaSuccess;
        cudaGraphNodeParams cp{};
        if (okc) okc = cudaStreamBeginCaptureToGraph(cs, g, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal) ==
                       cudaSuccess;
        long long c0[K_NKINDS], c1[K_NKINDS], c2[K_NKINDS];
        prof_snapshot(c0);
        std::copy(c0, c0 + K_NKINDS, c1);
        std::copy(c0, c0 + K_NKINDS, c2);
        if (okc) {
            h->stream = cs;
            const int rc = pre(hc);
            prof_snapshot(c1);
            cudaStreamCaptureStatus cst;
            cudaGraph_t gc = nullptr;
            const cudaGraphNode_t *deps = nullptr;
            const cudaGraphEdgeData *edata = nullptr;
            size_t nd = 0;
            okc = rc == 0 && cudaStreamGetCaptureInfo(cs, &cst, nullptr, &gc, &deps, &edata, &nd) == cudaSuccess &&
                  cst == cudaStreamCaptureStatusActive;
            cudaGraphNode_t node = nullptr;
            if (okc) {
                cp.type = cudaGraphNodeTypeConditional;
                cp.conditional.handle = hc;
                cp.conditional.type = cudaGraphCondTypeWhile;
                cp.conditional.size = 1;
                okc = cudaGraphAddNode(&node, gc, deps, edata, nd, &cp) == cudaSuccess &&
                      cudaStreamUpdateCaptureDependencies(cs, &node, nullptr, 1, cudaStreamSetCaptureDependencies) ==
                          cudaSuccess;
            }
            cudaGraph_t gend = nullptr;
            if (cudaStreamEndCapture(cs, &gend) != cudaSuccess) okc = false;
            if (okc) {
                cudaGraph_t bodyg = cp.conditional.phGraph_out[0];
                okc = cudaStreamBeginCaptureToGraph(cs, bodyg, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal) ==
                      cudaSuccess;
                if (okc) {
                    const int rb = body(hc);
                    prof_snapshot(c2);
                    cudaGraph_t gb = nullptr;
                    if (cudaStreamEndCapture(cs, &gb) != cudaSuccess || rb != 0) okc = false;
                }
            }
            h->stream = user;
        }
        if (okc) okc = cudaGraphInstantiate(&h->irg, g, 0) == cudaSuccess;
        if (g) cudaGraphDestroy(g);
        if (!okc) {
            h->irg = nullptr;
            cudaGetLastError();
            return 1;
        }
        h->irg_key = key;
        for (int k = 0; k < K_NKINDS; k++) {
            h->irg_pre[k] = c1[k] - c0[k];
            h->irg_body[k] = c2[k] - c1[k];
        }
        // the capture counted one pass of each part; replays are added below
        for (int k = 0; k < K_NKINDS; k++) g_launches[k].fetch_sub(c2[k] - c0[k], std::memory_order_relaxed);
    }
    if (cudaGraphLaunch(h->irg, h->stream) != cudaSuccess) return cuda_check(h, "refinement graph launch");
    RC(read_back(h, ird, IRD_RATIO + 3));
    prof_add(h->irg_pre, 1);
    prof_add(h->irg_body, (long long)h->hbuf[IRD_IT] - 0);
    *it_out = (int)h->hbuf[IRD_IT];
    *st_out = (int)h->hbuf[IRD_STATUS];
    for (int k = 0; k < 3; k++) ratio[k] = h->hbuf[IRD_RATIO + k];
    return 0;
}

// Stages s1, s2, ||.||_F, ||.||_F of the held factorization into ird.
static void ir_stage_scalars(mpir_ctx *h, double *ird)
{
    double *hb = h->hbuf + 48;
    hb[0] = h->fs.s1; hb[1] = h->fs.s2; hb[2] = h->fs.fro1; hb[3] = h->fs.fro2;
    cudaMemcpyAsync(ird + IRD_S1, hb, 4 * sizeof(double), cudaMemcpyHostToDevice, h->stream);
}

static bool ir_graph_usable(mpir_ctx *h) { return !h->irg_off && !g_prof; }

struct StopState {
    double best = INFINITY;
    int since_best = 0;
};

// The u_r < u variant (double-double residuals): once the backward error
// meets the stop test the refinement goes on while the corrections keep
// shrinking, until ||dx|| <= 4 u ||x|| or a correction is no smaller than
// half the previous one (the forward error then sits at about u).
struct FwdState {
    double last = INFINITY, prev = INFINITY;
    bool have = false;
    bool done(double nx) const { return have && (last <= 4.0 * 1.1102230246251565e-16 * nx || last > 0.5 * prev); }
    void push(double dx) { prev = last; last = dx; have = true; }
};

// eq. gls-stop / eq. lse-stop from squared norms; returns 1 if satisfied.
int stop_test(const double *nrm, const double den[3], double tol, double ratio[3])
{
    int ok = 1;
    for (int i = 0; i < 3; i++) {
        ratio[i] = den[i] > 0 ? nrm[i] / den[i] : (nrm[i] > 0 ? INFINITY : 0.0);
        if (!(nrm[i] <= tol * den[i])) ok = 0;
    }
    return ok;
}

void fill_opts(const mpir_opts *in, mpir_opts *o)
{
    mpir_default_opts(o);
    if (!in) return;
    *o = *in;
    if (o->tol <= 0) o->tol = 1e-15;
    if (o->maxit <= 0) o->maxit = 40;
    if (o->restart <= 0) o->restart = 30;
    if (o->inner_maxit <= 0) o->inner_maxit = 300;
    if (o->beta <= 0) o->beta = 1.0;
}

float ev_ms(cudaEvent_t a, cudaEvent_t b)
{
    float t = 0;
    cudaEventElapsedTime(&t, a, b);
    return t;
}


// ============================================== GMRES-IR (Sec. 5) ==
// Block-diagonal split preconditioners built from the held factors and
// applied in FP64 arithmetic to FP64 vectors (the factors stay in their
// storage precision), the scaled augmented operator F~(alpha, beta) on the
// FP64 originals, and the outer loop that solves each correction system with
// restarted GMRES instead of Alg. 1 / Alg. 3.
//
// Scaled factors.  The factors held are those of sA A, sB B (sW W, sV V), so
// R = R'/sB, T = T'/sA for LSE (R = R'/sW, T = T'/sV for GLS); the scalars
// below fold these ratios into the preconditioner's block scalings.

// Scratch of the operator and of the GMRES engine.
// dT, dR: FP64 inverses of the 32 x 32 diagonal blocks of the two
// triangular factors the preconditioners solve with (computed once per
// factorization from the stored factors; the solves then form each block
// by a 32-wide product instead of a substitution chain).
struct BDScratch {
    GmresWs gw;
    double *rhs, *t, *u, *gf, *w1, *w2, *w3;
    double *dT, *dR;
};

size_t bd_bytes(int N, int R, int mx)
{
    size_t b = gmres_ws_bytes(N, R);
    const size_t vn = ((size_t)N * sizeof(double) + 255) & ~(size_t)255;
    const size_t vm = ((size_t)std::max(mx, 1) * sizeof(double) + 255) & ~(size_t)255;
    const size_t vd = dinv_elems(mx) * sizeof(double);
    return b + 4 * vn + 3 * vm + 2 * vd;
}

BDScratch bd_layout(void *base, int N, int R, int mx)
{
    BDScratch b{};
    b.gw = gmres_layout(base, N, R);
    Carver c((char *)base + gmres_ws_bytes(N, R));
    b.rhs = c.take<double>(N); b.t = c.take<double>(N); b.u = c.take<double>(N); b.gf = c.take<double>(N);
    b.w1 = c.take<double>(std::max(mx, 1)); b.w2 = c.take<double>(std::max(mx, 1));
    b.w3 = c.take<double>(std::max(mx, 1));
    b.dT = c.take<double>(dinv_elems(mx));
    b.dR = c.take<double>(dinv_elems(mx));
    return b;
}

// Triangular solve and gemv in FP64 arithmetic on factors stored as T.
// FP32 factors of order <= 8192 use 64-row diagonal blocks (inverses from
// inv_diag_d), others 32-row blocks.
template <typename T>
int trsv_d(const T *U, int ldu, int n, int trans, double *x, const DevScratch &sc, cudaStream_t s,
           const double *Dinv, const float *pk = nullptr, int npk = 0)
{
    if constexpr (sizeof(T) == 4) {
        if (trsv64_ok(n, sizeof(T))) {
            const int rc = trsv64<double>(U, ldu, n, trans, x, Dinv, pk, npk, sc.err, s);
            if (rc >= 0) return rc;
            return trsv_upper_mixed<T, double>(U, ldu, n, trans, x, sc, s, nullptr);
        }
    }
    return trsv_upper_mixed<T, double>(U, ldu, n, trans, x, sc, s, Dinv);
}
template <typename T>
void inv_diag_d(const T *U, int ldu, int N, double *Dinv, int *status, cudaStream_t s)
{
    if constexpr (sizeof(T) == 4) {
        if (trsv64_ok(N, sizeof(T))) { invert_diag64<T, double>(U, ldu, N, Dinv, status, s); return; }
    }
    invert_diag32_mixed<T, double>(U, ldu, N, Dinv, status, s);
}
template <typename T>
int gemv_d(const T *M, int ld, int rows, int cols, int trans, double alpha, const double *x, double beta, double *y,
           int upper_mask, int diag_off, cudaStream_t s)
{
    return gemv_mixed<T, double>(M, ld, rows, cols, trans, alpha, x, beta, y, upper_mask, diag_off, s);
}

// Reflector set applied in FP64 arithmetic to an FP64 vector.
template <typename T>
int vapply_d(const T *V, int ldv, int M, int K, const T *Tw, const T *Tw128, const T *Tf, int ldt, void *wy,
             int trans, double *x, cudaStream_t s)
{
    if (sizeof(T) == 4 && Tf) return wy_apply_vec<T, double>(V, ldv, M, K, Tf, ldt, trans, x, wy, s);
    if (sizeof(T) == 4) return apply_reflectors_vec_blk<T, double>(V, ldv, M, K, Tw128, OUTER_NB, trans, x, s);
    return apply_reflectors_vec_blk<T, double>(V, ldv, M, K, Tw, panel_nb<T>(), trans, x, s);
}

// The triangular factor of the wide shapes (eq. lse-bdpre-nlarge,
// eq. gls-bdpre-nlarge): U = [T; 0, c I_{N-r}] (N x N) with T the r x N upper
// trapezoid held at (Tp, ld), r <= N (r = N: U = T's leading triangle).  c
// is the power-of-two scale of the factored matrix (T holds c times the
// factor of the unscaled one, so the identity block scales with it).
// Solves U x = t (trans 0) or U^T x = t (trans 1) in place: one triangular
// solve with T's leading r x r block and one product with its trailing
// r x (N - r) block.  Dinv: FP64 inverses of the diagonal blocks of the
// leading r x r block.
template <typename T>
int trsv_trap(mpir_ctx *h, const T *Tp, int ld, int r, int N, double c, int trans, double *x, const double *Dinv,
              cudaStream_t s, const float *pk = nullptr, int npk = 0)
{
    if (r >= N) return trsv_d<T>(Tp, ld, N, trans, x, h->sc, s, Dinv, pk, npk);
    if (!trans) {                      // c x2 = t2;  T11 x1 = t1 - T12 x2
        vcomb<double>(x + r, N - r, x + r, 0, 1.0 / c, nullptr, 0, 0.0, s);
        RC(gemv_d<T>(Tp + idx2(0, r, ld), ld, r, N - r, 0, -1.0, x + r, 1.0, x, 0, 0, s));
        return trsv_d<T>(Tp, ld, r, 0, x, h->sc, s, Dinv, pk, npk);
    }
    RC(trsv_d<T>(Tp, ld, r, 1, x, h->sc, s, Dinv, pk, npk));      // T11^T x1 = t1
    RC(gemv_d<T>(Tp + idx2(0, r, ld), ld, r, N - r, 1, -1.0, x, 1.0, x + r, 0, 0, s));   // t2 - T12^T x1
    vcomb<double>(x + r, N - r, x + r, 0, 1.0 / c, nullptr, 0, 0.0, s);                  // x2 = (...) / c
    return 0;
}

// y = S x (trans 0) or S^T x (trans 1) for the trailing block S = U(o:N, o:N)
// of the U above (k = N - o): its first r - o rows come from T (upper part),
// the others are c times identity rows.  x and y distinct, length k.
template <typename T>
int trap_tail_gemv(const T *Tp, int ld, int r, int N, int o, double c, int trans, const double *x, double *y,
                   cudaStream_t s)
{
    const int k = N - o, kr = std::max(std::min(r, N) - o, 0);
    const T *S = Tp + idx2(o, o, ld);
    if (kr >= k) return gemv_d<T>(S, ld, k, k, trans, 1.0, x, 0.0, y, 1, 0, s);
    if (!trans) {
        if (kr > 0) RC(gemv_d<T>(S, ld, kr, k, 0, 1.0, x, 0.0, y, 1, 0, s));
        vcomb<double>(y + kr, k - kr, x + kr, 0, c, nullptr, 0, 0.0, s);
        return 0;
    }
    vzero(y, sizeof(double) * (size_t)kr, s);
    vcomb<double>(y + kr, k - kr, x + kr, 0, c, nullptr, 0, 0.0, s);
    if (kr > 0) RC(gemv_d<T>(S, ld, kr, k, 1, 1.0, x, 1.0, y, 1, 0, s));
    return 0;
}

// GLS (Sec. 5.3):  F~ = [a I, V^T, 0; V, 0, b W; 0, b W^T, 0] on
// u = [u1 (p); u2 (n); u3 (m)];  T = [0, T2] (T2 n x n), S = T2(1:m, 1:m),
//   M_l = diag(a^-1/2 I, a^1/2 T2^-1 Q^T, a^-1/2 b^-1 S^T R^-T),
//   M_r = diag(a^-1/2 I, a^1/2 Q T2^-T,  a^-1/2 b^-1 R^-1 S).
// Reversed coordinates: T2 = P_n T~_n^T P_n (T~_n the leading n x n of the
// factor of C~) and S = P_m T~_S^T P_m, T~_S = T~_n(L:n, L:n), L = n - m.
// n > p (eq. gls-bdpre-nlarge): T = [T^1; T^2] (n x p), T2 = [I, T^1; 0, T^2],
// which reversed is T~_n = [T~; 0, I_{n-p}] with T~ the p x n factor of C~.
template <typename T>
struct GlsBDOp : LinOp {
    mpir_ctx *h;
    GlsWs<T> &w;
    BDScratch &b;
    const double *W, *V;
    int ldw, ldv;
    double al, be;
    GlsBDOp(mpir_ctx *h_, GlsWs<T> &w_, BDScratch &b_, const double *W_, int ldw_, const double *V_, int ldv_,
            double al_, double be_)
        : h(h_), w(w_), b(b_), W(W_), V(V_), ldw(ldw_), ldv(ldv_), al(al_), be(be_) {}

    // rows of the factor of C~ held (n > p: U = [T~; 0, I], eq. gls-bdpre-nlarge)
    int rT() const { return std::min(w.n, w.p); }

    // FP64 inverses of the diagonal blocks of T~_n and R
    void prepare()
    {
        inv_diag_d<T>(w.Ct, w.ldCt, rT(), b.dT, h->sc.status, h->stream);
        inv_diag_d<T>(w.Wf, w.ldW, w.m, b.dR, h->sc.status, h->stream);
    }

    int Mr(const double *t, double *u)
    {
        const int n = w.n, m = w.m, p = w.p;
        const double sW = h->fs.s1, sV = h->fs.s2, sa = std::sqrt(al);
        cudaStream_t s = h->stream;
        vcomb<double>(u, p, t, 0, 1.0 / sa, nullptr, 0, 0.0, s);
        // a^1/2 Q T2^-T t2 = a^1/2 sV Q P_n T~_n'^-1 P_n t2
        vcomb<double>(b.w1, n, t + p, 1, 1.0, nullptr, 0, 0.0, s);
        RC(trsv_trap<T>(h, w.Ct, w.ldCt, rT(), n, sV, 0, b.w1, b.dT, s, w.PkC, w.kC));
        vcomb<double>(u + p, n, b.w1, 1, sa * sV, nullptr, 0, 0.0, s);
        RC(vapply_d<T>(w.Wf, w.ldW, n, m, w.TwW, w.Tw128W, w.TfW, w.ldtW, w.wy, 0, u + p, s));
        if (m > 0) {
            // a^-1/2 b^-1 R^-1 S t3 = a^-1/2 b^-1 (sW/sV) R'^-1 P_m T~_S'^T P_m t3
            vcomb<double>(b.w1, m, t + p + n, 1, 1.0, nullptr, 0, 0.0, s);
            RC(trap_tail_gemv<T>(w.Ct, w.ldCt, rT(), n, w.L, sV, 1, b.w1, b.w2, s));
            vcomb<double>(u + p + n, m, b.w2, 1, sW / (sV * sa * be), nullptr, 0, 0.0, s);
            RC(trsv_d<T>(w.Wf, w.ldW, m, 0, u + p + n, h->sc, s, b.dR, w.PkW, w.m));
        }
        return 0;
    }

    int Fmul(const double *u, double *g)
    {
        const int n = w.n, m = w.m, p = w.p;
        cudaStream_t s = h->stream;
        if (m > 0) dual_gemv(W, ldw, n, m, u + p + n, u + p, w.pWx, w.pWtz, s);
        dual_gemv(V, ldv, n, p, u, u + p, w.pVy, w.pVtz, s);
        combine_parts(g, p, al, u, 1.0, w.pVtz, w.pv.nrb, p, 0.0, nullptr, 0, 0, s);
        combine_parts(g + p, n, 0.0, nullptr, 1.0, w.pVy, w.pv.ncb, n, be, m > 0 ? w.pWx : nullptr, w.pw.ncb, n,
                      s);
        if (m > 0) combine_parts(g + p + n, m, 0.0, nullptr, be, w.pWtz, w.pw.nrb, m, 0.0, nullptr, 0, 0, s);
        return 0;
    }

    int Ml(const double *g, double *o)
    {
        const int n = w.n, m = w.m, p = w.p;
        const double sW = h->fs.s1, sV = h->fs.s2, sa = std::sqrt(al);
        cudaStream_t s = h->stream;
        vcomb<double>(o, p, g, 0, 1.0 / sa, nullptr, 0, 0.0, s);
        // a^1/2 T2^-1 Q^T g2 = a^1/2 sV P_n T~_n'^-T P_n Q^T g2
        vcomb<double>(b.w1, n, g + p, 0, 1.0, nullptr, 0, 0.0, s);
        RC(vapply_d<T>(w.Wf, w.ldW, n, m, w.TwW, w.Tw128W, w.TfW, w.ldtW, w.wy, 1, b.w1, s));
        vcomb<double>(b.w2, n, b.w1, 1, 1.0, nullptr, 0, 0.0, s);
        RC(trsv_trap<T>(h, w.Ct, w.ldCt, rT(), n, sV, 1, b.w2, b.dT, s, w.PkC, w.kC));
        vcomb<double>(o + p, n, b.w2, 1, sa * sV, nullptr, 0, 0.0, s);
        if (m > 0) {
            // a^-1/2 b^-1 S^T R^-T g3 = a^-1/2 b^-1 (sW/sV) P_m T~_S' P_m R'^-T g3
            vcomb<double>(b.w1, m, g + p + n, 0, 1.0, nullptr, 0, 0.0, s);
            RC(trsv_d<T>(w.Wf, w.ldW, m, 1, b.w1, h->sc, s, b.dR, w.PkW, w.m));
            vcomb<double>(b.w2, m, b.w1, 1, 1.0, nullptr, 0, 0.0, s);
            RC(trap_tail_gemv<T>(w.Ct, w.ldCt, rT(), n, w.L, sV, 0, b.w2, b.w3, s));
            vcomb<double>(o + p + n, m, b.w3, 1, sW / (sV * sa * be), nullptr, 0, 0.0, s);
        }
        return 0;
    }

    int apply(const double *in, double *out) override
    {
        RC(Mr(in, b.u));
        RC(Fmul(b.u, b.gf));
        return Ml(b.gf, out);
    }
};

// One GMRES-IR correction (GLS): solve M_l F~ M_r t = M_l [a^1/2 f1;
// a^-1/2 f2; a^1/2 b f3], then [a^-1/2 dy; -a^1/2 dz; a^-1/2 b^-1 dx] = M_r t
// and the updates are added to (y, z, x).
template <typename T>
int gls_gmres_correction(mpir_ctx *h, GlsWs<T> &w, BDScratch &b, const double *W, int ldw, const double *V,
                         int ldv, double al, double be, double itol, int imax, double *y, double *z, double *x,
                         int *inner, bool first)
{
    const int n = w.n, m = w.m, p = w.p;
    cudaStream_t s = h->stream;
    const double sa = std::sqrt(al);
    GlsBDOp<T> op(h, w, b, W, ldw, V, ldv, al, be);
    if (first) op.prepare();
    vcomb<double>(b.t, p, w.f1, 0, sa, nullptr, 0, 0.0, s);
    vcomb<double>(b.t + p, n, w.f2, 0, 1.0 / sa, nullptr, 0, 0.0, s);
    vcomb<double>(b.t + p + n, m, w.f3, 0, sa * be, nullptr, 0, 0.0, s);
    RC(op.Ml(b.t, b.rhs));
    int k = 0;
    double rel = 0.0;
    RC(gmres_solve(op, b.rhs, b.t, b.gw, itol, imax, h->hbuf, s, &k, &rel));
    *inner += k;
    RC(op.Mr(b.t, b.u));
    vaxpy<double>(b.u, y, p, sa, 0, s);
    vaxpy<double>(b.u + p, z, n, -1.0 / sa, 0, s);
    vaxpy<double>(b.u + p + n, x, m, sa * be, 0, s);
    return cuda_check(h, "gls_gmres_correction");
}

// Sec. 5.1 (eq. gls-leftpre): the left preconditioner M ~ F~^-1, applied as
// the paper does by the correction solver on the held factors (Alg. 3): F~ u
// = g is the correction system with f = (g1, a g2, g3 / b), and its solution
// (dy, dz, dx) gives u = (dy / a, -dz, dx / (a b)).  M_r = I; every shape.
template <typename T>
struct GlsLeftOp : LinOp {
    GlsBDOp<T> bd;
    GlsLeftOp(mpir_ctx *h_, GlsWs<T> &w_, BDScratch &b_, const double *W_, int ldw_, const double *V_, int ldv_,
              double al_, double be_)
        : bd(h_, w_, b_, W_, ldw_, V_, ldv_, al_, be_) {}

    int Ml(const double *g, double *o)
    {
        mpir_ctx *h = bd.h;
        const int n = bd.w.n, m = bd.w.m, p = bd.w.p;
        const double al = bd.al, be = bd.be;
        BDScratch &b = bd.b;
        cudaStream_t s = h->stream;
        vcomb<double>(b.w1, p, g, 0, 1.0, nullptr, 0, 0.0, s);
        vcomb<double>(b.w2, n, g + p, 0, al, nullptr, 0, 0.0, s);
        vcomb<double>(b.w3, m, g + p + n, 0, 1.0 / be, nullptr, 0, 0.0, s);
        vzero(o, sizeof(double) * (size_t)(p + n + m), s);
        RC(gls_correction_impl<T>(h, b.w1, b.w2, b.w3, 1.0, o, o + p, o + p + n));
        vcomb<double>(o, p, o, 0, 1.0 / al, nullptr, 0, 0.0, s);
        vcomb<double>(o + p, n, o + p, 0, -1.0, nullptr, 0, 0.0, s);
        vcomb<double>(o + p + n, m, o + p + n, 0, 1.0 / (al * be), nullptr, 0, 0.0, s);
        return 0;
    }

    int apply(const double *in, double *out) override
    {
        RC(bd.Fmul(in, bd.b.gf));
        return Ml(bd.b.gf, out);
    }
};

// One GMRES-IR correction with the left preconditioner (GLS): GMRES on
// M F~ t = M [a^1/2 f1; a^-1/2 f2; a^1/2 b f3], then t = [a^-1/2 dy;
// -a^1/2 dz; a^-1/2 b^-1 dx] and the updates are added to (y, z, x).
template <typename T>
int gls_gmres_left_correction(mpir_ctx *h, GlsWs<T> &w, BDScratch &b, const double *W, int ldw, const double *V,
                              int ldv, double al, double be, double itol, int imax, double *y, double *z, double *x,
                              int *inner)
{
    const int n = w.n, m = w.m, p = w.p;
    cudaStream_t s = h->stream;
    const double sa = std::sqrt(al);
    GlsLeftOp<T> op(h, w, b, W, ldw, V, ldv, al, be);
    vcomb<double>(b.t, p, w.f1, 0, sa, nullptr, 0, 0.0, s);
    vcomb<double>(b.t + p, n, w.f2, 0, 1.0 / sa, nullptr, 0, 0.0, s);
    vcomb<double>(b.t + p + n, m, w.f3, 0, sa * be, nullptr, 0, 0.0, s);
    RC(op.Ml(b.t, b.rhs));
    int k = 0;
    double rel = 0.0;
    RC(gmres_solve(op, b.rhs, b.t, b.gw, itol, imax, h->hbuf, s, &k, &rel));
    *inner += k;
    vaxpy<double>(b.t, y, p, sa, 0, s);
    vaxpy<double>(b.t + p, z, n, -1.0 / sa, 0, s);
    vaxpy<double>(b.t + p + n, x, m, sa * be, 0, s);
    return cuda_check(h, "gls_gmres_left_correction");
}

double inner_tol_default(const mpir_opts &o, int fact)
{
    if (o.inner_tol > 0) return o.inner_tol;
    return (fact == MPIR_BF16 || fact == MPIR_TF32) ? 1e-4 : 1e-8;
}

// alpha of F~ (Sec. 5; floored so that a consistent problem keeps it > 0)
double bd_alpha(const mpir_opts &o, double lead, double fro, double other)
{
    if (o.alpha > 0) return o.alpha;
    const double sqrt_u = std::ldexp(1.0, -26) * std::sqrt(0.5);   // sqrt(2^-53)
    const double a = std::max(lead, sqrt_u * fro * other);
    return (a > 0 && std::isfinite(a)) ? a : 1.0;
}

template <typename T>
int gls_solve_once(mpir_ctx *h, int n, int m, int p, const double *W, int ldw, const double *V, int ldv,
                   const double *d, double *x, double *y, double *z_out, const mpir_opts &o, int fact,
                   mpir_info *info, bool factored = false)
{
    cudaStream_t s = h->stream;
    const bool left = o.refine == MPIR_GMRES_LEFT;
    const bool gm = o.refine == MPIR_GMRES || left;
    size_t main_bytes = 0;
    gls_layout<T>(nullptr, n, m, p, &main_bytes);
    const int NG = p + n + m, mx = std::max(std::max(m, n), std::max(p, 1));
    if (gm) {
        if (o.restart > GMRES_MAX_RESTART) return set_err(h, MPIR_UNSUPPORTED, "GMRES restart above 64");
        RC(ensure_ws(h, main_bytes + bd_bytes(NG, o.restart, mx)));
    }
    if (!factored) {              // else factored (and timed) by the caller
        cudaEventRecord(h->ev[0], s);
        RC(gls_factor_impl<T>(h, n, m, p, W, ldw, V, ldv, fact));
        cudaEventRecord(h->ev[1], s);
    }
    GlsWs<T> w = gls_layout<T>(h->ws, n, m, p, nullptr);
    BDScratch bs{};
    if (gm) bs = bd_layout((char *)h->ws + main_bytes, NG, o.restart, mx);
    double *z = z_out ? z_out : w.z;
    RC(gls_initial_impl<T>(h, d, x, y));
    int st = MPIR_OK;
    int it = 0, inner = 0;
    double ratio[3] = {0, 0, 0};
    double al = 1.0;
    float t_gm = 0;
    bool looped = false;
    if (o.refine != MPIR_DIRECT) RC(gls_multipliers_impl<T>(h, y, z));
    const bool dd = o.resid_dd != 0;
    if (dd) RC(ensure_rws(h, sizeof(double) * (2 * (size_t)(2 * n + m + p) + m + p + 8)));
    if (o.refine == MPIR_CLASSICAL && ir_graph_usable(h) && !dd) {
        unsigned long long key = ir_mix(ir_mix(ir_mix(0, 2), sizeof(T)), (unsigned long long)n);
        for (unsigned long long v_ : {(unsigned long long)m, (unsigned long long)p, (unsigned long long)ldw,
                                      (unsigned long long)ldv, (unsigned long long)(uintptr_t)W,
                                      (unsigned long long)(uintptr_t)V, (unsigned long long)(uintptr_t)d,
                                      (unsigned long long)(uintptr_t)x, (unsigned long long)(uintptr_t)y,
                                      (unsigned long long)(uintptr_t)z, (unsigned long long)(uintptr_t)h->ws,
                                      (unsigned long long)o.maxit,
                                      (unsigned long long)std::llround(-std::log2(o.tol) * 4096.0)})
            key = ir_mix(key, v_);
        ir_stage_scalars(h, w.ird);
        auto pre = [&](cudaGraphConditionalHandle hc) {
            k_ir_reset<<<1, 32, 0, h->stream>>>(w.ird);
            absmax_sumsq(d, std::max(n, 1), n, 1, w.part, w.ird + IRD_N1, h->stream);
            gls_residual_dev<T>(h, w, W, ldw, V, ldv, d, x, y, z);
            k_ir_control<<<1, 32, 0, h->stream>>>(w.norms2, w.ird, 1, o.tol, o.maxit, hc, 1);
            return cudaGetLastError() == cudaSuccess ? 0 : 1;
        };
        auto body = [&](cudaGraphConditionalHandle hc) {
            int rc = gls_correction_impl<T>(h, w.f1, w.f2, w.f3, 1.0, y, z, x, w.ird + IRD_C);
            gls_residual_dev<T>(h, w, W, ldw, V, ldv, d, x, y, z);
            k_ir_control<<<1, 32, 0, h->stream>>>(w.norms2, w.ird, 1, o.tol, o.maxit, hc, 1);
            return rc == 0 && cudaGetLastError() == cudaSuccess ? 0 : 1;
        };
        const int gr = ir_graph_run(h, w.ird, key, pre, body, &it, &st, ratio);
        if (gr < 0 || gr == MPIR_CUDA_ERROR) return gr;
        if (gr == 0) looped = true;
        else h->irg_off = true;
    }
    if (o.refine != MPIR_DIRECT && !looped) {
        cudaEventRecord(h->ev[2], s);
        StopState ss;
        st = MPIR_NOT_CONVERGED;
        const double fW = h->fs.fro1, fV = h->fs.fro2;
        const double nd = dnorm_host(h, d, n, w.part);
        float t_res = 0;
        double *dds = dd ? (double *)h->rws : nullptr;
        double *xyprev = dd ? dds + 2 * (size_t)(2 * n + m + p) : nullptr, *dxn = dd ? xyprev + m + p : nullptr;
        FwdState fw;
        bool bw = false;
        // after a correction (u_r < u variant): ||[dx; dy]||
        auto post = [&]() -> int {
            if (!dd) return 0;
            if (m > 0) diff_norm2(x, xyprev, m, dxn, 0, s);
            if (p > 0) diff_norm2(y, xyprev + m, p, dxn, m > 0, s);
            RC(read_back(h, dxn, 1));
            fw.push(std::sqrt(h->hbuf[0]));
            return 0;
        };
        for (it = 0; it < o.maxit; it++) {
            cudaEventRecord(h->ev[3], s);
            if (dd) {
                if (gls_resid_dd(n, m, p, W, ldw, V, ldv, d, x, y, z, dds, w.f1, w.f2, w.f3, w.norms2, s) !=
                    cudaSuccess)
                    return cuda_check(h, "gls double-double residual");
            } else {
                gls_residual_dev<T>(h, w, W, ldw, V, ldv, d, x, y, z);
            }
            cudaEventRecord(h->ev[4], s);
            RC(read_back(h, w.norms2, 6));
            t_res += ev_ms(h->ev[3], h->ev[4]);
            double nr[6];
            for (int i = 0; i < 6; i++) nr[i] = std::sqrt(h->hbuf[i]);
            // nr: f1 f2 f3 x y z
            double den[3] = {nr[4] + fV * nr[5], nd + fW * nr[3] + fV * nr[4], fW * nr[5]};
            for (int i = 0; i < 3; i++) if (!std::isfinite(nr[i])) { st = MPIR_NONFINITE; break; }
            if (st == MPIR_NONFINITE) break;
            bw = stop_test(nr, den, o.tol, ratio);
            if (bw && (!dd || fw.done(std::sqrt(nr[3] * nr[3] + nr[4] * nr[4])))) { st = MPIR_OK; break; }
            if (!bw) {
                const double eta = std::max(ratio[0], std::max(ratio[1], ratio[2]));
                if (eta < 0.5 * ss.best) { ss.best = eta; ss.since_best = 0; }
                else if (++ss.since_best >= 3) { st = ss.best <= 1e-14 ? MPIR_OK : MPIR_NOT_CONVERGED; break; }
            }
            if (dd) {
                if (m > 0) cudaMemcpyAsync(xyprev, x, sizeof(double) * m, cudaMemcpyDeviceToDevice, s);
                if (p > 0) cudaMemcpyAsync(xyprev + m, y, sizeof(double) * p, cudaMemcpyDeviceToDevice, s);
            }
            // normalize the right-hand side of the scaled correction system
            // (f1, sV f2, sW/sV f3), not the raw blocks
            if (gm) {
                // Sec. 5.3: correction from GMRES on the preconditioned F~
                if (it == 0) al = bd_alpha(o, nr[4], fV, nr[5]);
                cudaEventRecord(h->ev[5], s);
                if (left)       // Sec. 5.1: M = F~^-1 applied by Alg. 3
                    RC(gls_gmres_left_correction<T>(h, w, bs, W, ldw, V, ldv, al, o.beta,
                                                    inner_tol_default(o, fact), o.inner_maxit, y, z, x, &inner));
                else
                    RC(gls_gmres_correction<T>(h, w, bs, W, ldw, V, ldv, al, o.beta, inner_tol_default(o, fact),
                                               o.inner_maxit, y, z, x, &inner, it == 0));
                cudaEventRecord(h->ev[6], s);
                cudaEventSynchronize(h->ev[6]);
                t_gm += ev_ms(h->ev[5], h->ev[6]);
                RC(post());
                continue;
            }
            const double sW = h->fs.s1, sV = h->fs.s2;
            const double fmax = std::max(nr[0], std::max(nr[1] * sV, nr[2] * sW / sV));
            const double gamma = pow2_norm(fmax);
            RC(gls_correction_impl<T>(h, w.f1, w.f2, w.f3, gamma, y, z, x));
            RC(post());
        }
        if (st == MPIR_NOT_CONVERGED && bw) st = MPIR_OK;     // maxit with the backward test met
        if (info) { info->time_ms[2] = t_res; info->time_ms[4] = t_gm; info->inner_iters = inner; }
    }
    RC(check_dev_flags(h));
    cudaEventRecord(h->ev[7], s);
    cudaEventSynchronize(h->ev[7]);
    if (info) {
        info->status = st;
        info->iters = it;
        info->fact_used = fact;
        info->refine_used = o.refine;
        for (int i = 0; i < 3; i++) info->stop_ratio[i] = ratio[i];
        info->time_ms[0] = ev_ms(h->ev[0], h->ev[1]);
        info->time_ms[5] = ev_ms(h->ev[0], h->ev[7]);
    }
    return st;
}

// ================================================================= LSE ==

template <typename T>
int lse_factor_impl(mpir_ctx *h, int m, int n, int p, const double *A, int lda, const double *B, int ldb,
                    int fact)
{
    size_t bytes = 0;
    lse_layout<T>(nullptr, m, n, p, &bytes);
    RC(ensure_ws(h, bytes));
    LseWs<T> w = lse_layout<T>(h->ws, m, n, p, nullptr);
    cudaStream_t s = h->stream;
    join_side(h, s);
    clear_dev_flags(h);
    absmax_sumsq(A, lda, m, n, w.part, w.scal + 0, s);
    absmax_sumsq(B, ldb, p, n, w.part, w.scal + 2, s);
    RC(read_back(h, w.scal, 4));
    if (!std::isfinite(h->hbuf[1]) || !std::isfinite(h->hbuf[3]))
        return set_err(h, MPIR_NONFINITE, "non-finite entry in A or B");
    const double sA = pow2_scale(h->hbuf[0]), sB = pow2_scale(h->hbuf[2]);
    h->fs.kind = Kind::LSE;
    h->fs.fact = fact;
    h->fs.m = m; h->fs.n = n; h->fs.p = p;
    h->fs.s1 = sA; h->fs.s2 = sB;
    h->fs.fro1 = std::sqrt(h->hbuf[1]);
    h->fs.fro2 = std::sqrt(h->hbuf[3]);
    const GemmPrec gp = gemm_prec(fact);
    // BF16 / TF32 factors: power-of-two column scaling D of [sA A; sB B]
    // (Sec. 6.1 scaling before down-conversion), so every column enters the
    // low-precision factorization with its largest entry in [0.5, 1); the
    // factors are then those of (sA A D, sB B D) and x = D y
    h->fs.colscale = sizeof(T) == 4 && (fact == MPIR_BF16 || fact == MPIR_TF32);
    const double *Dc = h->fs.colscale ? w.D : nullptr;
    if (Dc) colscale_pow2(A, lda, m, B, ldb, p, n, sA, sB, w.D, s);
    // RQ of B as QR of B~ = P_n B^T P_p (Lemma 4.5, first factorization),
    // with X = Q~^T P_n A^T = P_n (A Q^T)^T formed by the same trailing
    // updates: [B~ X] factored through its first p columns
    mconvert<double, T>(B, ldb, w.Bt, w.ldBt, n, p, 1, 1, 1, sB, s, Dc, 1);
    mconvert<double, T>(A, lda, w.X, w.ldX, n, m, 1, 1, 0, sA, s, Dc, 1);
    // the low-precision classes (BF16, TF32) run the dominant factorization
    // (QR of A Q^T) at their precision; the RQ of B and the application of
    // its Q to A stay FP32-class, so that kappa(B) multiplies an FP32-sized
    // error rather than a bfloat16 one
    const GemmPrec gp1 = gp == GemmPrec::FP64 ? gp : GemmPrec::FP32;
    RC(geqrf<T>(w.Bt, w.ldBt, n, p + m, w.tauB, w.TwB, w.Tw128B, gp1, w.gws, h->sc.err, s,
                tfjob(h, w.TfB, w.ldtB, w.gws2), p));
    // A Q^T = X^T P_n, then its QR  (A Q^T = Z T)
    mconvert<T, T>(w.X, w.ldX, w.At, w.ldAt, m, n, 1, 0, 1, 1.0, s);
    RC(geqrf<T>(w.At, w.ldAt, m, n, w.tauA, w.TwA, w.Tw128A, gp, w.gws, h->sc.err, s, tfjob(h, w.TfA, w.ldtA, w.gws2)));
    // inverses of the 32 x 32 diagonal blocks of R~ and T for the solves
    inv_diag<T>(w.Bt, w.ldBt, p, w.DinvB, h->sc.status, s);
    inv_diag<T>(w.At, w.ldAt, w.q, w.DinvA, h->sc.status, s);   // T11, the block that is solved
    if constexpr (sizeof(T) == 4) {
        // block columns of R~ and of the whole T (the preconditioners solve
        // with its leading min(m, n) block) in the solves' read order
        RC(t64_pack(w.Bt, w.ldBt, p, w.PkB, s));
        RC(t64_pack(w.At, w.ldAt, w.kA, w.PkA, s));
    }
    if (sizeof(T) == 4) join_side(h, s);
    return cuda_check(h, "lse_factor");
}

// Null-space method (Sec. 2.1) with the scaled factors: R y2 = sB d,
// T11 y1 = c1 - T12 y2 (c = Z^T (sA b)), x = Q^T y.
template <typename T>
int lse_initial_impl(mpir_ctx *h, const double *b, const double *d, double *x)
{
    const FactorState &fs = h->fs;
    LseWs<T> w = lse_layout<T>(h->ws, fs.m, fs.n, fs.p, nullptr);
    const int m = w.m, n = w.n, p = w.p, q = w.q;
    cudaStream_t s = h->stream;
    // common power-of-two normalization g of (sA b, sB d); x = result / g
    double *g = w.scal + 8;
    pow2_normalizer(b, m, fs.s1, d, p, fs.s2, g, s);
    vcopy<double, T>(b, w.tw, m, fs.s1, 0, s, g);
    RC(vapply<T>(w.At, w.ldAt, m, w.kA, w.TwA, w.Tw128A, w.TfA, w.ldtA, w.wy, 1, w.tw, h->sc, s));
    // R y2 = sB d  <=>  R~^T y~2 = P_p (sB d)
    vcopy<double, T>(d, w.tb, p, fs.s2, 1, s, g);
    RC(tsolve<T>(w.Bt, w.ldBt, p, 1, w.tb, h->sc, s, w.DinvB, w.PkB, w.p));
    // ty = [y1; y2], y2 = P_p y~2
    vcomb<T>(w.ty + q, p, w.tb, 1, T(1), nullptr, 0, T(0), s);
    vcomb<T>(w.ty, q, w.tw, 0, T(1), nullptr, 0, T(0), s);
    RC(gemv<T>(w.At + idx2(0, q, w.ldAt), w.ldAt, q, p, 0, T(-1), w.ty + q, T(1), w.ty, 0, 0, s));
    RC(tsolve<T>(w.At, w.ldAt, q, 0, w.ty, h->sc, s, w.DinvA, w.PkA, w.kA));
    // x = Q^T y = P_n Q~ P_n y
    vcomb<T>(w.tt, n, w.ty, 1, T(1), nullptr, 0, T(0), s);
    RC(vapply<T>(w.Bt, w.ldBt, n, p, w.TwB, w.Tw128B, w.TfB, w.ldtB, w.wy, 0, w.tt, h->sc, s));
    vcopy<T, double>(w.tt, x, n, 1.0, 1, s, g + 1);
    if (fs.colscale) vdiag<double>(x, w.D, n, 0, s);          // x = D y
    return cuda_check(h, "lse_initial");
}

// r0 = b - A x (FP64), R^T v0 = (Q A^T r0)(n-p+1:n) (Alg. 2 steps 3-4).
template <typename T>
int lse_multipliers_impl(mpir_ctx *h, const double *A, int lda, const double *b, const double *x, double *r,
                         double *v)
{
    const FactorState &fs = h->fs;
    LseWs<T> w = lse_layout<T>(h->ws, fs.m, fs.n, fs.p, nullptr);
    const int m = w.m, n = w.n, p = w.p;
    cudaStream_t s = h->stream;
    cudaMemcpyAsync(r, b, sizeof(double) * m, cudaMemcpyDeviceToDevice, s);
    RC(gemv<double>(A, lda, m, n, 0, -1.0, x, 1.0, r, 0, 0, s));
    if (p == 0) return cuda_check(h, "lse_multipliers");
    RC(gemv<double>(A, lda, m, n, 1, 1.0, r, 0.0, w.f3, 0, 0, s));
    if (fs.colscale) vdiag<double>(w.f3, w.D, n, 0, s);       // (A D)^T r
    // u~ = Q~^T P_n (g sA A^T r), g a power-of-two normalizer
    double *g = w.scal + 8;
    pow2_normalizer(w.f3, n, fs.s1, nullptr, 0, 0.0, g, s);
    vcopy<double, T>(w.f3, w.tu, n, fs.s1, 1, s, g);
    RC(vapply<T>(w.Bt, w.ldBt, n, p, w.TwB, w.Tw128B, w.TfB, w.ldtB, w.wy, 1, w.tu, h->sc, s));
    // R~ (P_p v') = u~[0:p]
    RC(tsolve<T>(w.Bt, w.ldBt, p, 0, w.tu, h->sc, s, w.DinvB, w.PkB, w.p));
    vcopy<T, double>(w.tu, v, p, fs.s2 / fs.s1, 1, s, g + 1);
    return cuda_check(h, "lse_multipliers");
}

// Alg. 1 in reversed coordinates; results are ADDED to (dr, dv, dx).
template <typename T>
int lse_correction_impl(mpir_ctx *h, const double *f1, const double *f2, const double *f3, double gamma,
                        double *dr, double *dv, double *dx, const double *dsc = nullptr)
{
    const FactorState &fs = h->fs;
    LseWs<T> w = lse_layout<T>(h->ws, fs.m, fs.n, fs.p, nullptr);
    const int m = w.m, n = w.n, p = w.p, q = w.q;
    const double sA = fs.s1, sB = fs.s2;
    // scales of the right-hand side blocks and of the outputs: host values,
    // or (dsc != NULL) device scalars c1, c2, c3, i1, i2, i3 left by the
    // device-side loop's control kernel
    const double c1 = dsc ? 1.0 : gamma, c2 = dsc ? 1.0 : gamma * sB / sA, c3 = dsc ? 1.0 : gamma * sA;
    const double i1 = dsc ? 1.0 : 1.0 / gamma, i2 = dsc ? 1.0 : sB / sA / gamma, i3 = dsc ? 1.0 : sA / gamma;
    const double *d1 = dsc, *d2 = dsc ? dsc + 1 : nullptr, *d3 = dsc ? dsc + 2 : nullptr;
    const double *e1 = dsc ? dsc + 3 : nullptr, *e2 = dsc ? dsc + 4 : nullptr, *e3 = dsc ? dsc + 5 : nullptr;
    cudaStream_t s = h->stream;
    // step 1: u~ = Q~^T P_n f3' ;  u1 = P_q u~[p:n], u2 = P_p u~[0:p]
    // (with column scaling the third block of the scaled system is D f3)
    vcopy<double, T>(f3, w.tu, n, c3, 1, s, d3);
    if (fs.colscale) vdiag<T>(w.tu, w.D, n, 1, s);
    RC(vapply<T>(w.Bt, w.ldBt, n, p, w.TwB, w.Tw128B, w.TfB, w.ldtB, w.wy, 1, w.tu, h->sc, s));
    // step 2: w = Z^T f1'
    vcopy<double, T>(f1, w.tw, m, c1, 0, s, d1);
    RC(vapply<T>(w.At, w.ldAt, m, w.kA, w.TwA, w.Tw128A, w.TfA, w.ldtA, w.wy, 1, w.tw, h->sc, s));
    // step 3: R y2 = f2'  <=>  R~^T y~2 = P_p f2'
    if (p > 0) {
        vcopy<double, T>(f2, w.tb, p, c2, 1, s, d2);
        RC(tsolve<T>(w.Bt, w.ldBt, p, 1, w.tb, h->sc, s, w.DinvB, w.PkB, w.p));
        vcomb<T>(w.ty + q, p, w.tb, 1, T(1), nullptr, 0, T(0), s);
    }
    // step 4: T11^T q1 = u1
    if (q > 0) {
        vcomb<T>(w.tq, q, w.tu + p, 1, T(1), nullptr, 0, T(0), s);
        RC(tsolve<T>(w.At, w.ldAt, q, 1, w.tq, h->sc, s, w.DinvA, w.PkA, w.kA));
        // step 5: T11 y1 = w1 - q1 - T12 y2
        vcomb<T>(w.ty, q, w.tw, 0, T(1), w.tq, 0, T(-1), s);
        if (p > 0) RC(gemv<T>(w.At + idx2(0, q, w.ldAt), w.ldAt, q, p, 0, T(-1), w.ty + q, T(1), w.ty, 0, 0, s));
        RC(tsolve<T>(w.At, w.ldAt, q, 0, w.ty, h->sc, s, w.DinvA, w.PkA, w.kA));
    }
    // step 6: q2 = w2 - T22 y2
    if (m - q > 0) {
        vcomb<T>(w.tq + q, m - q, w.tw + q, 0, T(1), nullptr, 0, T(0), s);
        if (p > 0) RC(gemv<T>(w.At + idx2(q, q, w.ldAt), w.ldAt, m - q, p, 0, T(-1), w.ty + q, T(1), w.tq + q, 1, 0, s));
    }
    // step 8: R^T dv = T12^T q1 + T22^T q2 - u2  <=>  R~ (P_p dv) = P_p(T12^T q1 + T22^T q2) - u~[0:p]
    if (p > 0) {
        vzero(w.tt, sizeof(T) * p, s);
        if (q > 0) RC(gemv<T>(w.At + idx2(0, q, w.ldAt), w.ldAt, q, p, 1, T(1), w.tq, T(0), w.tt, 0, 0, s));
        if (m - q > 0) RC(gemv<T>(w.At + idx2(q, q, w.ldAt), w.ldAt, m - q, p, 1, T(1), w.tq + q, T(1), w.tt, 1, 0, s));
        vcomb<T>(w.tb, p, w.tt, 1, T(1), w.tu, 0, T(-1), s);
        RC(tsolve<T>(w.Bt, w.ldBt, p, 0, w.tb, h->sc, s, w.DinvB, w.PkB, w.p));
        vaxpy<T>(w.tb, dv, p, i2, 1, s, e2);
    }
    // step 7: dr = Z q ; dx = Q^T y = P_n Q~ P_n y
    RC(vapply<T>(w.At, w.ldAt, m, w.kA, w.TwA, w.Tw128A, w.TfA, w.ldtA, w.wy, 0, w.tq, h->sc, s));
    vaxpy<T>(w.tq, dr, m, i1, 0, s, e1);
    vcomb<T>(w.tt2, n, w.ty, 1, T(1), nullptr, 0, T(0), s);
    RC(vapply<T>(w.Bt, w.ldBt, n, p, w.TwB, w.Tw128B, w.TfB, w.ldtB, w.wy, 0, w.tt2, h->sc, s));
    if (fs.colscale) vdiag<T>(w.tt2, w.D, n, 1, s);           // dx = D dy
    vaxpy<T>(w.tt2, dx, n, i3, 1, s, e3);
    return cuda_check(h, "lse_correction");
}

template <typename T>
void lse_residual_dev(mpir_ctx *h, LseWs<T> &w, const double *A, int lda, const double *B, int ldb,
                      const double *b, const double *d, const double *x, const double *r, const double *v)
{
    cudaStream_t s = h->stream;
    const int m = w.m, n = w.n, p = w.p;
    dual_gemv(A, lda, m, n, x, r, w.pAx, w.pAtr, s);
    if (p > 0) dual_gemv(B, ldb, p, n, x, v, w.pBx, w.pBtv, s);
    lse_resid_finalize(m, n, p, b, d, x, r, v, w.pAx, w.pa.ncb, w.pAtr, w.pa.nrb, w.pBx, w.pb.ncb, w.pBtv,
                       p > 0 ? w.pb.nrb : 0, w.f1, w.f2, w.f3, w.normpart, w.norms2, s);
}

double dnorm_host(mpir_ctx *h, const double *dvec, int n, double *scratch)
{
    // ||vec||_2 via absmax_sumsq on an n x 1 matrix
    absmax_sumsq(dvec, std::max(n, 1), n, 1, scratch, scratch + 4096 - 4, h->stream);
    read_back(h, scratch + 4096 - 4, 2);
    return std::sqrt(h->hbuf[1]);
}


// LSE (Sec. 5.2):  F~ = [a I, 0, A; 0, 0, b B; A^T, b B^T, 0] on
// u = [u1 (m); u2 (p); u3 (n)];  T1 = T(1:n, 1:n), S = T1(q+1:n, q+1:n)
// (n > m, eq. lse-bdpre-nlarge: T is m x n and T1 = [T; 0, I_{n-m}]),
//   M_l = diag(a^-1/2 I, a^-1/2 b^-1 S R^-1, a^1/2 T1^-T Q),
//   M_r = diag(a^-1/2 I, a^-1/2 b^-1 R^-T S^T, a^1/2 Q^T T1^-1).
// Reversed coordinates: R = P_p R~^T P_p, Q = P_n Q~^T P_n; T is held as is.
template <typename T>
struct LseBDOp : LinOp {
    mpir_ctx *h;
    LseWs<T> &w;
    BDScratch &b;
    const double *A, *B;
    int lda, ldb;
    double al, be;
    LseBDOp(mpir_ctx *h_, LseWs<T> &w_, BDScratch &b_, const double *A_, int lda_, const double *B_, int ldb_,
            double al_, double be_)
        : h(h_), w(w_), b(b_), A(A_), B(B_), lda(lda_), ldb(ldb_), al(al_), be(be_) {}

    // rows of T held (n > m: T1 = [T; 0, I], eq. lse-bdpre-nlarge)
    int rT() const { return std::min(w.m, w.n); }

    // FP64 inverses of the diagonal blocks of T1 and R~
    void prepare()
    {
        inv_diag_d<T>(w.At, w.ldAt, rT(), b.dT, h->sc.status, h->stream);
        inv_diag_d<T>(w.Bt, w.ldBt, w.p, b.dR, h->sc.status, h->stream);
    }

    int Mr(const double *t, double *u)
    {
        const int m = w.m, n = w.n, p = w.p;
        const double sA = h->fs.s1, sB = h->fs.s2, sa = std::sqrt(al);
        cudaStream_t s = h->stream;
        vcomb<double>(u, m, t, 0, 1.0 / sa, nullptr, 0, 0.0, s);
        if (p > 0) {
            // a^-1/2 b^-1 R^-T S^T t2 = a^-1/2 b^-1 (sB/sA) P_p R~'^-1 P_p S'^T t2
            RC(trap_tail_gemv<T>(w.At, w.ldAt, rT(), n, w.q, sA, 1, t + m, b.w1, s));
            vcomb<double>(b.w2, p, b.w1, 1, 1.0, nullptr, 0, 0.0, s);
            RC(trsv_d<T>(w.Bt, w.ldBt, p, 0, b.w2, h->sc, s, b.dR, w.PkB, w.p));
            vcomb<double>(u + m, p, b.w2, 1, sB / (sA * sa * be), nullptr, 0, 0.0, s);
        }
        // a^1/2 Q^T T1^-1 t3 = a^1/2 sA P_n Q~ P_n T1'^-1 t3
        vcomb<double>(b.w1, n, t + m + p, 0, 1.0, nullptr, 0, 0.0, s);
        RC(trsv_trap<T>(h, w.At, w.ldAt, rT(), n, sA, 0, b.w1, b.dT, s, w.PkA, w.kA));
        vcomb<double>(b.w2, n, b.w1, 1, 1.0, nullptr, 0, 0.0, s);
        RC(vapply_d<T>(w.Bt, w.ldBt, n, p, w.TwB, w.Tw128B, w.TfB, w.ldtB, w.wy, 0, b.w2, s));
        vcomb<double>(u + m + p, n, b.w2, 1, sa * sA, nullptr, 0, 0.0, s);
        if (h->fs.colscale) vdiag<double>(u + m + p, w.D, n, 0, s);     // D (Q'^T T1'^-1) t3
        return 0;
    }

    int Fmul(const double *u, double *g)
    {
        const int m = w.m, n = w.n, p = w.p;
        cudaStream_t s = h->stream;
        dual_gemv(A, lda, m, n, u + m + p, u, w.pAx, w.pAtr, s);
        if (p > 0) dual_gemv(B, ldb, p, n, u + m + p, u + m, w.pBx, w.pBtv, s);
        combine_parts(g, m, al, u, 1.0, w.pAx, w.pa.ncb, m, 0.0, nullptr, 0, 0, s);
        if (p > 0) combine_parts(g + m, p, 0.0, nullptr, be, w.pBx, w.pb.ncb, p, 0.0, nullptr, 0, 0, s);
        combine_parts(g + m + p, n, 0.0, nullptr, 1.0, w.pAtr, w.pa.nrb, n, be, p > 0 ? w.pBtv : nullptr,
                      w.pb.nrb, n, s);
        return 0;
    }

    int Ml(const double *g, double *o)
    {
        const int m = w.m, n = w.n, p = w.p;
        const double sA = h->fs.s1, sB = h->fs.s2, sa = std::sqrt(al);
        cudaStream_t s = h->stream;
        vcomb<double>(o, m, g, 0, 1.0 / sa, nullptr, 0, 0.0, s);
        if (p > 0) {
            // a^-1/2 b^-1 S R^-1 g2 = a^-1/2 b^-1 (sB/sA) S' P_p R~'^-T P_p g2
            vcomb<double>(b.w1, p, g + m, 1, 1.0, nullptr, 0, 0.0, s);
            RC(trsv_d<T>(w.Bt, w.ldBt, p, 1, b.w1, h->sc, s, b.dR, w.PkB, w.p));
            vcomb<double>(b.w2, p, b.w1, 1, 1.0, nullptr, 0, 0.0, s);
            RC(trap_tail_gemv<T>(w.At, w.ldAt, rT(), n, w.q, sA, 0, b.w2, b.w3, s));
            vcomb<double>(o + m, p, b.w3, 0, sB / (sA * sa * be), nullptr, 0, 0.0, s);
        }
        // a^1/2 T1^-T Q g3 = a^1/2 sA T1'^-T P_n Q~^T P_n g3  (g3 -> D g3 with column scaling)
        vcomb<double>(b.w1, n, g + m + p, 1, 1.0, nullptr, 0, 0.0, s);
        if (h->fs.colscale) vdiag<double>(b.w1, w.D, n, 1, s);
        RC(vapply_d<T>(w.Bt, w.ldBt, n, p, w.TwB, w.Tw128B, w.TfB, w.ldtB, w.wy, 1, b.w1, s));
        vcomb<double>(b.w2, n, b.w1, 1, 1.0, nullptr, 0, 0.0, s);
        RC(trsv_trap<T>(h, w.At, w.ldAt, rT(), n, sA, 1, b.w2, b.dT, s, w.PkA, w.kA));
        vcomb<double>(o + m + p, n, b.w2, 0, sa * sA, nullptr, 0, 0.0, s);
        return 0;
    }

    int apply(const double *in, double *out) override
    {
        RC(Mr(in, b.u));
        RC(Fmul(b.u, b.gf));
        return Ml(b.gf, out);
    }
};

// One GMRES-IR correction (LSE): right-hand side [a^1/2 f1; a^1/2 b f2;
// a^-1/2 f3], solution [a^-1/2 dr; -a^-1/2 b^-1 dv; a^1/2 dx] = M_r t.
template <typename T>
int lse_gmres_correction(mpir_ctx *h, LseWs<T> &w, BDScratch &b, const double *A, int lda, const double *B,
                         int ldb, double al, double be, double itol, int imax, double *r, double *v, double *x,
                         int *inner, bool first)
{
    const int m = w.m, n = w.n, p = w.p;
    cudaStream_t s = h->stream;
    const double sa = std::sqrt(al);
    LseBDOp<T> op(h, w, b, A, lda, B, ldb, al, be);
    if (first) op.prepare();
    vcomb<double>(b.t, m, w.f1, 0, sa, nullptr, 0, 0.0, s);
    vcomb<double>(b.t + m, p, w.f2, 0, sa * be, nullptr, 0, 0.0, s);
    vcomb<double>(b.t + m + p, n, w.f3, 0, 1.0 / sa, nullptr, 0, 0.0, s);
    RC(op.Ml(b.t, b.rhs));
    int k = 0;
    double rel = 0.0;
    RC(gmres_solve(op, b.rhs, b.t, b.gw, itol, imax, h->hbuf, s, &k, &rel));
    *inner += k;
    RC(op.Mr(b.t, b.u));
    vaxpy<double>(b.u, r, m, sa, 0, s);
    vaxpy<double>(b.u + m, v, p, -sa * be, 0, s);
    vaxpy<double>(b.u + m + p, x, n, 1.0 / sa, 0, s);
    return cuda_check(h, "lse_gmres_correction");
}


// Sec. 5.1 (eq. lse-leftpre): M ~ F~^-1 applied by Alg. 1 on the held
// factors: F~ u = g is the correction system with f = (g1, g2 / b, a g3), and
// its solution (dr, dv, dx) gives u = (dr / a, -dv / (a b), dx).  M_r = I;
// every shape.
template <typename T>
struct LseLeftOp : LinOp {
    LseBDOp<T> bd;
    LseLeftOp(mpir_ctx *h_, LseWs<T> &w_, BDScratch &b_, const double *A_, int lda_, const double *B_, int ldb_,
              double al_, double be_)
        : bd(h_, w_, b_, A_, lda_, B_, ldb_, al_, be_) {}

    int Ml(const double *g, double *o)
    {
        mpir_ctx *h = bd.h;
        const int m = bd.w.m, n = bd.w.n, p = bd.w.p;
        const double al = bd.al, be = bd.be;
        BDScratch &b = bd.b;
        cudaStream_t s = h->stream;
        vcomb<double>(b.w1, m, g, 0, 1.0, nullptr, 0, 0.0, s);
        if (p > 0) vcomb<double>(b.w2, p, g + m, 0, 1.0 / be, nullptr, 0, 0.0, s);
        vcomb<double>(b.w3, n, g + m + p, 0, al, nullptr, 0, 0.0, s);
        vzero(o, sizeof(double) * (size_t)(m + p + n), s);
        RC(lse_correction_impl<T>(h, b.w1, b.w2, b.w3, 1.0, o, o + m, o + m + p));
        vcomb<double>(o, m, o, 0, 1.0 / al, nullptr, 0, 0.0, s);
        if (p > 0) vcomb<double>(o + m, p, o + m, 0, -1.0 / (al * be), nullptr, 0, 0.0, s);
        return 0;
    }

    int apply(const double *in, double *out) override
    {
        RC(bd.Fmul(in, bd.b.gf));
        return Ml(bd.b.gf, out);
    }
};

template <typename T>
int lse_gmres_left_correction(mpir_ctx *h, LseWs<T> &w, BDScratch &b, const double *A, int lda, const double *B,
                              int ldb, double al, double be, double itol, int imax, double *r, double *v, double *x,
                              int *inner)
{
    const int m = w.m, n = w.n, p = w.p;
    cudaStream_t s = h->stream;
    const double sa = std::sqrt(al);
    LseLeftOp<T> op(h, w, b, A, lda, B, ldb, al, be);
    vcomb<double>(b.t, m, w.f1, 0, sa, nullptr, 0, 0.0, s);
    vcomb<double>(b.t + m, p, w.f2, 0, sa * be, nullptr, 0, 0.0, s);
    vcomb<double>(b.t + m + p, n, w.f3, 0, 1.0 / sa, nullptr, 0, 0.0, s);
    RC(op.Ml(b.t, b.rhs));
    int k = 0;
    double rel = 0.0;
    RC(gmres_solve(op, b.rhs, b.t, b.gw, itol, imax, h->hbuf, s, &k, &rel));
    *inner += k;
    vaxpy<double>(b.t, r, m, sa, 0, s);
    vaxpy<double>(b.t + m, v, p, -sa * be, 0, s);
    vaxpy<double>(b.t + m + p, x, n, 1.0 / sa, 0, s);
    return cuda_check(h, "lse_gmres_left_correction");
}

template <typename T>
int lse_solve_once(mpir_ctx *h, int m, int n, int p, const double *A, int lda, const double *B, int ldb,
                   const double *b, const double *d, double *x, double *r_out, double *v_out,
                   const mpir_opts &o, int fact, mpir_info *info, bool factored = false)
{
    cudaStream_t s = h->stream;
    const bool left = o.refine == MPIR_GMRES_LEFT;
    const bool gm = o.refine == MPIR_GMRES || left;
    size_t main_bytes = 0;
    lse_layout<T>(nullptr, m, n, p, &main_bytes);
    const int NG = m + p + n, mx = std::max(std::max(m, n), std::max(p, 1));
    if (gm) {
        if (o.restart > GMRES_MAX_RESTART) return set_err(h, MPIR_UNSUPPORTED, "GMRES restart above 64");
        RC(ensure_ws(h, main_bytes + bd_bytes(NG, o.restart, mx)));
    }
    if (!factored) {              // else factored (and timed) by the caller
        cudaEventRecord(h->ev[0], s);
        RC(lse_factor_impl<T>(h, m, n, p, A, lda, B, ldb, fact));
        cudaEventRecord(h->ev[1], s);
    }
    LseWs<T> w = lse_layout<T>(h->ws, m, n, p, nullptr);
    BDScratch bs{};
    if (gm) bs = bd_layout((char *)h->ws + main_bytes, NG, o.restart, mx);
    double *r = r_out ? r_out : w.r;
    double *v = v_out ? v_out : w.v;
    RC(lse_initial_impl<T>(h, b, d, x));
    int st = MPIR_OK, it = 0, inner = 0;
    double ratio[3] = {0, 0, 0};
    double al = 1.0;
    float t_gm = 0;
    if (o.refine != MPIR_DIRECT || r_out || v_out) RC(lse_multipliers_impl<T>(h, A, lda, b, x, r, v));
    bool looped = false;
    const bool dd = o.resid_dd != 0;
    if (dd) RC(ensure_rws(h, sizeof(double) * (2 * (size_t)(m + p + 2 * n) + n + 8)));
    if (o.refine == MPIR_CLASSICAL && ir_graph_usable(h) && !dd) {
        // the loop on the device (one CUDA-graph launch, one host read)
        unsigned long long key = ir_mix(ir_mix(ir_mix(0, 1), sizeof(T)), (unsigned long long)m);
        for (unsigned long long v_ : {(unsigned long long)n, (unsigned long long)p, (unsigned long long)lda,
                                      (unsigned long long)ldb, (unsigned long long)(uintptr_t)A,
                                      (unsigned long long)(uintptr_t)B, (unsigned long long)(uintptr_t)b,
                                      (unsigned long long)(uintptr_t)d, (unsigned long long)(uintptr_t)x,
                                      (unsigned long long)(uintptr_t)r, (unsigned long long)(uintptr_t)v,
                                      (unsigned long long)(uintptr_t)h->ws, (unsigned long long)o.maxit,
                                      (unsigned long long)std::llround(-std::log2(o.tol) * 4096.0),
                                      (unsigned long long)h->fs.colscale})
            key = ir_mix(key, v_);
        ir_stage_scalars(h, w.ird);
        auto pre = [&](cudaGraphConditionalHandle hc) {
            k_ir_reset<<<1, 32, 0, h->stream>>>(w.ird);
            absmax_sumsq(b, std::max(m, 1), m, 1, w.part, w.ird + IRD_N1, h->stream);
            if (p > 0) absmax_sumsq(d, std::max(p, 1), p, 1, w.part, w.ird + IRD_N2, h->stream);
            lse_residual_dev<T>(h, w, A, lda, B, ldb, b, d, x, r, v);
            k_ir_control<<<1, 32, 0, h->stream>>>(w.norms2, w.ird, 0, o.tol, o.maxit, hc, 1);
            return cudaGetLastError() == cudaSuccess ? 0 : 1;
        };
        auto body = [&](cudaGraphConditionalHandle hc) {
            int rc = lse_correction_impl<T>(h, w.f1, w.f2, w.f3, 1.0, r, v, x, w.ird + IRD_C);
            lse_residual_dev<T>(h, w, A, lda, B, ldb, b, d, x, r, v);
            k_ir_control<<<1, 32, 0, h->stream>>>(w.norms2, w.ird, 0, o.tol, o.maxit, hc, 1);
            return rc == 0 && cudaGetLastError() == cudaSuccess ? 0 : 1;
        };
        const int gr = ir_graph_run(h, w.ird, key, pre, body, &it, &st, ratio);
        if (gr < 0 || gr == MPIR_CUDA_ERROR) return gr;
        if (gr == 0) looped = true;
        else h->irg_off = true;       // capture not available: the host loop from now on
    }
    if (o.refine != MPIR_DIRECT && !looped) {
        const double nb = dnorm_host(h, b, m, w.part), nd = p > 0 ? dnorm_host(h, d, p, w.part) : 0.0;
        const double fA = h->fs.fro1, fB = h->fs.fro2;
        StopState ss;
        st = MPIR_NOT_CONVERGED;
        float t_res = 0;
        double *dds = dd ? (double *)h->rws : nullptr;
        double *xprev = dd ? dds + 2 * (size_t)(m + p + 2 * n) : nullptr, *dxn = dd ? xprev + n : nullptr;
        FwdState fw;
        bool bw = false;
        auto post = [&]() -> int {              // after a correction (u_r < u variant): ||dx||
            if (!dd) return 0;
            diff_norm2(x, xprev, n, dxn, 0, s);
            RC(read_back(h, dxn, 1));
            fw.push(std::sqrt(h->hbuf[0]));
            return 0;
        };
        for (it = 0; it < o.maxit; it++) {
            cudaEventRecord(h->ev[3], s);
            if (dd) {
                if (lse_resid_dd(m, n, p, A, lda, B, ldb, b, d, x, r, v, dds, w.f1, w.f2, w.f3, w.norms2, s) !=
                    cudaSuccess)
                    return cuda_check(h, "lse double-double residual");
            } else {
                lse_residual_dev<T>(h, w, A, lda, B, ldb, b, d, x, r, v);
            }
            cudaEventRecord(h->ev[4], s);
            RC(read_back(h, w.norms2, 6));
            t_res += ev_ms(h->ev[3], h->ev[4]);
            double nr[6];
            for (int i = 0; i < 6; i++) nr[i] = std::sqrt(h->hbuf[i]);
            // nr: f1 f2 f3 x r v
            double den[3] = {nb + nr[4] + fA * nr[3], nd + fB * nr[3], fA * nr[4] + fB * nr[5]};
            bool bad = false;
            for (int i = 0; i < 3; i++) if (!std::isfinite(nr[i])) bad = true;
            if (bad) { st = MPIR_NONFINITE; break; }
            bw = stop_test(nr, den, o.tol, ratio);
            if (bw && (!dd || fw.done(nr[3]))) { st = MPIR_OK; break; }
            if (!bw) {
                const double eta = std::max(ratio[0], std::max(ratio[1], ratio[2]));
                if (eta < 0.5 * ss.best) { ss.best = eta; ss.since_best = 0; }
                else if (++ss.since_best >= 3) { st = ss.best <= 1e-14 ? MPIR_OK : MPIR_NOT_CONVERGED; break; }
            }
            if (dd) cudaMemcpyAsync(xprev, x, sizeof(double) * n, cudaMemcpyDeviceToDevice, s);
            // normalize the right-hand side of the scaled correction system
            // (f1, sB/sA f2, sA f3), not the raw blocks
            if (gm) {
                // Sec. 5.2: correction from GMRES on the preconditioned F~
                if (it == 0) al = bd_alpha(o, nr[4], fA, nr[3]);
                cudaEventRecord(h->ev[5], s);
                if (left)       // Sec. 5.1: M = F~^-1 applied by Alg. 1
                    RC(lse_gmres_left_correction<T>(h, w, bs, A, lda, B, ldb, al, o.beta,
                                                    inner_tol_default(o, fact), o.inner_maxit, r, v, x, &inner));
                else
                    RC(lse_gmres_correction<T>(h, w, bs, A, lda, B, ldb, al, o.beta, inner_tol_default(o, fact),
                                               o.inner_maxit, r, v, x, &inner, it == 0));
                cudaEventRecord(h->ev[6], s);
                cudaEventSynchronize(h->ev[6]);
                t_gm += ev_ms(h->ev[5], h->ev[6]);
                RC(post());
                continue;
            }
            const double sA = h->fs.s1, sB = h->fs.s2;
            const double gamma = pow2_norm(std::max(nr[0], std::max(nr[1] * sB / sA, nr[2] * sA)));
            RC(lse_correction_impl<T>(h, w.f1, w.f2, w.f3, gamma, r, v, x));
            RC(post());
        }
        if (st == MPIR_NOT_CONVERGED && bw) st = MPIR_OK;     // maxit with the backward test met
        if (info) { info->time_ms[2] = t_res; info->time_ms[4] = t_gm; info->inner_iters = inner; }
    }
    RC(check_dev_flags(h));
    cudaEventRecord(h->ev[7], s);
    cudaEventSynchronize(h->ev[7]);
    if (info) {
        info->status = st;
        info->iters = it;
        info->fact_used = fact;
        info->refine_used = o.refine;
        for (int i = 0; i < 3; i++) info->stop_ratio[i] = ratio[i];
        info->time_ms[0] = ev_ms(h->ev[0], h->ev[1]);
        info->time_ms[5] = ev_ms(h->ev[0], h->ev[7]);
    }
    return st;
}

int next_prec(int fact)
{
    if (fact == MPIR_BF16 || fact == MPIR_TF32) return MPIR_FP32;
    if (fact == MPIR_FP32) return MPIR_FP64;
    return -1;
}

bool is_fp64(int fact) { return fact == MPIR_FP64; }

} // namespace

// ============================================================== C ABI ==

extern "C" {

const char *mpir_version(void) { return MPIR_VERSION_STRING; }

int mpir_profile(int enable)
{
    g_prof = enable != 0;
    g_nrec = 0;
    g_open = false;
    if (g_prof && g_ev.size() < 2 * PROF_CAP) {
        const size_t old = g_ev.size();
        g_ev.resize(2 * PROF_CAP);
        for (size_t i = old; i < g_ev.size(); i++) cudaEventCreate(&g_ev[i]);
        g_kind.resize(PROF_CAP);
    }
    return 0;
}

int mpir_profile_read(double *ms, long long *launches, int nkinds)
{
    if (nkinds > K_NKINDS) nkinds = K_NKINDS;
    for (int k = 0; k < nkinds; k++) { if (ms) ms[k] = 0.0; if (launches) launches[k] = 0; }
    if (g_nrec) cudaEventSynchronize(g_ev[2 * g_nrec - 1]);
    for (size_t i = 0; i < g_nrec; i++) {
        float t = 0;
        cudaEventElapsedTime(&t, g_ev[2 * i], g_ev[2 * i + 1]);
        int k = g_kind[i];
        if (k < nkinds) { if (ms) ms[k] += t; if (launches) launches[k]++; }
    }
    return nkinds;
}

long long mpir_launch_count(int kind)
{
    if (kind < 0) {
        long long t = 0;
        for (int k = 0; k < K_NKINDS; k++) t += g_launches[k].load(std::memory_order_relaxed);
        return t;
    }
    return kind < K_NKINDS ? g_launches[kind].load(std::memory_order_relaxed) : 0;
}

const char *mpir_kernel_kind_name(int kind)
{
    return (kind >= 0 && kind < K_NKINDS) ? g_kind_names[kind] : "";
}

void mpir_default_opts(mpir_opts *o)
{
    if (!o) return;
    std::memset(o, 0, sizeof(*o));
    o->fact = MPIR_FP32;
    o->refine = MPIR_CLASSICAL;
    o->tol = 1e-15;
    o->maxit = 40;
    o->restart = 30;
    o->inner_maxit = 300;
    o->inner_tol = 0;
    o->alpha = 0;
    o->beta = 1.0;
    o->escalate = 1;
}

int mpir_create(mpir_handle *handle, int device, void *stream)
{
    if (!handle) return -1;
    *handle = nullptr;
    if (device < 0 && cudaGetDevice(&device) != cudaSuccess) { cudaGetLastError(); return MPIR_CUDA_ERROR; }
    DeviceScope ds(device);
    if (!ds.ok) return MPIR_CUDA_ERROR;
    mpir_ctx *h = new mpir_ctx();
    h->device = device;
    h->stream = (cudaStream_t)stream;
    const size_t part_bytes = 1 << 20;
    if (cudaMalloc(&h->scratch_base, 4096 + part_bytes) != cudaSuccess) { delete h; cudaGetLastError(); return MPIR_CUDA_ERROR; }
    cudaMemset(h->scratch_base, 0, 4096 + part_bytes);
    char *b = (char *)h->scratch_base;
    h->sc.barrier = (unsigned int *)b;
    h->sc.err = (int *)(b + 256);
    h->sc.status = (int *)(b + 512);
    h->sc.part = b + 4096;
    h->sc.part_bytes = part_bytes;
    if (cudaMallocHost(&h->hbuf, 64 * sizeof(double)) != cudaSuccess) { cudaFree(h->scratch_base); delete h; cudaGetLastError(); return MPIR_CUDA_ERROR; }
    for (int i = 0; i < 8; i++) cudaEventCreate(&h->ev[i]);
    cudaEventCreateWithFlags(&h->sw_ev, cudaEventDisableTiming);
    cudaDeviceSynchronize();
    *handle = h;
    return 0;
}

int mpir_destroy(mpir_handle h)
{
    if (!h) return -1;
    DeviceScope ds(h->device);
    cudaStreamSynchronize(h->stream);
    if (h->side) cudaStreamSynchronize(h->side);
    if (h->crit) cudaStreamSynchronize(h->crit);
    if (h->aux) cudaStreamSynchronize(h->aux);
    if (h->ws && h->ws_owned) cudaFree(h->ws);
    if (h->scratch_base) cudaFree(h->scratch_base);
    if (h->rws) cudaFree(h->rws);
    if (h->zbuf) cudaFree(h->zbuf);
    if (h->hbuf) cudaFreeHost(h->hbuf);
    {
        BatchArena &a = h->ba;
        if (a.graph) cudaGraphExecDestroy(a.graph);
        cudaFree(a.tab); cudaFree(a.order); cudaFree(a.res); cudaFree(a.next); cudaFree(a.gscr);
        if (a.htab) cudaFreeHost(a.htab);
        if (a.hres) cudaFreeHost(a.hres);
        if (a.horder) cudaFreeHost(a.horder);
        if (h->irg) cudaGraphExecDestroy(h->irg);
        if (h->cap_stream) cudaStreamDestroy(h->cap_stream);
    }
    if (h->side) {
        cudaStreamSynchronize(h->side);
        cudaStreamDestroy(h->side);
        cudaEventDestroy(h->side_fork);
        cudaEventDestroy(h->side_join);
    }
    if (h->crit) {
        cudaStreamSynchronize(h->crit);
        cudaStreamDestroy(h->crit);
        cudaEventDestroy(h->la_a);
        cudaEventDestroy(h->la_b);
    }
    if (h->aux) {
        cudaStreamSynchronize(h->aux);
        cudaStreamDestroy(h->aux);
        cudaEventDestroy(h->ax_a);
        cudaEventDestroy(h->ax_b);
    }
    if (h->sel_stream) {
        cudaStreamSynchronize(h->sel_stream);
        cudaStreamDestroy(h->sel_stream);
        cudaEventDestroy(h->sel_ev);
    }
    if (h->sel_host) cudaFreeHost(h->sel_host);
    if (h->sel) cudaFree(h->sel);
    if (h->sel_s) cudaFree(h->sel_s);
    for (int i = 0; i < 8; i++) cudaEventDestroy(h->ev[i]);
    if (h->sw_ev) cudaEventDestroy(h->sw_ev);
    delete h;
    return 0;
}

int mpir_set_stream(mpir_handle h, void *stream)
{
    if (!h) return -1;
    const cudaStream_t ns = (cudaStream_t)stream;
    if (ns != h->stream && h->sw_ev) {
        // work queued on the old stream, and on the internal streams joined
        // into it, finishes before the new stream touches the handle's buffers
        join_side(h, h->stream);
        cudaEventRecord(h->sw_ev, h->stream);
        cudaStreamWaitEvent(ns, h->sw_ev, 0);
    }
    h->stream = ns;
    return 0;
}

int mpir_set_workspace(mpir_handle h, void *ptr, size_t bytes)
{
    if (!h) return -1;
    if (((uintptr_t)ptr & 255) != 0) return -2;
    if (h->side) cudaStreamSynchronize(h->side);
    if (h->crit) cudaStreamSynchronize(h->crit);
    if (h->aux) cudaStreamSynchronize(h->aux);
    if (h->ws && h->ws_owned) { cudaStreamSynchronize(h->stream); cudaFree(h->ws); }
    h->ws = ptr;
    h->ws_bytes = ptr ? bytes : 0;
    h->ws_owned = false;
    h->fs.kind = Kind::NONE;             // held factors lived in the previous workspace
    return 0;
}

const char *mpir_last_error(mpir_handle h)
{
    static const char *none = "";
    if (!h) return none;
    // a size or launch-shape limit inside a kernel's host code records only
    // its source location
    if (h->err.empty() && unsupported_where()) return unsupported_where();
    return h->err.c_str();
}

int mpir_lse_workspace_size(int m, int n, int p, const mpir_opts *opts, size_t *bytes)
{
    if (!bytes) return -5;
    if (m < 0) return -1;
    if (n < 0) return -2;
    if (p < 0 || p > n || n > m + p) return -3;
    mpir_opts o;
    fill_opts(opts, &o);
    size_t b32 = 0, b64 = 0;
    lse_layout<float>(nullptr, m, n, p, &b32);
    lse_layout<double>(nullptr, m, n, p, &b64);
    *bytes = (o.fact == MPIR_FP64 || o.escalate) ? std::max(b32, b64) : b32;
    if (o.refine == MPIR_GMRES || o.refine == MPIR_GMRES_LEFT)
        *bytes += bd_bytes(m + p + n, std::min(o.restart, GMRES_MAX_RESTART), std::max(std::max(m, n), std::max(p, 1)));
    return 0;
}

int mpir_gls_workspace_size(int n, int m, int p, const mpir_opts *opts, size_t *bytes)
{
    if (!bytes) return -5;
    if (n < 0) return -1;
    if (m < 0 || m > n) return -2;
    if (p < 0 || n > m + p) return -3;
    mpir_opts o;
    fill_opts(opts, &o);
    size_t b32 = 0, b64 = 0;
    gls_layout<float>(nullptr, n, m, p, &b32);
    gls_layout<double>(nullptr, n, m, p, &b64);
    *bytes = (o.fact == MPIR_FP64 || o.escalate) ? std::max(b32, b64) : b32;
    if (o.refine == MPIR_GMRES || o.refine == MPIR_GMRES_LEFT)
        *bytes += bd_bytes(p + n + m, std::min(o.restart, GMRES_MAX_RESTART), std::max(std::max(m, n), std::max(p, 1)));
    return 0;
}

static int lse_check_args(int m, int n, int p, const double *A, int lda, const double *B, int ldb,
                          const double *b, const double *d, const double *x)
{
    if (m < 0) return -2;
    if (n < 1) return -3;
    if (p < 0 || p > n || n > m + p) return -4;
    if (!A) return -5;
    if (lda < std::max(1, m)) return -6;
    if (p > 0 && !B) return -7;
    if (ldb < std::max(1, p)) return -8;
    if (!b && m > 0) return -9;
    if (!d && p > 0) return -10;
    if (!x) return -11;
    return 0;
}

static int gls_check_args(int n, int m, int p, const double *W, int ldw, const double *V, int ldv,
                          const double *d, const double *x, const double *y)
{
    if (n < 1) return -2;
    if (m < 0 || m > n) return -3;
    if (p < 0 || n > m + p) return -4;
    if (!W && m > 0) return -5;
    if (ldw < std::max(1, n)) return -6;
    if (!V && p > 0) return -7;
    if (ldv < std::max(1, n)) return -8;
    if (!d) return -9;
    if (!x && m > 0) return -10;
    if (!y && p > 0) return -11;
    return 0;
}

// ------------------------------------------------------------ selector --
// splitmix64 (Steele, Lea, Flood 2014) of seed + j mapped to [-1, 1).
static double splitmix_unit(unsigned long long x)
{
    unsigned long long z = x + 0x9E3779B97F4A7C15ULL;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
    z ^= z >> 31;
    return (double)(z >> 11) * (1.0 / 9007199254740992.0) * 2.0 - 1.0;
}

static int sel_start_vector(mpir_ctx *h, int len)
{
    if ((size_t)len <= h->sel_s_len) return 0;
    if (h->sel_s) { cudaStreamSynchronize(h->stream); cudaFree(h->sel_s); h->sel_s = nullptr; h->sel_s_len = 0; }
    std::vector<double> v(len);
    for (int j = 0; j < len; j++) v[j] = splitmix_unit(0x5EEDULL + (unsigned long long)j);
    if (cudaMalloc(&h->sel_s, sizeof(double) * len) != cudaSuccess) {
        cudaGetLastError();
        return set_err(h, MPIR_CUDA_ERROR, "selector: cudaMalloc failed");
    }
    cudaMemcpy(h->sel_s, v.data(), sizeof(double) * len, cudaMemcpyHostToDevice);
    h->sel_s_len = len;
    return 0;
}

// Features -> standardized input -> MLP -> most probable class, on the
// selector's own stream: sel_begin enqueues the features (and their copy to
// pinned host memory) and returns at once, so the caller can put the
// likeliest path (the FP32 factorization) on the GPU meanwhile; sel_end
// waits for the features, runs the MLP and returns the class.
static int sel_begin(mpir_ctx *h, int kind, int d0, int d1, int d2, const double *M1, int ld1, const double *M2,
                     int ld2, const double *v1, int n1, const double *v2, int n2)
{
    if (!h->sel) return set_err(h, MPIR_UNSUPPORTED, "fact = MPIR_AUTO needs a selector (mpir_selector_set)");
    const int R = kind == 0 ? d0 + d2 : d0, C = kind == 0 ? d1 : d1 + d2;
    RC(sel_start_vector(h, C));
    RC(ensure_rws(h, sizeof(double) * features_ws_doubles(R, C)));
    if (!h->sel_stream) {
        if (cudaStreamCreateWithFlags(&h->sel_stream, cudaStreamNonBlocking) != cudaSuccess ||
            cudaEventCreateWithFlags(&h->sel_ev, cudaEventDisableTiming) != cudaSuccess ||
            cudaMallocHost(&h->sel_host, 32 * sizeof(float)) != cudaSuccess) {
            cudaGetLastError();
            return set_err(h, MPIR_CUDA_ERROR, "selector: stream or pinned buffer");
        }
    }
    // the selector stream starts where the caller's stream is (inputs ready)
    cudaEventRecord(h->sel_ev, h->stream);
    cudaStreamWaitEvent(h->sel_stream, h->sel_ev, 0);
    float *feat = h->sel + MLP_PARAMS + 16 + 8;
    cudaStream_t ss = h->sel_stream;
    // features_launch takes GLS dimensions as (columns of W, rows, columns of V)
    const int fm = kind == 0 ? d0 : d1, fn = kind == 0 ? d1 : d0;
    RC(features_launch(kind, fm, fn, d2, M1, ld1, M2, ld2, h->sel_s, v1, n1, v2, n2, 16, (double *)h->rws, feat,
                       ss));
    cudaMemcpyAsync(h->sel_host, feat, 16 * sizeof(float), cudaMemcpyDeviceToHost, ss);
    cudaEventRecord(h->sel_ev, ss);
    return 0;
}

static int sel_end(mpir_ctx *h, int *cls)
{
    float *X = h->sel + MLP_PARAMS, *prob = X + 16;
    cudaStream_t ss = h->sel_stream;
    if (cudaEventSynchronize(h->sel_ev) != cudaSuccess) return cuda_check(h, "selector features");
    float f[16];
    for (int q = 0; q < 16; q++) f[q] = (h->sel_host[q] - h->sel_mean[q]) / h->sel_scale[q];
    std::memcpy(h->sel_host + 16, f, 16 * sizeof(float));
    cudaMemcpyAsync(X, h->sel_host + 16, sizeof(f), cudaMemcpyHostToDevice, ss);
    RC(mlp_forward(h->sel, X, 1, prob, ss));
    cudaMemcpyAsync(h->sel_host, prob, sizeof(float) * NCLASS, cudaMemcpyDeviceToHost, ss);
    if (cudaStreamSynchronize(ss) != cudaSuccess) return cuda_check(h, "selector forward");
    int best = 0;
    for (int c = 1; c < NCLASS; c++) if (h->sel_host[c] > h->sel_host[best]) best = c;
    *cls = best;
    return 0;
}

static void sel_apply(int cls, mpir_opts *o)
{
    static const int facts[3] = {MPIR_BF16, MPIR_FP32, MPIR_FP64};
    o->fact = facts[cls / 2];
    o->refine = (cls % 2) ? MPIR_GMRES : MPIR_CLASSICAL;
}

int lse_solve(mpir_handle h, int m, int n, int p, const double *A, int lda, const double *B, int ldb,
              const double *b, const double *d, double *x, double *r, double *v, const mpir_opts *opts,
              mpir_info *info)
{
    if (!h) return -1;
    int a = lse_check_args(m, n, p, A, lda, B, ldb, b, d, x);
    if (a) return set_err(h, a, "illegal argument");
    mpir_opts o;
    fill_opts(opts, &o);
    if (info) std::memset(info, 0, sizeof(*info));
    bool factored = false;
    if (o.fact == MPIR_AUTO) {
        // the FP32 factors are computed while the selector decides; they are
        // kept when it picks an FP32 class
        size_t mb = 0;
        lse_layout<float>(nullptr, m, n, p, &mb);
        const int NG = m + p + n, mx = std::max(std::max(m, n), std::max(p, 1));
        RC(ensure_ws(h, mb + bd_bytes(NG, std::min(o.restart, GMRES_MAX_RESTART), mx)));
        RC(sel_begin(h, 0, m, n, p, A, lda, B, std::max(ldb, 1), b, m, d, p));
        cudaEventRecord(h->ev[0], h->stream);
        RC(lse_factor_impl<float>(h, m, n, p, A, lda, B, ldb, MPIR_FP32));
        cudaEventRecord(h->ev[1], h->stream);
        int cls = 0;
        RC(sel_end(h, &cls));
        sel_apply(cls, &o);
        factored = o.fact == MPIR_FP32;
    }
    if (o.fact < MPIR_BF16 || o.fact > MPIR_FP64) return set_err(h, -14, "illegal opts->fact");
    int fact = o.fact;
    int esc = 0, st = 0;
    while (true) {
        st = is_fp64(fact) ? lse_solve_once<double>(h, m, n, p, A, lda, B, ldb, b, d, x, r, v, o, fact, info)
                           : lse_solve_once<float>(h, m, n, p, A, lda, B, ldb, b, d, x, r, v, o, fact, info,
                                                   factored && esc == 0);
        if (st == MPIR_OK || st < 0 || st == MPIR_CUDA_ERROR || st == MPIR_UNSUPPORTED ||
            st == MPIR_DEVICE_TIMEOUT || !o.escalate || o.refine == MPIR_DIRECT)
            break;
        int nf = next_prec(fact);
        if (nf < 0) break;
        fact = nf;
        esc++;
    }
    if (info) info->escalated = esc;
    return st;
}

int gls_solve(mpir_handle h, int n, int m, int p, const double *W, int ldw, const double *V, int ldv,
              const double *d, double *x, double *y, double *z, const mpir_opts *opts, mpir_info *info)
{
    if (!h) return -1;
    int a = gls_check_args(n, m, p, W, ldw, V, ldv, d, x, y);
    if (a) return set_err(h, a, "illegal argument");
    mpir_opts o;
    fill_opts(opts, &o);
    if (info) std::memset(info, 0, sizeof(*info));
    bool factored = false;
    if (o.fact == MPIR_AUTO) {
        size_t mb = 0;
        gls_layout<float>(nullptr, n, m, p, &mb);
        const int NG = p + n + m, mx = std::max(std::max(m, n), std::max(p, 1));
        RC(ensure_ws(h, mb + bd_bytes(NG, std::min(o.restart, GMRES_MAX_RESTART), mx)));
        RC(sel_begin(h, 1, n, m, p, W, ldw, V, ldv, d, n, nullptr, 0));
        cudaEventRecord(h->ev[0], h->stream);
        RC(gls_factor_impl<float>(h, n, m, p, W, ldw, V, ldv, MPIR_FP32));
        cudaEventRecord(h->ev[1], h->stream);
        int cls = 0;
        RC(sel_end(h, &cls));
        sel_apply(cls, &o);
        factored = o.fact == MPIR_FP32;
    }
    if (o.fact < MPIR_BF16 || o.fact > MPIR_FP64) return set_err(h, -14, "illegal opts->fact");
    int fact = o.fact;
    int esc = 0, st = 0;
    while (true) {
        st = is_fp64(fact) ? gls_solve_once<double>(h, n, m, p, W, ldw, V, ldv, d, x, y, z, o, fact, info)
                           : gls_solve_once<float>(h, n, m, p, W, ldw, V, ldv, d, x, y, z, o, fact, info,
                                                   factored && esc == 0);
        if (st == MPIR_OK || st < 0 || st == MPIR_CUDA_ERROR || st == MPIR_UNSUPPORTED ||
            st == MPIR_DEVICE_TIMEOUT || !o.escalate || o.refine == MPIR_DIRECT)
            break;
        int nf = next_prec(fact);
        if (nf < 0) break;
        fact = nf;
        esc++;
    }
    if (info) info->escalated = esc;
    return st;
}

// Complex LSE / GLS (the problems of Sec. 1 over C) through the real 2 x 2
// block embedding E(Z) = [Re Z, -Im Z; Im Z, Re Z] (complex.cu): the
// embedded problem has the same solution (as [Re; Im]), the same singular
// values and the same stop-test quantities, and runs the real path.
int zlse_solve(mpir_handle h, int m, int n, int p, const double *A, int lda, const double *B, int ldb,
               const double *b, const double *d, double *x, double *r, double *v, const mpir_opts *opts,
               mpir_info *info)
{
    if (!h) return -1;
    int a = lse_check_args(m, n, p, A, lda, B, ldb, b, d, x);
    if (a) return set_err(h, a, "illegal argument");
    const int M = 2 * m, N = 2 * n, P = 2 * p;
    const size_t words = (size_t)M * N + (size_t)P * N + (size_t)2 * M + (size_t)2 * P + N;
    RC(ensure_zbuf(h, sizeof(double) * std::max<size_t>(words, 1)));
    double *Ah = h->zbuf, *Bh = Ah + (size_t)M * N, *bh = Bh + (size_t)P * N, *dh = bh + M, *xh = dh + P;
    double *rh = xh + N, *vh = rh + M;
    cudaStream_t s = h->stream;
    RC(zembed_mat(A, m, n, lda, Ah, std::max(M, 1), s));
    RC(zembed_mat(B, p, n, ldb, Bh, std::max(P, 1), s));
    RC(zembed_vec(b, m, bh, s));
    RC(zembed_vec(d, p, dh, s));
    const int st = lse_solve(h, M, N, P, Ah, std::max(M, 1), p > 0 ? Bh : nullptr, std::max(P, 1), bh,
                             p > 0 ? dh : nullptr, xh, r ? rh : nullptr, (v && p > 0) ? vh : nullptr, opts, info);
    if (st < 0 || st == MPIR_CUDA_ERROR) return st;
    RC(zunembed_vec(xh, n, x, s));
    if (r) RC(zunembed_vec(rh, m, r, s));
    if (v && p > 0) RC(zunembed_vec(vh, p, v, s));
    if (cudaStreamSynchronize(s) != cudaSuccess) return cuda_check(h, "zlse_solve");
    return st;
}

int zgls_solve(mpir_handle h, int n, int m, int p, const double *W, int ldw, const double *V, int ldv,
               const double *d, double *x, double *y, double *z, const mpir_opts *opts, mpir_info *info)
{
    if (!h) return -1;
    int a = gls_check_args(n, m, p, W, ldw, V, ldv, d, x, y);
    if (a) return set_err(h, a, "illegal argument");
    const int Nn = 2 * n, M = 2 * m, P = 2 * p;
    const size_t words = (size_t)Nn * M + (size_t)Nn * P + (size_t)2 * Nn + M + P;
    RC(ensure_zbuf(h, sizeof(double) * std::max<size_t>(words, 1)));
    double *Wh = h->zbuf, *Vh = Wh + (size_t)Nn * M, *dh = Vh + (size_t)Nn * P, *xh = dh + Nn, *yh = xh + M;
    double *zh = yh + P;
    cudaStream_t s = h->stream;
    RC(zembed_mat(W, n, m, ldw, Wh, Nn, s));
    RC(zembed_mat(V, n, p, ldv, Vh, Nn, s));
    RC(zembed_vec(d, n, dh, s));
    const int st = gls_solve(h, Nn, M, P, m > 0 ? Wh : nullptr, Nn, Vh, Nn, dh, xh, yh, z ? zh : nullptr, opts,
                             info);
    if (st < 0 || st == MPIR_CUDA_ERROR) return st;
    RC(zunembed_vec(xh, m, x, s));
    RC(zunembed_vec(yh, p, y, s));
    if (z) RC(zunembed_vec(zh, n, z, s));
    if (cudaStreamSynchronize(s) != cudaSuccess) return cuda_check(h, "zgls_solve");
    return st;
}

// Per-problem loop over the single-problem solver: GMRES-IR requests and
// the escalation of problems the batched kernel did not converge.
static int lse_solve_each(mpir_handle h, const std::vector<int> &which, const int *m, const int *n, const int *p,
                          const double *const *A, const int *lda, const double *const *B, const int *ldb,
                          const double *const *b, const double *const *d, double *const *x, const mpir_opts &o,
                          mpir_info *infos, int esc_base)
{
    int worst = 0;
    for (int i : which) {
        mpir_info inf;
        int st = lse_solve(h, m[i], n[i], p[i], A[i], lda[i], B[i], ldb[i], b[i], d[i], x[i], nullptr, nullptr, &o,
                           &inf);
        if (st < 0) return st;
        inf.escalated += esc_base;
        if (infos) infos[i] = inf;
        worst = std::max(worst, st);
    }
    return worst;
}

static int batch_reserve(mpir_ctx *h, int count, size_t gscr_bytes)
{
    BatchArena &a = h->ba;
    if ((size_t)count > a.cap) {
        cudaStreamSynchronize(h->stream);
        cudaFree(a.tab); cudaFree(a.order); cudaFree(a.res); cudaFree(a.next);
        a.tab = nullptr; a.order = nullptr; a.res = nullptr; a.next = nullptr; a.cap = 0;
        if (a.graph) { cudaGraphExecDestroy(a.graph); a.graph = nullptr; a.graph_key = 0; }
        const size_t c = std::max<size_t>(count, 256);
        if (cudaMalloc(&a.tab, c * sizeof(BInst)) != cudaSuccess || cudaMalloc(&a.order, c * sizeof(int)) != cudaSuccess ||
            cudaMalloc(&a.res, c * sizeof(BResult)) != cudaSuccess || cudaMalloc(&a.next, 256) != cudaSuccess) {
            cudaGetLastError();
            return set_err(h, MPIR_CUDA_ERROR, "batched tables: cudaMalloc failed");
        }
        a.cap = c;
    }
    if ((size_t)count > a.hcap) {
        if (a.htab) cudaFreeHost(a.htab);
        if (a.hres) cudaFreeHost(a.hres);
        if (a.horder) cudaFreeHost(a.horder);
        a.htab = nullptr; a.hres = nullptr; a.horder = nullptr; a.hcap = 0;
        const size_t c = std::max<size_t>(count, 256);
        if (cudaMallocHost(&a.htab, c * sizeof(BInst)) != cudaSuccess ||
            cudaMallocHost(&a.hres, c * sizeof(BResult)) != cudaSuccess ||
            cudaMallocHost(&a.horder, c * sizeof(int)) != cudaSuccess) {
            cudaGetLastError();
            return set_err(h, MPIR_CUDA_ERROR, "batched staging: cudaMallocHost failed");
        }
        a.hcap = c;
    }
    if (gscr_bytes > a.gscr_bytes) {
        cudaStreamSynchronize(h->stream);
        cudaFree(a.gscr);
        a.gscr = nullptr; a.gscr_bytes = 0;
        if (a.graph) { cudaGraphExecDestroy(a.graph); a.graph = nullptr; a.graph_key = 0; }
        if (cudaMalloc(&a.gscr, gscr_bytes) != cudaSuccess) {
            cudaGetLastError();
            return set_err(h, MPIR_CUDA_ERROR, "batched scratch: cudaMalloc failed");
        }
        a.gscr_bytes = gscr_bytes;
    }
    if (!h->cap_stream && cudaStreamCreateWithFlags(&h->cap_stream, cudaStreamNonBlocking) != cudaSuccess) {
        cudaGetLastError();
        return set_err(h, MPIR_CUDA_ERROR, "batched: stream creation failed");
    }
    return 0;
}

static unsigned long long mix64(unsigned long long h, unsigned long long v)
{
    h ^= v + 0x9e3779b97f4a7c15ULL + (h << 6) + (h >> 2);
    return h;
}

// Candidate launch shapes for a bucket of problems: 512-thread CTAs split
// into groups of 512, 256, 128 or 64 threads (one problem per group), each
// group with an equal share of the shared memory, as much as the bucket's
// largest problem can use (smem_full) but at least what every problem needs
// with its factors in global scratch (smem_min).
static std::vector<BConfig> batch_candidates(size_t smem_min, size_t smem_full, size_t optin)
{
    std::vector<BConfig> c;
    for (int gt : {512, 256, 128, 64}) {
        const int G = 512 / gt;
        size_t per = std::min(smem_full, (optin / G) & ~(size_t)15);
        per = (std::max(per, smem_min) + 15) & ~(size_t)15;
        if (per * G > optin) continue;
        c.push_back(BConfig{gt, per * G});
    }
    return c;
}

// Time each candidate on a stratified sample of the bucket (every k-th
// problem of its largest-first order) and keep the fastest; cached per
// handle by a signature of the bucket.
static int batch_tune(mpir_ctx *h, bool fp64, const int *border, int bcount, int *dsamp, int *next,
                      unsigned long long sig, size_t smem_min, size_t smem_full, size_t gstride,
                      const BParams &prm, BConfig *out)
{
    BatchArena &a = h->ba;
    sig = mix64(sig, (unsigned long long)a.force_group);
    for (const auto &t : a.tuned)
        if (t.sig == sig && t.fp64 == fp64) { *out = t.cfg; return 0; }
    int dev = 0, sms = 0, optin = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    const size_t cap = (size_t)optin - 2048;   // static shared memory of the kernel
    std::vector<BConfig> cand = batch_candidates(smem_min, smem_full, cap);
    if (a.force_group) {
        std::vector<BConfig> f;
        for (const BConfig &c : cand)
            if (c.group == a.force_group) f.push_back(c);
        if (!f.empty()) cand = f;
    }
    if (cand.empty()) return set_err(h, MPIR_UNSUPPORTED, "batched: a problem needs more shared memory than a CTA has");
    const int want = std::min(bcount, 8 * sms);
    const int stride = std::max(1, bcount / std::max(want, 1));
    std::vector<int> samp;
    for (int k = 0; k < bcount && (int)samp.size() < want; k += stride) samp.push_back(border[k]);
    cudaMemcpyAsync(dsamp, samp.data(), samp.size() * sizeof(int), cudaMemcpyHostToDevice, h->stream);
    float best = INFINITY;
    BConfig pick = cand[0];
    for (const BConfig &c : cand) {
        const int per = batched_ctas_per_sm(c, fp64);
        if (per <= 0) continue;
        const int grid = sms * per;
        if ((size_t)grid * (512 / c.group) * gstride * (fp64 ? 8 : 4) > a.gscr_bytes) continue;
        RC(batched_launch(c, fp64, a.tab, dsamp, (int)samp.size(), next, a.res, a.gscr, gstride, grid, prm,
                          h->stream));   // warm-up (module load, caches)
        cudaEventRecord(h->ev[5], h->stream);
        RC(batched_launch(c, fp64, a.tab, dsamp, (int)samp.size(), next, a.res, a.gscr, gstride, grid, prm,
                          h->stream));
        cudaEventRecord(h->ev[6], h->stream);
        if (cudaEventSynchronize(h->ev[6]) != cudaSuccess) return cuda_check(h, "batched tune");
        const float t = ev_ms(h->ev[5], h->ev[6]);
        if (t < best) { best = t; pick = c; }
    }
    if (!(best < INFINITY)) return set_err(h, MPIR_UNSUPPORTED, "batched: no launch shape fits");
    a.tuned.push_back({sig, fp64, pick});
    *out = pick;
    return 0;
}

// The persistent batched launch over a table of problems (LSE or GLS, any
// mix): two size buckets, an autotuned launch shape per bucket, the launches
// captured once in a CUDA graph and replayed.  Fills infos (when given) and
// returns the worst status; `redo` receives the problems to escalate.
static int batched_core(mpir_ctx *h, int count, const std::vector<BInst> &insts, const mpir_opts &o,
                        mpir_info *infos, std::vector<int> &redo)
{
    const bool fp64 = o.fact == MPIR_FP64;
    int dev = 0, sms = 0, optin = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    // two size buckets: problems whose whole state fits a quarter of a CTA's
    // shared memory (several problems per CTA) and the others
    const size_t cut = ((size_t)optin - 2048) / 4;
    struct Bucket { std::vector<int> idx; size_t smin = 0, sfull = 0, big = 0; int mmax = 0, nmax = 0, pmax = 0;
                    unsigned kinds = 0; };
    Bucket bk[2];
    std::vector<double> work(count);
    for (int i = 0; i < count; i++) {
        const BInst &t = insts[i];
        const size_t sf = batched_smem_full(t.kind, t.m, t.n, t.p, fp64);
        Bucket &u = bk[sf <= cut ? 1 : 0];
        u.idx.push_back(i);
        u.smin = std::max(u.smin, batched_smem_min(t.kind, t.m, t.n, t.p, fp64));
        u.sfull = std::max(u.sfull, sf);
        u.big = std::max(u.big, batched_big_words(t.kind, t.m, t.n, t.p));
        u.mmax = std::max(u.mmax, t.m); u.nmax = std::max(u.nmax, t.n); u.pmax = std::max(u.pmax, t.p);
        u.kinds |= 1u << t.kind;
        work[i] = batched_work(t.kind, t.m, t.n, t.p);
    }
    const size_t gstride = (std::max(bk[0].big, bk[1].big) + 63) & ~(size_t)63;
    RC(batch_reserve(h, 2 * count, (size_t)8 * sms * gstride * (fp64 ? 8 : 4)));
    BatchArena &a = h->ba;
    for (int i = 0; i < count; i++) a.htab[i] = insts[i];
    // order: bucket 0 (large) then bucket 1, each largest work first
    int off[3] = {0, 0, 0};
    for (int u = 0; u < 2; u++) {
        std::stable_sort(bk[u].idx.begin(), bk[u].idx.end(), [&](int s1, int s2) { return work[s1] > work[s2]; });
        std::copy(bk[u].idx.begin(), bk[u].idx.end(), a.horder + off[u]);
        off[u + 1] = off[u] + (int)bk[u].idx.size();
    }
    cudaStream_t s = h->stream;
    cudaMemcpyAsync(a.tab, a.htab, sizeof(BInst) * count, cudaMemcpyHostToDevice, s);
    cudaMemcpyAsync(a.order, a.horder, sizeof(int) * count, cudaMemcpyHostToDevice, s);
    BParams prm{o.tol, o.maxit, o.refine == MPIR_DIRECT ? MPIR_DIRECT : MPIR_CLASSICAL, 1};
    BConfig cfg[2] = {};
    int grid[2] = {0, 0};
    unsigned long long key = mix64(mix64(0, (unsigned long long)count), fp64);
    for (int u = 0; u < 2; u++) {
        const int bc = off[u + 1] - off[u];
        if (bc == 0) continue;
        unsigned long long sig = mix64(mix64(mix64(mix64(u + 1, bc), bk[u].mmax), bk[u].nmax), bk[u].pmax);
        sig = mix64(sig, bk[u].kinds);
        RC(batch_tune(h, fp64, a.horder + off[u], bc, a.order + count, a.next + 32 * u, sig, bk[u].smin,
                      bk[u].sfull, gstride, prm, &cfg[u]));
        grid[u] = sms * std::max(1, batched_ctas_per_sm(cfg[u], fp64));
        key = mix64(mix64(mix64(mix64(key, sig), cfg[u].group), cfg[u].smem), grid[u]);
    }
    for (int u = 0; u < 2; u++) { a.last[u] = cfg[u]; a.last_count[u] = off[u + 1] - off[u]; }
    key = mix64(mix64(key, (unsigned long long)(uintptr_t)a.gscr), (unsigned long long)(uintptr_t)a.tab);
    key = mix64(mix64(key, o.maxit), prm.refine);
    key = mix64(key, (unsigned long long)std::llround(-std::log2(o.tol) * 1024));
    // the launches, captured once per (shapes, buffers) and replayed
    if (!a.graph || a.graph_key != key) {
        if (a.graph) { cudaGraphExecDestroy(a.graph); a.graph = nullptr; }
        cudaGraph_t g = nullptr;
        if (cudaStreamBeginCapture(h->cap_stream, cudaStreamCaptureModeThreadLocal) != cudaSuccess)
            return cuda_check(h, "batched capture");
        int rc = 0;
        for (int u = 0; u < 2 && !rc; u++)
            rc = batched_launch(cfg[u], fp64, a.tab, a.order + off[u], off[u + 1] - off[u], a.next + 32 * u, a.res,
                                a.gscr, gstride, grid[u], prm, h->cap_stream);
        const cudaError_t ce = cudaStreamEndCapture(h->cap_stream, &g);
        if (rc || ce != cudaSuccess) {
            if (g) cudaGraphDestroy(g);
            cudaGetLastError();
            return set_err(h, rc ? rc : MPIR_CUDA_ERROR, "batched: graph capture failed");
        }
        const cudaError_t ie = cudaGraphInstantiate(&a.graph, g, 0);
        cudaGraphDestroy(g);
        if (ie != cudaSuccess) { a.graph = nullptr; return cuda_check(h, "batched graph instantiate"); }
        a.graph_key = key;
    }
    {
        ProfScope ps(K_BATCHED, s);
        if (cudaGraphLaunch(a.graph, s) != cudaSuccess) return cuda_check(h, "batched graph launch");
    }
    cudaMemcpyAsync(a.hres, a.res, sizeof(BResult) * count, cudaMemcpyDeviceToHost, s);
    if (cudaStreamSynchronize(s) != cudaSuccess) return cuda_check(h, "batched");
    int worst = 0;
    redo.clear();
    for (int i = 0; i < count; i++) {
        const BResult &r = a.hres[i];
        if (infos) {
            mpir_info &f = infos[i];
            f.status = r.status;
            f.iters = r.iters;
            f.fact_used = fp64 ? MPIR_FP64 : MPIR_FP32;
            f.refine_used = prm.refine;
            for (int k = 0; k < 3; k++) f.stop_ratio[k] = r.ratio[k];
        }
        if (r.status != MPIR_OK && o.escalate && !fp64 && prm.refine != MPIR_DIRECT) redo.push_back(i);
        else worst = std::max(worst, r.status);
    }
    return worst;
}

int lse_solve_batched(mpir_handle h, int count, const int *m, const int *n, const int *p,
                      const double *const *A, const int *lda, const double *const *B, const int *ldb,
                      const double *const *b, const double *const *d, double *const *x,
                      const mpir_opts *opts, mpir_info *infos)
{
    if (!h) return -1;
    if (count < 0) return -2;
    if (count == 0) return 0;
    if (!m) return -3;
    if (!n) return -4;
    if (!p) return -5;
    if (!A) return -6;
    if (!lda) return -7;
    if (!B) return -8;
    if (!ldb) return -9;
    if (!b) return -10;
    if (!d) return -11;
    if (!x) return -12;
    for (int i = 0; i < count; i++) {
        const int a = lse_check_args(m[i], n[i], p[i], A[i], lda[i], B[i], ldb[i], b[i], d[i], x[i]);
        if (a) {
            char msg[96];
            std::snprintf(msg, sizeof(msg), "problem %d: illegal argument %d of lse_solve", i, -a);
            return set_err(h, -3, msg);
        }
    }
    mpir_opts o;
    fill_opts(opts, &o);
    if (infos) std::memset(infos, 0, sizeof(mpir_info) * count);
    std::vector<int> all(count);
    for (int i = 0; i < count; i++) all[i] = i;
    // GMRES-IR, the learned selector and double-double residuals run problem by problem
    if (o.refine == MPIR_GMRES || o.refine == MPIR_GMRES_LEFT || o.fact == MPIR_AUTO || o.resid_dd)
        return lse_solve_each(h, all, m, n, p, A, lda, B, ldb, b, d, x, o, infos, 0);
    std::vector<BInst> insts(count);
    for (int i = 0; i < count; i++)
        insts[i] = BInst{A[i], B[i], b[i], d[i], x[i], nullptr, m[i], n[i], p[i], lda[i], std::max(ldb[i], 1),
                         BKIND_LSE};
    std::vector<int> redo;
    int worst = batched_core(h, count, insts, o, infos, redo);
    if (worst < 0) return worst;
    if (!redo.empty()) {
        // escalation: re-solve with an FP64 factorization
        mpir_opts o64 = o;
        o64.fact = MPIR_FP64;
        const int st = lse_solve_each(h, redo, m, n, p, A, lda, B, ldb, b, d, x, o64, infos, 1);
        if (st < 0) return st;
        worst = std::max(worst, st);
    }
    return worst;
}

static int gls_solve_each(mpir_handle h, const std::vector<int> &which, const int *n, const int *m, const int *p,
                          const double *const *W, const int *ldw, const double *const *V, const int *ldv,
                          const double *const *d, double *const *x, double *const *y, const mpir_opts &o,
                          mpir_info *infos, int esc_base)
{
    int worst = 0;
    for (int i : which) {
        mpir_info inf;
        int st = gls_solve(h, n[i], m[i], p[i], W[i], ldw[i], V[i], ldv[i], d[i], x[i], y[i], nullptr, &o, &inf);
        if (st < 0) return st;
        inf.escalated += esc_base;
        if (infos) infos[i] = inf;
        worst = std::max(worst, st);
    }
    return worst;
}

int gls_solve_batched(mpir_handle h, int count, const int *n, const int *m, const int *p,
                      const double *const *W, const int *ldw, const double *const *V, const int *ldv,
                      const double *const *d, double *const *x, double *const *y, const mpir_opts *opts,
                      mpir_info *infos)
{
    if (!h) return -1;
    if (count < 0) return -2;
    if (count == 0) return 0;
    if (!n) return -3;
    if (!m) return -4;
    if (!p) return -5;
    if (!W) return -6;
    if (!ldw) return -7;
    if (!V) return -8;
    if (!ldv) return -9;
    if (!d) return -10;
    if (!x) return -11;
    if (!y) return -12;
    for (int i = 0; i < count; i++) {
        const int a = gls_check_args(n[i], m[i], p[i], W[i], ldw[i], V[i], ldv[i], d[i], x[i], y[i]);
        if (a) {
            char msg[96];
            std::snprintf(msg, sizeof(msg), "problem %d: illegal argument %d of gls_solve", i, -a);
            return set_err(h, -3, msg);
        }
    }
    mpir_opts o;
    fill_opts(opts, &o);
    if (infos) std::memset(infos, 0, sizeof(mpir_info) * count);
    std::vector<int> all(count);
    for (int i = 0; i < count; i++) all[i] = i;
    if (o.refine == MPIR_GMRES || o.refine == MPIR_GMRES_LEFT || o.fact == MPIR_AUTO || o.resid_dd)
        return gls_solve_each(h, all, n, m, p, W, ldw, V, ldv, d, x, y, o, infos, 0);
    std::vector<BInst> insts(count);
    for (int i = 0; i < count; i++)
        insts[i] = BInst{W[i], V[i], nullptr, d[i], x[i], y[i], m[i], n[i], p[i], std::max(ldw[i], 1),
                         std::max(ldv[i], 1), BKIND_GLS};
    std::vector<int> redo;
    int worst = batched_core(h, count, insts, o, infos, redo);
    if (worst < 0) return worst;
    if (!redo.empty()) {
        mpir_opts o64 = o;
        o64.fact = MPIR_FP64;
        const int st = gls_solve_each(h, redo, n, m, p, W, ldw, V, ldv, d, x, y, o64, infos, 1);
        if (st < 0) return st;
        worst = std::max(worst, st);
    }
    return worst;
}

// ------------------------------------------------------- step-level API --

int mpir_larfb(mpir_handle h, int prec, int M, int N, int K, const float *V, int ldv, const float *T, int trans,
               float *C, int ldc)
{
    if (!h) return -1;
    if (prec != MPIR_FP32 && prec != MPIR_TF32 && prec != MPIR_BF16) return -2;
    if (M < 0) return -3;
    if (N < 0) return -4;
    if (K < 0 || K > OUTER_NB || K > M) return -5;
    if (!V && K > 0) return -6;
    if (ldv < std::max(1, M)) return -7;
    if (!T && K > 0) return -8;
    if (!C && M * N > 0) return -10;
    if (ldc < std::max(1, M) || ldc % 4) return -11;
    RC(ensure_ws(h, geqrf_ws_bytes(M, N)));
    h->fs.kind = Kind::NONE;             // the workspace holding any factors is used as scratch
    clear_dev_flags(h);
    RC(larfb_tc(V, ldv, M, K, T, trans, C, ldc, N, gemm_prec(prec), h->ws, h->sc.err, h->stream));
    RC(cuda_check(h, "mpir_larfb"));
    return check_dev_flags(h);
}

int mpir_lse_factor(mpir_handle h, int m, int n, int p, const double *A, int lda, const double *B, int ldb,
                    int fact)
{
    if (!h) return -1;
    if (m < 0) return -2;
    if (n < 1) return -3;
    if (p < 0 || p > n || n > m + p) return -4;
    if (!A) return -5;
    if (lda < std::max(1, m)) return -6;
    if (p > 0 && !B) return -7;
    if (ldb < std::max(1, p)) return -8;
    if (fact < MPIR_BF16 || fact > MPIR_FP64) return -9;
    int rc = is_fp64(fact) ? lse_factor_impl<double>(h, m, n, p, A, lda, B, ldb, fact)
                           : lse_factor_impl<float>(h, m, n, p, A, lda, B, ldb, fact);
    if (rc) return rc;
    return check_dev_flags(h);
}

int mpir_gls_factor(mpir_handle h, int n, int m, int p, const double *W, int ldw, const double *V, int ldv,
                    int fact)
{
    if (!h) return -1;
    if (n < 1) return -2;
    if (m < 0 || m > n) return -3;
    if (p < 0 || n > m + p) return -4;
    if (!W && m > 0) return -5;
    if (ldw < std::max(1, n)) return -6;
    if (!V && p > 0) return -7;
    if (ldv < std::max(1, n)) return -8;
    if (fact < MPIR_BF16 || fact > MPIR_FP64) return -9;
    int rc = is_fp64(fact) ? gls_factor_impl<double>(h, n, m, p, W, ldw, V, ldv, fact)
                           : gls_factor_impl<float>(h, n, m, p, W, ldw, V, ldv, fact);
    if (rc) return rc;
    return check_dev_flags(h);
}

#define DISPATCH(kind_, call64, call32)                                                        \
    do {                                                                                       \
        if (!h) return -1;                                                                     \
        if (h->fs.kind != kind_) return set_err(h, MPIR_UNSUPPORTED, "no matching factors");   \
        int _rc = is_fp64(h->fs.fact) ? (call64) : (call32);                                   \
        if (_rc) return _rc;                                                                   \
        return check_dev_flags(h);                                                             \
    } while (0)

int mpir_lse_initial(mpir_handle h, const double *b, const double *d, double *x)
{
    DISPATCH(Kind::LSE, lse_initial_impl<double>(h, b, d, x), lse_initial_impl<float>(h, b, d, x));
}

int mpir_gls_initial(mpir_handle h, const double *d, double *x, double *y)
{
    DISPATCH(Kind::GLS, gls_initial_impl<double>(h, d, x, y), gls_initial_impl<float>(h, d, x, y));
}

int mpir_lse_multipliers(mpir_handle h, const double *A, int lda, const double *b, const double *x, double *r,
                         double *v)
{
    DISPATCH(Kind::LSE, lse_multipliers_impl<double>(h, A, lda, b, x, r, v),
             lse_multipliers_impl<float>(h, A, lda, b, x, r, v));
}

int mpir_gls_multipliers(mpir_handle h, const double *y, double *z)
{
    DISPATCH(Kind::GLS, gls_multipliers_impl<double>(h, y, z), gls_multipliers_impl<float>(h, y, z));
}

} // extern "C"

template <typename T>
static int lse_corr_api(mpir_ctx *h, const double *f1, const double *f2, const double *f3, double *dr,
                        double *dv, double *dx)
{
    const FactorState &fs = h->fs;
    cudaStream_t s = h->stream;
    vzero(dr, sizeof(double) * fs.m, s);
    vzero(dv, sizeof(double) * fs.p, s);
    vzero(dx, sizeof(double) * fs.n, s);
    return lse_correction_impl<T>(h, f1, f2, f3, 1.0, dr, dv, dx);
}

extern "C" {

} // extern "C"

template <typename T>
static int gls_corr_api(mpir_ctx *h, const double *f1, const double *f2, const double *f3, double *dy,
                        double *dz, double *dx)
{
    const FactorState &fs = h->fs;
    cudaStream_t s = h->stream;
    vzero(dy, sizeof(double) * fs.p, s);
    vzero(dz, sizeof(double) * fs.n, s);
    vzero(dx, sizeof(double) * fs.m, s);
    return gls_correction_impl<T>(h, f1, f2, f3, 1.0, dy, dz, dx);
}

extern "C" {

int mpir_lse_correction(mpir_handle h, const double *f1, const double *f2, const double *f3, double *dr,
                        double *dv, double *dx)
{
    DISPATCH(Kind::LSE, lse_corr_api<double>(h, f1, f2, f3, dr, dv, dx),
             lse_corr_api<float>(h, f1, f2, f3, dr, dv, dx));
}

int mpir_gls_correction(mpir_handle h, const double *f1, const double *f2, const double *f3, double *dy,
                        double *dz, double *dx)
{
    DISPATCH(Kind::GLS, gls_corr_api<double>(h, f1, f2, f3, dy, dz, dx),
             gls_corr_api<float>(h, f1, f2, f3, dy, dz, dx));
}

int mpir_lse_residual(mpir_handle h, int m, int n, int p, const double *A, int lda, const double *B, int ldb,
                      const double *b, const double *d, const double *x, const double *r, const double *v,
                      double *f1, double *f2, double *f3, double *norms)
{
    if (!h) return -1;
    if (m < 0) return -2;
    if (n < 1) return -3;
    if (p < 0 || p > n || n > m + p) return -4;
    if (!A || lda < std::max(1, m)) return -6;
    if ((p > 0 && !B) || ldb < std::max(1, p)) return -8;
    size_t bytes = 0;
    res_layout(nullptr, m, n, p, n, &bytes);
    RC(ensure_rws(h, bytes));
    ResWs w = res_layout(h->rws, m, n, p, n, nullptr);
    cudaStream_t s = h->stream;
    dual_gemv(A, lda, m, n, x, r, w.pA1, w.pA2, s);
    if (p > 0) dual_gemv(B, ldb, p, n, x, v, w.pB1, w.pB2, s);
    lse_resid_finalize(m, n, p, b, d, x, r, v, w.pA1, w.pa.ncb, w.pA2, w.pa.nrb, w.pB1, w.pb.ncb, w.pB2,
                       p > 0 ? w.pb.nrb : 0, f1, f2, f3, w.normpart, w.norms2, s);
    if (norms) {
        absmax_sumsq(A, lda, m, n, w.part, w.scal, s);
        absmax_sumsq(B, ldb, p, n, w.part, w.scal + 2, s);
        cudaMemcpyAsync(w.scal + 4, w.norms2, 6 * sizeof(double), cudaMemcpyDeviceToDevice, s);
        RC(read_back(h, w.scal, 10));
        for (int i = 0; i < 6; i++) norms[i] = std::sqrt(h->hbuf[4 + i]);
        norms[6] = std::sqrt(h->hbuf[1]);
        norms[7] = std::sqrt(h->hbuf[3]);
    }
    return cuda_check(h, "lse_residual");
}

int mpir_gls_residual(mpir_handle h, int n, int m, int p, const double *W, int ldw, const double *V, int ldv,
                      const double *d, const double *x, const double *y, const double *z, double *f1,
                      double *f2, double *f3, double *norms)
{
    if (!h) return -1;
    if (n < 1) return -2;
    if (m < 0 || m > n) return -3;
    if (p < 0 || n > m + p) return -4;
    if ((m > 0 && !W) || ldw < std::max(1, n)) return -6;
    if ((p > 0 && !V) || ldv < std::max(1, n)) return -8;
    size_t bytes = 0;
    res_layout(nullptr, n, m, n, p, &bytes);
    RC(ensure_rws(h, bytes));
    ResWs w = res_layout(h->rws, n, m, n, p, nullptr);
    cudaStream_t s = h->stream;
    dual_gemv(W, ldw, n, m, x, z, w.pA1, w.pA2, s);
    dual_gemv(V, ldv, n, p, y, z, w.pB1, w.pB2, s);
    gls_resid_finalize(n, m, p, d, x, y, z, w.pA1, w.pa.ncb, w.pA2, w.pa.nrb, w.pB1, w.pb.ncb, w.pB2,
                       w.pb.nrb, f1, f2, f3, w.normpart, w.norms2, s);
    if (norms) {
        absmax_sumsq(W, ldw, n, m, w.part, w.scal, s);
        absmax_sumsq(V, ldv, n, p, w.part, w.scal + 2, s);
        cudaMemcpyAsync(w.scal + 4, w.norms2, 6 * sizeof(double), cudaMemcpyDeviceToDevice, s);
        RC(read_back(h, w.scal, 10));
        for (int i = 0; i < 6; i++) norms[i] = std::sqrt(h->hbuf[4 + i]);
        norms[6] = std::sqrt(h->hbuf[1]);
        norms[7] = std::sqrt(h->hbuf[3]);
    }
    return cuda_check(h, "gls_residual");
}

} // extern "C"

template <typename T>
static int get_RT_impl(mpir_ctx *h, double *R, int ldr, double *Tm, int ldt)
{
    const FactorState &fs = h->fs;
    cudaStream_t s = h->stream;
    if (fs.kind == Kind::LSE) {
        LseWs<T> w = lse_layout<T>(h->ws, fs.m, fs.n, fs.p, nullptr);
        const int m = w.m, n = w.n, p = w.p;
        if (R && p > 0) {
            // R(i, j) = R~(p-1-j, p-1-i) = Bt(p-1-j, p-1-i) / sB
            mconvert<T, double>(w.Bt, w.ldBt, R, ldr, p, p, 1, 1, 1, 1.0 / fs.s2, s);
            { ProfScope ps(K_ELEMWISE, s); k_mask_lower<<<dim3(ceil_div(p, 256), p), 256, 0, s>>>(R, ldr, p, p, 0); }
        }
        if (Tm) {
            mconvert<T, double>(w.At, w.ldAt, Tm, ldt, m, n, 0, 0, 0, 1.0 / fs.s1, s);
            { ProfScope ps(K_ELEMWISE, s); k_mask_lower<<<dim3(ceil_div(m, 256), n), 256, 0, s>>>(Tm, ldt, m, n, 0); }
        }
    } else {
        GlsWs<T> w = gls_layout<T>(h->ws, fs.n, fs.m, fs.p, nullptr);
        const int n = w.n, m = w.m, p = w.p;
        if (R && m > 0) {
            mconvert<T, double>(w.Wf, w.ldW, R, ldr, m, m, 0, 0, 0, 1.0 / fs.s1, s);
            { ProfScope ps(K_ELEMWISE, s); k_mask_lower<<<dim3(ceil_div(m, 256), m), 256, 0, s>>>(R, ldr, m, m, 0); }
        }
        if (Tm) {
            // T(r, j) = T~(p-1-j, n-1-r) = Ct(p-1-j, n-1-r) / sV ; zero for r > j + n - p
            mconvert<T, double>(w.Ct, w.ldCt, Tm, ldt, n, p, 1, 1, 1, 1.0 / fs.s2, s);
            { ProfScope ps(K_ELEMWISE, s); k_mask_lower<<<dim3(ceil_div(n, 256), p), 256, 0, s>>>(Tm, ldt, n, p, n - p); }
        }
    }
    return cuda_check(h, "get_RT");
}

extern "C" {

int mpir_get_RT(mpir_handle h, double *R, int ldr, double *T, int ldt)
{
    if (!h) return -1;
    if (h->fs.kind == Kind::NONE) return set_err(h, MPIR_UNSUPPORTED, "no factors held");
    int rc = is_fp64(h->fs.fact) ? get_RT_impl<double>(h, R, ldr, T, ldt) : get_RT_impl<float>(h, R, ldr, T, ldt);
    if (rc) return rc;
    return cudaStreamSynchronize(h->stream) == cudaSuccess ? 0 : cuda_check(h, "get_RT");
}

} // extern "C"

template <typename T>
static int apply_factor_impl(mpir_ctx *h, int which, int trans, double *vec)
{
    const FactorState &fs = h->fs;
    cudaStream_t s = h->stream;
    if (fs.kind == Kind::LSE) {
        LseWs<T> w = lse_layout<T>(h->ws, fs.m, fs.n, fs.p, nullptr);
        if (which == 0) {
            // Q = P_n Q~^T P_n ; Q^T = P_n Q~ P_n
            const int n = w.n;
            vcopy<double, T>(vec, w.tt, n, 1.0, 1, s);
            RC(vapply<T>(w.Bt, w.ldBt, n, w.p, w.TwB, w.Tw128B, w.TfB, w.ldtB, w.wy, trans ? 0 : 1, w.tt, h->sc, s));
            vcopy<T, double>(w.tt, vec, n, 1.0, 1, s);
        } else {
            const int m = w.m;
            vcopy<double, T>(vec, w.tt, m, 1.0, 0, s);
            RC(vapply<T>(w.At, w.ldAt, m, w.kA, w.TwA, w.Tw128A, w.TfA, w.ldtA, w.wy, trans, w.tt, h->sc, s));
            vcopy<T, double>(w.tt, vec, m, 1.0, 0, s);
        }
    } else {
        GlsWs<T> w = gls_layout<T>(h->ws, fs.n, fs.m, fs.p, nullptr);
        if (which == 0) {
            const int n = w.n;
            vcopy<double, T>(vec, w.tt, n, 1.0, 0, s);
            RC(vapply<T>(w.Wf, w.ldW, n, w.m, w.TwW, w.Tw128W, w.TfW, w.ldtW, w.wy, trans, w.tt, h->sc, s));
            vcopy<T, double>(w.tt, vec, n, 1.0, 0, s);
        } else {
            // Z = P_p Z~^T P_p ; Z^T = P_p Z~ P_p
            const int p = w.p;
            vcopy<double, T>(vec, w.tt, p, 1.0, 1, s);
            RC(vapply<T>(w.Ct, w.ldCt, p, w.kC, w.TwC, w.Tw128C, w.TfC, w.ldtC, w.wy, trans ? 0 : 1, w.tt, h->sc, s));
            vcopy<T, double>(w.tt, vec, p, 1.0, 1, s);
        }
    }
    return cuda_check(h, "apply_factor");
}

extern "C" {

int mpir_apply_factor(mpir_handle h, int which, int trans, double *vec)
{
    if (!h) return -1;
    if (h->fs.kind == Kind::NONE) return set_err(h, MPIR_UNSUPPORTED, "no factors held");
    if (which != 0 && which != 1) return -2;
    if (!vec) return -4;
    int rc = is_fp64(h->fs.fact) ? apply_factor_impl<double>(h, which, trans, vec)
                                 : apply_factor_impl<float>(h, which, trans, vec);
    if (rc) return rc;
    return check_dev_flags(h);
}

} // extern "C"

// --------------------------------------- GMRES-IR operator (step level) --
template <typename Op>
static int bd_dispatch(Op &op, int which, const double *in, double *out, BDScratch &b)
{
    switch (which) {
    case 0: return op.Fmul(in, out);
    case 1: return op.Ml(in, out);
    case 2: return op.Mr(in, out);
    default: return op.apply(in, out);
    }
}

template <typename T>
static int lse_bd_apply_impl(mpir_ctx *h, const double *A, int lda, const double *B, int ldb, double al,
                             double be, int which, const double *in, double *out)
{
    const FactorState &fs = h->fs;
    const int N = fs.m + fs.p + fs.n, mx = std::max(std::max(fs.m, fs.n), std::max(fs.p, 1));
    RC(ensure_rws(h, bd_bytes(N, 1, mx)));
    BDScratch b = bd_layout(h->rws, N, 1, mx);
    LseWs<T> w = lse_layout<T>(h->ws, fs.m, fs.n, fs.p, nullptr);
    if (which >= 4) {           // left preconditioner (Sec. 5.1)
        LseLeftOp<T> op(h, w, b, A, lda, B, ldb, al, be);
        RC(which == 4 ? op.Ml(in, out) : op.apply(in, out));
        return cuda_check(h, "lse_bd_apply");
    }
    LseBDOp<T> op(h, w, b, A, lda, B, ldb, al, be);
    op.prepare();
    RC(bd_dispatch(op, which, in, out, b));
    return cuda_check(h, "lse_bd_apply");
}

template <typename T>
static int gls_bd_apply_impl(mpir_ctx *h, const double *W, int ldw, const double *V, int ldv, double al,
                             double be, int which, const double *in, double *out)
{
    const FactorState &fs = h->fs;
    const int N = fs.p + fs.n + fs.m, mx = std::max(std::max(fs.m, fs.n), std::max(fs.p, 1));
    RC(ensure_rws(h, bd_bytes(N, 1, mx)));
    BDScratch b = bd_layout(h->rws, N, 1, mx);
    GlsWs<T> w = gls_layout<T>(h->ws, fs.n, fs.m, fs.p, nullptr);
    if (which >= 4) {           // left preconditioner (Sec. 5.1)
        GlsLeftOp<T> op(h, w, b, W, ldw, V, ldv, al, be);
        RC(which == 4 ? op.Ml(in, out) : op.apply(in, out));
        return cuda_check(h, "gls_bd_apply");
    }
    GlsBDOp<T> op(h, w, b, W, ldw, V, ldv, al, be);
    op.prepare();
    RC(bd_dispatch(op, which, in, out, b));
    return cuda_check(h, "gls_bd_apply");
}

extern "C" {

int mpir_lse_bd_apply(mpir_handle h, const double *A, int lda, const double *B, int ldb, double alpha,
                      double beta, int which, const double *in, double *out)
{
    if (!h) return -1;
    const FactorState &fs = h->fs;
    if (fs.kind != Kind::LSE) return set_err(h, MPIR_UNSUPPORTED, "no LSE factors held");
    if (!A) return -2;
    if (lda < std::max(1, fs.m)) return -3;
    if (fs.p > 0 && !B) return -4;
    if (ldb < std::max(1, fs.p)) return -5;
    if (!(alpha > 0) || !std::isfinite(alpha)) return -6;
    if (!(beta > 0) || !std::isfinite(beta)) return -7;
    if (which < 0 || which > 5) return -8;
    if (!in) return -9;
    if (!out || out == in) return -10;
    clear_dev_flags(h);
    int rc = is_fp64(fs.fact) ? lse_bd_apply_impl<double>(h, A, lda, B, ldb, alpha, beta, which, in, out)
                              : lse_bd_apply_impl<float>(h, A, lda, B, ldb, alpha, beta, which, in, out);
    if (rc) return rc;
    return check_dev_flags(h);
}

int mpir_gls_bd_apply(mpir_handle h, const double *W, int ldw, const double *V, int ldv, double alpha,
                      double beta, int which, const double *in, double *out)
{
    if (!h) return -1;
    const FactorState &fs = h->fs;
    if (fs.kind != Kind::GLS) return set_err(h, MPIR_UNSUPPORTED, "no GLS factors held");
    if (fs.m > 0 && !W) return -2;
    if (ldw < std::max(1, fs.n)) return -3;
    if (!V) return -4;
    if (ldv < std::max(1, fs.n)) return -5;
    if (!(alpha > 0) || !std::isfinite(alpha)) return -6;
    if (!(beta > 0) || !std::isfinite(beta)) return -7;
    if (which < 0 || which > 5) return -8;
    if (!in) return -9;
    if (!out || out == in) return -10;
    clear_dev_flags(h);
    int rc = is_fp64(fs.fact) ? gls_bd_apply_impl<double>(h, W, ldw, V, ldv, alpha, beta, which, in, out)
                              : gls_bd_apply_impl<float>(h, W, ldw, V, ldv, alpha, beta, which, in, out);
    if (rc) return rc;
    return check_dev_flags(h);
}

} // extern "C"

extern "C" {

// Complex batches through the real embedding (complex.cu): every problem's
// E(A), E(B), e(b), e(d) and e(x) in the handle's embedding buffer, one
// embedding launch, the real batched solve, one read-back launch.
int zlse_solve_batched(mpir_handle h, int count, const int *m, const int *n, const int *p,
                       const double *const *A, const int *lda, const double *const *B, const int *ldb,
                       const double *const *b, const double *const *d, double *const *x,
                       const mpir_opts *opts, mpir_info *infos)
{
    if (!h) return -1;
    if (count < 0) return -2;
    if (count == 0) return 0;
    if (!m || !n || !p || !A || !lda || !B || !ldb || !b || !d || !x) return -3;
    for (int i = 0; i < count; i++) {
        const int a = lse_check_args(m[i], n[i], p[i], A[i], lda[i], B[i], ldb[i], b[i], d[i], x[i]);
        if (a) {
            char msg[96];
            std::snprintf(msg, sizeof(msg), "problem %d: illegal argument %d of zlse_solve", i, -a);
            return set_err(h, -3, msg);
        }
    }
    std::vector<size_t> off(count + 1, 0);
    for (int i = 0; i < count; i++) {
        const size_t M = 2 * (size_t)m[i], N = 2 * (size_t)n[i], P = 2 * (size_t)p[i];
        off[i + 1] = off[i] + ((M * N + P * N + M + P + N + 31) & ~(size_t)31);
    }
    const size_t njobs_max = (size_t)5 * count;
    const size_t table_words = (njobs_max * sizeof(ZEmbedJob) + 7) / 8;
    RC(ensure_zbuf(h, sizeof(double) * (off[count] + table_words)));
    double *base = h->zbuf;
    ZEmbedJob *table = reinterpret_cast<ZEmbedJob *>(base + off[count]);
    std::vector<int> M2(count), N2(count), P2(count), lda2(count), ldb2(count);
    std::vector<const double *> Ah(count), Bh(count), bh(count), dh(count);
    std::vector<double *> xh(count);
    std::vector<ZEmbedJob> jobs, back;
    for (int i = 0; i < count; i++) {
        M2[i] = 2 * m[i]; N2[i] = 2 * n[i]; P2[i] = 2 * p[i];
        lda2[i] = std::max(M2[i], 1); ldb2[i] = std::max(P2[i], 1);
        double *q = base + off[i];
        double *a_ = q, *b_ = a_ + (size_t)M2[i] * N2[i], *bv = b_ + (size_t)P2[i] * N2[i], *dv = bv + M2[i];
        double *xv = dv + P2[i];
        Ah[i] = a_; Bh[i] = p[i] > 0 ? b_ : nullptr; bh[i] = bv; dh[i] = p[i] > 0 ? dv : nullptr; xh[i] = xv;
        if (m[i] > 0) {
            jobs.push_back(ZEmbedJob{A[i], a_, m[i], n[i], lda[i], lda2[i], 0});
            jobs.push_back(ZEmbedJob{b[i], bv, m[i], 1, std::max(m[i], 1), M2[i], 1});
        }
        if (p[i] > 0) {
            jobs.push_back(ZEmbedJob{B[i], b_, p[i], n[i], ldb[i], ldb2[i], 0});
            jobs.push_back(ZEmbedJob{d[i], dv, p[i], 1, std::max(p[i], 1), P2[i], 1});
        }
        back.push_back(ZEmbedJob{x[i], xv, n[i], 1, n[i], N2[i], 1});
    }
    cudaStream_t s = h->stream;
    if (cudaMemcpyAsync(table, jobs.data(), sizeof(ZEmbedJob) * jobs.size(), cudaMemcpyHostToDevice, s) !=
        cudaSuccess)
        return cuda_check(h, "zlse_solve_batched");
    RC(zembed_batch(table, (int)jobs.size(), 0, s));
    const int st = lse_solve_batched(h, count, M2.data(), N2.data(), P2.data(), Ah.data(), lda2.data(), Bh.data(),
                                     ldb2.data(), bh.data(), dh.data(), xh.data(), opts, infos);
    if (st < 0 || st == MPIR_CUDA_ERROR) return st;
    if (cudaMemcpyAsync(table, back.data(), sizeof(ZEmbedJob) * back.size(), cudaMemcpyHostToDevice, s) !=
        cudaSuccess)
        return cuda_check(h, "zlse_solve_batched");
    RC(zembed_batch(table, (int)back.size(), 1, s));
    if (cudaStreamSynchronize(s) != cudaSuccess) return cuda_check(h, "zlse_solve_batched");
    return st;
}

int zgls_solve_batched(mpir_handle h, int count, const int *n, const int *m, const int *p,
                       const double *const *W, const int *ldw, const double *const *V, const int *ldv,
                       const double *const *d, double *const *x, double *const *y, const mpir_opts *opts,
                       mpir_info *infos)
{
    if (!h) return -1;
    if (count < 0) return -2;
    if (count == 0) return 0;
    if (!n || !m || !p || !W || !ldw || !V || !ldv || !d || !x || !y) return -3;
    for (int i = 0; i < count; i++) {
        const int a = gls_check_args(n[i], m[i], p[i], W[i], ldw[i], V[i], ldv[i], d[i], x[i], y[i]);
        if (a) {
            char msg[96];
            std::snprintf(msg, sizeof(msg), "problem %d: illegal argument %d of zgls_solve", i, -a);
            return set_err(h, -3, msg);
        }
    }
    std::vector<size_t> off(count + 1, 0);
    for (int i = 0; i < count; i++) {
        const size_t Nn = 2 * (size_t)n[i], M = 2 * (size_t)m[i], P = 2 * (size_t)p[i];
        off[i + 1] = off[i] + ((Nn * M + Nn * P + Nn + M + P + 31) & ~(size_t)31);
    }
    const size_t njobs_max = (size_t)5 * count;
    const size_t table_words = (njobs_max * sizeof(ZEmbedJob) + 7) / 8;
    RC(ensure_zbuf(h, sizeof(double) * (off[count] + table_words)));
    double *base = h->zbuf;
    ZEmbedJob *table = reinterpret_cast<ZEmbedJob *>(base + off[count]);
    std::vector<int> N2(count), M2(count), P2(count), ldn(count);
    std::vector<const double *> Wh(count), Vh(count), dh(count);
    std::vector<double *> xh(count), yh(count);
    std::vector<ZEmbedJob> jobs, back;
    for (int i = 0; i < count; i++) {
        N2[i] = 2 * n[i]; M2[i] = 2 * m[i]; P2[i] = 2 * p[i];
        ldn[i] = N2[i];
        double *q = base + off[i];
        double *w_ = q, *v_ = w_ + (size_t)N2[i] * M2[i], *dv = v_ + (size_t)N2[i] * P2[i], *xv = dv + N2[i];
        double *yv = xv + M2[i];
        Wh[i] = m[i] > 0 ? w_ : nullptr; Vh[i] = v_; dh[i] = dv; xh[i] = m[i] > 0 ? xv : nullptr;
        yh[i] = p[i] > 0 ? yv : nullptr;
        if (m[i] > 0) jobs.push_back(ZEmbedJob{W[i], w_, n[i], m[i], ldw[i], N2[i], 0});
        if (p[i] > 0) jobs.push_back(ZEmbedJob{V[i], v_, n[i], p[i], ldv[i], N2[i], 0});
        jobs.push_back(ZEmbedJob{d[i], dv, n[i], 1, n[i], N2[i], 1});
        if (m[i] > 0) back.push_back(ZEmbedJob{x[i], xv, m[i], 1, m[i], M2[i], 1});
        if (p[i] > 0) back.push_back(ZEmbedJob{y[i], yv, p[i], 1, p[i], P2[i], 1});
    }
    cudaStream_t s = h->stream;
    if (cudaMemcpyAsync(table, jobs.data(), sizeof(ZEmbedJob) * jobs.size(), cudaMemcpyHostToDevice, s) !=
        cudaSuccess)
        return cuda_check(h, "zgls_solve_batched");
    RC(zembed_batch(table, (int)jobs.size(), 0, s));
    const int st = gls_solve_batched(h, count, N2.data(), M2.data(), P2.data(), Wh.data(), ldn.data(), Vh.data(),
                                     ldn.data(), dh.data(), xh.data(), yh.data(), opts, infos);
    if (st < 0 || st == MPIR_CUDA_ERROR) return st;
    if (!back.empty()) {
        if (cudaMemcpyAsync(table, back.data(), sizeof(ZEmbedJob) * back.size(), cudaMemcpyHostToDevice, s) !=
            cudaSuccess)
            return cuda_check(h, "zgls_solve_batched");
        RC(zembed_batch(table, (int)back.size(), 1, s));
    }
    if (cudaStreamSynchronize(s) != cudaSuccess) return cuda_check(h, "zgls_solve_batched");
    return st;
}

int mpir_batched_set_shape(mpir_handle h, int group)
{
    if (!h) return -1;
    if (group != 0 && group != 512 && group != 256 && group != 128 && group != 64) return -2;
    h->ba.force_group = group;
    return 0;
}

int mpir_batched_get_shape(mpir_handle h, int bucket, int *group, size_t *smem_bytes, int *problems)
{
    if (!h) return -1;
    if (bucket < 0 || bucket > 1) return -2;
    if (group) *group = h->ba.last[bucket].group;
    if (smem_bytes) *smem_bytes = h->ba.last[bucket].smem;
    if (problems) *problems = h->ba.last_count[bucket];
    return 0;
}

} // extern "C"

extern "C" {

int mpir_lse_features(mpir_handle h, int m, int n, int p, const double *A, int lda, const double *B, int ldb,
                      const double *b, const double *d, const double *s, float *features)
{
    if (!h) return -1;
    if (m < 1) return -2;
    if (n < 1) return -3;
    if (p < 0) return -4;
    if (!A || lda < m) return -5;
    if ((p > 0 && !B) || ldb < std::max(1, p)) return -7;
    if (!b) return -9;
    if (p > 0 && !d) return -10;
    if (!s) return -11;
    if (!features) return -12;
    RC(ensure_rws(h, sizeof(double) * features_ws_doubles(m + p, n)));
    RC(features_launch(0, m, n, p, A, lda, B, std::max(ldb, 1), s, b, m, d, p, 16, (double *)h->rws, features,
                       h->stream));
    return cuda_check(h, "mpir_lse_features");
}

int mpir_gls_features(mpir_handle h, int n, int m, int p, const double *W, int ldw, const double *V, int ldv,
                      const double *d, const double *s, float *features)
{
    if (!h) return -1;
    if (n < 1) return -2;
    if (m < 0) return -3;
    if (p < 1) return -4;
    if ((m > 0 && !W) || ldw < n) return -5;
    if (!V || ldv < n) return -7;
    if (!d) return -9;
    if (!s) return -10;
    if (!features) return -11;
    RC(ensure_rws(h, sizeof(double) * features_ws_doubles(n, m + p)));
    RC(features_launch(1, m, n, p, W, std::max(ldw, 1), V, ldv, s, d, n, nullptr, 0, 16, (double *)h->rws, features,
                       h->stream));
    return cuda_check(h, "mpir_gls_features");
}

int mpir_mlp_param_count(void) { return MLP_PARAMS; }

int mpir_mlp_forward(mpir_handle h, const float *params, const float *X, int count, float *prob)
{
    if (!h) return -1;
    if (!params) return -2;
    if (!X && count > 0) return -3;
    if (count < 0) return -4;
    if (!prob && count > 0) return -5;
    RC(mlp_forward(params, X, count, prob, h->stream));
    return cuda_check(h, "mpir_mlp_forward");
}

int mpir_mlp_train_step(mpir_handle h, float *params, float *adam_m, float *adam_v, int step, float lr,
                        const float *X, const int *labels, int count, float *grad, float *loss)
{
    if (!h) return -1;
    if (!params) return -2;
    if (step < 1) return -5;
    if (!X) return -7;
    if (!labels) return -8;
    if (count < 1) return -9;
    RC(ensure_rws(h, sizeof(float) * mlp_ws_floats(count)));
    RC(mlp_train_step(params, adam_m, adam_v, step, lr, X, labels, count, (float *)h->rws, grad, loss, h->stream));
    return cuda_check(h, "mpir_mlp_train_step");
}

int mpir_selector_set(mpir_handle h, const float *params, const float *mean, const float *scale)
{
    if (!h) return -1;
    if (!params) {
        if (h->sel) { cudaStreamSynchronize(h->stream); cudaFree(h->sel); h->sel = nullptr; }
        return 0;
    }
    if (!mean) return -3;
    if (!scale) return -4;
    for (int q = 0; q < 16; q++) if (!(scale[q] != 0.0f)) return -4;
    if (!h->sel && cudaMalloc(&h->sel, sizeof(float) * (MLP_PARAMS + 64)) != cudaSuccess) {
        cudaGetLastError();
        return set_err(h, MPIR_CUDA_ERROR, "selector: cudaMalloc failed");
    }
    cudaMemcpy(h->sel, params, sizeof(float) * MLP_PARAMS, cudaMemcpyHostToDevice);
    std::memcpy(h->sel_mean, mean, sizeof(h->sel_mean));
    std::memcpy(h->sel_scale, scale, sizeof(h->sel_scale));
    return cuda_check(h, "mpir_selector_set");
}

} // extern "C"
