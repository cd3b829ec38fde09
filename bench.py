#!/usr/bin/env python3
"""Benchmark: solves/s of the mixed-precision LSE solve (FP32 GRQ + FP64
classical iterative refinement, Alg. 2) on one GB300, next to the plain
FP64 GRQ solve on the same GPU and the CPU oracle on the host cores.

Workload (one "step" = one complete solve, factorization included):
  LSE min ||A x - b|| s.t. B x = d, m = 16384, n = 8192, p = 1024:
  A = U diag(logspace) V^T with cond(A) = 1e4, B likewise with cond(B) =
  1e2 (seeded Haar factors drawn on the GPU), right-hand sides from the
  known-solution construction (x* ~ N(0,1); r* with A^T r* = B^T v*;
  b = A x* + r*, d = B x*), so every result's forward error is measured.
The same line reports the sweep cond(A) in {1e1, 1e4, 1e8} (FP32 and TF32
factors, classical IR and GMRES-IR, FP64 direct), the GLS n = 4096 AR(1)
workload, and 10,000 uneven batched LSE problems.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Prints ONE JSON line (rank 0).  For N > 1 it is launched with torchrun; each
rank solves its own independent problem (replicas, no collective on the data
path); the time is the max over ranks.
"""
import argparse
import hashlib
import json
import os
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "solves/s at FP64-level accuracy: mixed-precision IR vs FP64 GRQ/GQR, same GB300"
M_, N_, P_ = 16384, 8192, 1024
COND_A, COND_B = 1e4, 1e2
CONDS = (1e1, 1e4, 1e8)
SEED = 20243623
WORKLOAD = ("LSE m=16384 n=8192 p=1024: A = U diag(logspace) V^T with cond(A)=1e4, B likewise with cond(B)=1e2 "
            "(seeded Haar factors), known-solution right-hand sides (b = A x* + r*, d = B x*, A^T r* = B^T v*)")
GLS_WORKLOAD = ("GLS n=4096 m=1024 p=4096 (xGGGLM shapes): W cond 1e3 SVD construction, "
                "V = Cholesky factor of AR(1) covariance rho=0.9, d = W x + V y")
GLS_N, GLS_M, GLS_SEED = 4096, 1024, 20242623
U64 = 1.1e-16
L2_FLUSH_BYTES = 256 << 20


def config(fact="fp32"):
    """The workload description both arms print (identical dicts)."""
    return {"workload": WORKLOAD, "fact": fact, "refine": "classical", "cond_a": COND_A,
            "l2": "inputs 1.14 GB FP64 > 129 MB L2 (no flush needed)"}


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--fact", default="fp32", choices=["bf16", "tf32", "fp32", "fp64"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-complex", action="store_true",
                    help="skip the complex LSE / GLS solves (zlse_solve, zgls_solve)")
    ap.add_argument("--quick", action="store_true",
                    help="time the headline solve only (for profiler runs)")
    ap.add_argument("--no-sweep", action="store_true", help="skip the cond(A) sweep")
    ap.add_argument("--no-gls", action="store_true", help="skip the GLS n=4096 workload")
    ap.add_argument("--no-paper-shapes", action="store_true", help="skip the Sec. 6.2 / 6.3 shape sweep")
    ap.add_argument("--paper-shapes-full", action="store_true",
                    help="every Sec. 6.2 / 6.3 shape and conditioning (default: the corners)")
    ap.add_argument("--paper-shapes-only", action="store_true",
                    help="run only the Sec. 6.2 / 6.3 shape sweep (prints its JSON object)")
    ap.add_argument("--batched-count", type=int, default=10000,
                    help="problems of the uneven batched LSE workload (0: skip it)")
    ap.add_argument("--batched-gls-count", type=int, default=4000,
                    help="problems of the uneven batched GLS workload (0: skip it)")
    ap.add_argument("--selector-count", type=int, default=100,
                    help="held-out LSE and GLS problems of the selector comparison (0: skip it)")
    ap.add_argument("--batched-only", action="store_true",
                    help="run only the batched LSE workload (prints its JSON object)")
    ap.add_argument("--profile-range", action="store_true",
                    help="with --quick: bracket the timed steps by cudaProfilerStart/Stop (for ncu "
                         "--profile-from-start off)")
    ap.add_argument("--size", type=int, nargs=3, metavar=("M", "N", "P"),
                    help="with --quick: another LSE shape of the same construction (small ncu captures)")
    return ap.parse_args()


def dist_env():
    return (int(os.environ.get("RANK", "0")), int(os.environ.get("WORLD_SIZE", "1")),
            int(os.environ.get("LOCAL_RANK", "0")))


def rank_max(x, world, device=None):
    """The largest x over the ranks of the process group (x when alone):
    the slowest rank sets the job's time."""
    if world <= 1:
        return float(x)
    import torch
    import torch.distributed as dist
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def nproc():
    """Host cores available to this process (what `nproc` prints)."""
    try:
        return len(os.sched_getaffinity(0))
    except AttributeError:
        return os.cpu_count()


def job_value(world, ms_per_step):
    """Whole-job throughput in solves/s: every rank solves one problem per
    step (replicas), and the step takes the slowest rank's time."""
    return world * 1000.0 / ms_per_step


# --------------------------------------------------------------- clocks --

class ClockSampler:
    """nvidia-smi sampling every 50 ms while the benchmark loads the GPU."""
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.path = None
        self.out = None

    def start(self):
        try:
            fd, self.path = tempfile.mkstemp(suffix=".csv")
            os.close(fd)
            self.out = open(self.path, "w")
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), "--query-gpu=" + self.Q, "--format=csv,noheader,nounits",
                 "-lms", "50"], stdout=self.out, stderr=subprocess.DEVNULL)
        except OSError:                       # no nvidia-smi: no clock record
            self.proc = None
            return
        # wait (at most 3 s) for the first sample, so that sampling covers
        # the work that follows
        t0 = time.time()
        while self.proc.poll() is None and time.time() - t0 < 3.0:
            if os.path.getsize(self.path) > 0:
                break
            time.sleep(0.02)

    def stop(self):
        out = {"sm_mhz": None, "sm_max_mhz": None, "reasons": [], "samples": 0}
        if self.proc is None:
            return out
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
            self.proc.wait()
        self.out.close()
        rows = []
        for line in open(self.path):
            f = [x.strip() for x in line.split(",")]
            if len(f) >= 9:
                rows.append(f)
        os.unlink(self.path)
        if not rows:
            return out
        sm = sorted(float(r[1]) for r in rows if r[1].replace(".", "").isdigit())
        out["samples"] = len(rows)
        out["sm_mhz"] = sm[len(sm) // 2] if sm else None
        try:
            out["sm_max_mhz"] = float(rows[0][2])
        except ValueError:
            pass
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = set()
        for r in rows:
            for k, nm in enumerate(names):
                if r[5 + k].lower().startswith("active"):
                    reasons.add(nm)
        out["reasons"] = sorted(reasons)
        return out


# ------------------------------------------------------- algorithmic work --

def qr_work(M, N, nb=32):
    """(panel flops, larfb flops) of the blocked Householder QR of M x N as
    the library runs it (panels of nb columns, trailing update per panel)."""
    k = min(M, N)
    pf = lf = 0.0
    for j0 in range(0, k, nb):
        nc = min(nb, N - j0)
        L = M - j0
        kb = min(nc, L)
        pf += 4.0 * L * kb * nc - 2.0 * kb * kb * nc          # panel (unblocked Householder)
        Nc = N - j0 - nc
        if Nc > 0:
            lf += 4.0 * L * kb * Nc + 2.0 * kb * kb * Nc        # V^T C, Tw^T W, C - V W
    return pf, lf


def apply_work(M, K, Nc, nb=32):
    lf = 0.0
    for j0 in range(0, K, nb):
        kb = min(nb, K - j0)
        L = M - j0
        lf += 4.0 * L * kb * Nc + 2.0 * kb * kb * Nc
    return lf


def qr_split(M, N, nb=32, outer=128):
    """(panel, inner, outer) flops of the two-level blocked QR as the
    library runs it: 32-wide panels, SIMT updates of the rest of each
    128-wide outer block (inner), tensor-core updates of the trailing
    matrix per outer block (outer)."""
    k = min(M, N)
    pf = inner = outer_f = 0.0
    for J0 in range(0, k, outer):
        no = min(outer, k - J0)
        for j0 in range(J0, J0 + no, nb):
            nc = min(nb, J0 + no - j0)
            L = M - j0
            kb = min(nc, L)
            pf += 4.0 * L * kb * nc - 2.0 * kb * kb * nc
            rest = J0 + no - j0 - nc
            if rest > 0:
                inner += 4.0 * L * kb * rest + 2.0 * kb * kb * rest
        Nc = N - J0 - no
        L = M - J0
        kb = min(no, L)
        if Nc > 0:
            outer_f += 4.0 * L * kb * Nc + 2.0 * kb * kb * Nc
    return pf, inner, outer_f


def lse_work(m, n, p):
    """Algorithmic work of one LSE solve as the library runs it: the QR of
    B~ (n x p) with Q~^T applied to the n x m X = P A^T (the RQ of B and
    A Q^T, Lemma 4.5), the QR of A Q^T (m x n); FP64 residual bytes and
    flops of one refinement step (one read of A and B, 4 (mn + pn) flops,
    t_r of Sec. 3.1)."""
    p1, i1, o1 = qr_split(n, p)
    o2 = 4.0 * n * p * m - 2.0 * p * p * m
    p3, i3, o3 = qr_split(m, n)
    return dict(panel_flops=p1 + p3, inner_flops=i1 + i3, tc_flops=o1 + o2 + o3,
                factor_flops=p1 + i1 + o1 + o2 + p3 + i3 + o3,
                resid_bytes=8.0 * (m * n + p * n), resid_flops=4.0 * (m * n + p * n))


def gls_work(n, m, p, nb=32):
    p1, l1 = qr_work(n, m, nb)
    l2 = apply_work(n, m, p, nb)
    p3, l3 = qr_work(p, n, nb)
    return dict(panel_flops=p1 + p3, larfb_flops=l1 + l2 + l3,
                factor_flops=p1 + p3 + l1 + l2 + l3,
                resid_bytes=8.0 * (n * m + n * p), resid_flops=4.0 * (m * n + n * p))


def fp32_simt_peak(sm_mhz, sms=152):
    """SMs x 128 FP32 lanes x 2 flop/FMA at the given SM clock (TFLOP/s);
    the SM count is read from the device at run time."""
    return sms * 128 * 2 * sm_mhz * 1e6 / 1e12


def tf32_peak(peaks, sustained=True):
    """Dense TF32 tensor peak: the measured BF16 cuBLAS figure (sustained:
    for a kernel timed inside a long step) times the nominal TF32 / BF16
    ratio 1.1 / 2.25."""
    bf = peaks.get("bf16_tflops_sustained" if sustained else "bf16_tflops") or peaks["bf16_tflops"]
    return bf * 1.1 / 2.25


def measured_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f)
    except (OSError, ValueError):
        return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "bf16_tflops_sustained": 1700.0,
                "sm_max_mhz": 2070.0, "_fallback": True}


def traffic_record(kind):
    """Per-launch DRAM traffic of `kind` from the committed ncu summary, if
    it was taken on the current source of the kernel (else None)."""
    try:
        with open(os.path.join(ROOT, "profiles", "traffic.json")) as f:
            rec = json.load(f)
    except (OSError, ValueError):
        return None
    r = rec.get(kind)
    if not r:
        return None
    src = os.path.join(ROOT, "paper_2406_16499_gb300", "csrc", r["source"])
    try:
        with open(src, "rb") as f:
            sha = hashlib.sha256(f.read()).hexdigest()[:16]
    except OSError:
        return None
    return r["bytes_per_launch"] if sha == r.get("source_sha") else None


# ------------------------------------------------------ batched workload --

def batch_work(m, n, p):
    """Algorithmic flops of one batched problem: the GRQ (QR of the n x p
    B~, At P_n Q~ P_n, QR of the m x n At) plus one FP64 residual."""
    kA = min(m, n)
    f = 2.0 * n * p * p - 2.0 * p ** 3 / 3.0 + 4.0 * m * n * p
    f += 2.0 * m * n * kA - 2.0 * kA ** 3 / 3.0
    return f


def run_batched(count, h, dev, stream, rank=0, sample_every=500):
    """Uneven batch of `count` LSE problems (m ~ U[32,512], n ~ U[16,m/2],
    p ~ U[1,n/4], cond(A) log-uniform in [1e1,1e6]) solved in one persistent
    launch; FP64-comparator on the same kernel; sampled oracle accuracy."""
    import numpy as np
    import torch
    from paper_2406_16499_gb300 import inputs as I, mpir
    specs = I.lse_batch_specs(count=count)
    t0 = time.perf_counter()
    probs = I.lse_batch_torch(specs, dev)
    torch.cuda.synchronize(dev)
    gen_s = time.perf_counter() - t0
    xs = [torch.zeros(sp[2], dtype=torch.float64, device=dev) for sp in specs]
    batch = mpir.LseBatch(probs, xs)

    def timed(opts, reps):
        st, infos = h.lse_solve_batched(batch, opts=opts)     # tune + capture on first sight
        torch.cuda.synchronize(dev)
        call, devt = [], []
        for _ in range(reps):
            mpir.profile(True)
            t0 = time.perf_counter()
            st, infos = h.lse_solve_batched(batch, opts=opts)
            torch.cuda.synchronize(dev)
            call.append((time.perf_counter() - t0) * 1e3)
            devt.append(mpir.profile_read()["batched"][0])
            mpir.profile(False)
        return st, infos, sorted(call)[len(call) // 2], sorted(devt)[len(devt) // 2]

    launches0 = mpir.launch_count(13)
    st, infos, ms, dms = timed(mpir.make_opts(fact="fp32"), 3)
    launches = (mpir.launch_count(13) - launches0) // 4
    shapes = [h.batched_get_shape(b) for b in (0, 1)]
    n_esc = sum(1 for f in infos if f.escalated)
    n_bad = sum(1 for f in infos if f.status != 0)
    iters = [f.iters for f in infos]
    eta_kernel = max(max(f.stop_ratio) for f in infos)
    # the answers of the timed mixed-precision call (the FP64 comparator below
    # writes the same output vectors)
    ks = list(range(0, count, max(1, sample_every)))
    x_snap = {k: xs[k].cpu().numpy() for k in ks} if rank == 0 else {}
    st64, infos64, ms64, dms64 = timed(mpir.make_opts(fact="fp64", refine="direct", escalate=False), 2)
    flops = sum(batch_work(m, n, p) for _, m, n, p, _ in specs)
    in_bytes = sum(8.0 * (m * n + p * n + m + p) for _, m, n, p, _ in specs)
    peaks = measured_peaks()
    sms = torch.cuda.get_device_properties(dev).multi_processor_count
    out = {"workload": "batched uneven LSE, %d problems, m~U[32,512] n~U[16,m/2] p~U[1,n/4], "
                       "cond(A) log-U[1e1,1e6], cond(B)=10" % count,
           "value": count * 1000.0 / ms, "unit": "solves/s", "ms": ms,
           "device": {"value": count * 1000.0 / dms, "ms": dms,
                      "what": "graph launch of the persistent kernels alone (CUDA events)"},
           "status": st, "not_converged": n_bad, "escalated": n_esc, "iters_mean": float(np.mean(iters)),
           "eta_kernel_max": eta_kernel,
           "shapes": shapes,
           "fp64_direct": {"value": count * 1000.0 / ms64, "unit": "solves/s", "ms": ms64,
                           "device_ms": dms64, "status": st64},
           "speedup_vs_fp64_direct": ms64 / ms,
           "device_speedup_vs_fp64_direct": dms64 / dms,
           "gflops": flops / (dms * 1e-3) / 1e9,
           "roofline": {"fp32_frac": flops / (dms * 1e-3) / 1e12 / fp32_simt_peak(peaks.get("sm_max_mhz", 2070.0), sms),
                        "hbm_frac": in_bytes / (dms * 1e-3) / 1e9 / peaks["hbm_gbs"],
                        "note": "device time; FP32 GRQ flops vs FP32 SIMT peak; FP64 input bytes vs measured HBM"},
           "persistent_launches_per_solve_call": int(launches),
           "input_generation_s": gen_s}
    if rank == 0:
        import oracle
        worst = {"eta": 0.0, "e_con": 0.0, "fe_over_bound": 0.0}
        for k in ks:
            P = {key: v.cpu().numpy() for key, v in probs[k].items()}
            x = x_snap[k]
            A, B, b, d = P["A"], P["B"], P["b"], P["d"]
            t = oracle.lse_truth(A, B, b, d)
            F = oracle.lse_factor(A, B, "fp64")
            r = b - A @ x
            v = oracle.lse_init_v(F, A, r)
            met = oracle.lse_metrics(A, B, b, d, x, r, v)
            kap = oracle.lse_kappa(F, t["x"], t["r"])[0]
            fe = float(np.linalg.norm(x - t["x"]) / np.linalg.norm(t["x"]))
            worst["eta"] = max(worst["eta"], met["eta"])
            worst["e_con"] = max(worst["e_con"], met["e_con"])
            worst["fe_over_bound"] = max(worst["fe_over_bound"], fe / (10 * kap * 1.1e-16))
        worst.pop("eta")
        out["accuracy_sample"] = dict(worst, problems=len(ks),
                                      note="oracle e_con and forward error / (10 kappa u) on every "
                                           "%d-th problem; eta from the kernel's FP64 residual" % sample_every)
    return out


def gls_batch_work(n, m, p):
    """Algorithmic flops of one batched GLS problem: the GQR (QR of the
    n x m W, its reflectors applied to the p columns of V, QR of the p x n
    C~) plus one residual."""
    kC = min(n, p)
    f = 2.0 * n * m * m - 2.0 * m ** 3 / 3.0 + 4.0 * n * m * p - 2.0 * m * m * p
    f += 2.0 * p * n * kC - 2.0 * kC ** 3 / 3.0
    return f + 8.0 * (n * m + n * p)


def run_batched_gls(count, h, dev, rank=0, sample_every=250):
    """Uneven batch of `count` GLS problems (n ~ U[32,512], m ~ U[4,n/2],
    p ~ U[n,5n/4], cond(W) log-uniform in [1e1,1e5]) in one persistent
    launch; FP64 comparator on the same kernel; oracle accuracy on a
    sample."""
    import numpy as np
    import torch
    from paper_2406_16499_gb300 import inputs as I, mpir
    specs = I.gls_batch_specs(count=count)
    t0 = time.perf_counter()
    probs = I.gls_batch_torch(specs, dev)
    torch.cuda.synchronize(dev)
    gen_s = time.perf_counter() - t0
    xs = [torch.zeros(sp[2], dtype=torch.float64, device=dev) for sp in specs]
    ys = [torch.zeros(sp[3], dtype=torch.float64, device=dev) for sp in specs]
    batch = mpir.GlsBatch(probs, xs, ys)

    def timed(opts, reps):
        h.gls_solve_batched(batch, opts=opts)
        torch.cuda.synchronize(dev)
        call, devt = [], []
        st, infos = 0, None
        for _ in range(reps):
            mpir.profile(True)
            t0 = time.perf_counter()
            st, infos = h.gls_solve_batched(batch, opts=opts)
            torch.cuda.synchronize(dev)
            call.append((time.perf_counter() - t0) * 1e3)
            devt.append(mpir.profile_read()["batched"][0])
            mpir.profile(False)
        return st, infos, sorted(call)[len(call) // 2], sorted(devt)[len(devt) // 2]

    st, infos, ms, dms = timed(mpir.make_opts(fact="fp32"), 3)
    # statistics and answers of the mixed-precision call, before the FP64
    # comparator overwrites the batch's result records and output vectors
    stats = {"not_converged": sum(1 for f in infos if f.status != 0),
             "escalated": sum(1 for f in infos if f.escalated),
             "iters_mean": float(np.mean([f.iters for f in infos]))}
    ks = list(range(0, count, max(1, sample_every)))
    snap = {k: (xs[k].cpu().numpy(), ys[k].cpu().numpy()) for k in ks} if rank == 0 else {}
    st64, _, ms64, dms64 = timed(mpir.make_opts(fact="fp64", refine="direct", escalate=False), 2)
    flops = sum(gls_batch_work(n, m, p) for _, n, m, p, _ in specs)
    out = {"workload": "batched uneven GLS, %d problems, n~U[32,512] m~U[4,n/2] p~U[n,5n/4], "
                       "cond(W) log-U[1e1,1e5], cond(V)=10" % count,
           "value": count * 1000.0 / ms, "unit": "solves/s", "ms": ms,
           "device": {"value": count * 1000.0 / dms, "ms": dms,
                      "what": "graph launch of the persistent kernels alone (CUDA events)"},
           "status": st, **stats,
           "fp64_direct": {"value": count * 1000.0 / ms64, "unit": "solves/s", "ms": ms64, "device_ms": dms64,
                           "status": st64},
           "speedup_vs_fp64_direct": ms64 / ms, "device_speedup_vs_fp64_direct": dms64 / dms,
           "gflops": flops / (dms * 1e-3) / 1e9, "input_generation_s": gen_s}
    if rank == 0:
        import oracle
        worst = {"e_con": 0.0, "fe_over_bound": 0.0}
        for k in ks:
            W, V, d = (probs[k][key].cpu().numpy() for key in ("W", "V", "d"))
            x, y = snap[k]
            t = oracle.gls_truth(W, V, d)
            F = oracle.gls_factor(W, V, "fp64")
            kap = oracle.gls_kappa(F, t["x"], t["y"])[0]
            f2 = d - W @ x - V @ y
            e_con = np.linalg.norm(f2) / (np.linalg.norm(W) * np.linalg.norm(x) + np.linalg.norm(V) *
                                          np.linalg.norm(y) + np.linalg.norm(d))
            fe = float(np.linalg.norm(x - t["x"]) / np.linalg.norm(t["x"]))
            worst["e_con"] = max(worst["e_con"], e_con)
            worst["fe_over_bound"] = max(worst["fe_over_bound"], fe / (10 * kap * U64))
        out["accuracy_sample"] = dict(worst, problems=len(ks),
                                      note="oracle e_con and forward error / (10 kappa u) on every "
                                           "%d-th problem" % sample_every)
    return out


def run_selector(h, rank, count=100):
    """The learned selector with the shipped weights on a held-out mixed set
    (`count` LSE and `count` GLS problems, kappa_2 log-uniform in [1, 1e12]):
    total wall time of fact = AUTO (features, network, chosen solve,
    escalation) against fixed FP32 + classical IR with escalation, every
    AUTO answer judged by the oracle (FP64-level bar)."""
    import numpy as np
    import torch
    from paper_2406_16499_gb300 import inputs as I, mpir, selector as SEL
    path = os.path.join(ROOT, "paper_2406_16499_gb300", "selector_weights.npz")
    if not os.path.exists(path):
        return {"skipped": "no trained selector weights (python -m paper_2406_16499_gb300.train_selector)"}
    sel = SEL.Selector.load(path)
    sel.install(h)
    held = [("lse", P) for P in I.selector_lse_problems(909, count)]
    held += [("gls", G) for G in I.selector_gls_problems(910, count)]

    def dev(a):
        a = np.asarray(a, dtype=np.float64)
        return torch.from_numpy(a.copy()).cuda() if a.ndim == 1 else torch.from_numpy(np.ascontiguousarray(a.T)).cuda().t()

    def run(kind, P, fact):
        if kind == "lse":
            A, B, b, d = (dev(P[k]) for k in ("A", "B", "b", "d"))
            m, n = P["A"].shape
            p = P["B"].shape[0]
            x, r, v = (torch.zeros(k, dtype=torch.float64, device="cuda") for k in (n, m, max(p, 1)))
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            st, info = h.lse_solve(A, B, b, d, x, r, v if p else None, mpir.make_opts(fact=fact))
            torch.cuda.synchronize()
            return st, info, time.perf_counter() - t0, (x.cpu().numpy(), r.cpu().numpy(), v.cpu().numpy()[:p])
        W, V, d = (dev(P[k]) for k in ("W", "V", "d"))
        n, m = P["W"].shape
        p = P["V"].shape[1]
        x, y, z = (torch.zeros(k, dtype=torch.float64, device="cuda") for k in (m, p, n))
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        st, info = h.gls_solve(W, V, d, x, y, z, mpir.make_opts(fact=fact))
        torch.cuda.synchronize()
        return st, info, time.perf_counter() - t0, (x.cpu().numpy(), y.cpu().numpy(), z.cpu().numpy())

    run(*held[0], "fp32")
    run(*held[0], "auto")
    t_auto = t_fixed = 0.0
    worst_eta = worst_econ = 0.0
    chosen = [0] * 6
    fails = esc_auto = esc_fixed = 0
    for kind, P in held:
        st0, inf0, tf, _ = run(kind, P, "fp32")
        st1, inf1, ta, sol = run(kind, P, "auto")
        t_fixed += tf
        t_auto += ta
        esc_fixed += inf0.escalated
        esc_auto += inf1.escalated
        if st1 != 0:
            fails += 1
        cls = 2 * {0: 0, 1: 0, 2: 1, 3: 2}.get(inf1.fact_used, 1) + (1 if inf1.refine_used == 1 else 0)
        chosen[min(cls, 5)] += 1
        if rank == 0:
            import oracle
            if kind == "lse":
                met = oracle.lse_metrics(P["A"], P["B"], P["b"], P["d"], *sol)
            else:
                met = oracle.gls_metrics(P["W"], P["V"], P["d"], *sol)
            worst_eta = max(worst_eta, met["eta"])
            worst_econ = max(worst_econ, met["e_con"])
    h.selector_set(None, None, None)
    n_all = len(held)
    return {"workload": "held-out mixed set: %d LSE (m~U[64,400]) + %d GLS (n~U[64,400]), kappa log-U[1,1e12]"
                        % (count, count),
            "auto": {"value": n_all / t_auto, "unit": "solves/s", "seconds": t_auto, "escalated": esc_auto,
                     "failed": fails},
            "fixed_fp32_escalating": {"value": n_all / t_fixed, "unit": "solves/s", "seconds": t_fixed,
                                      "escalated": esc_fixed},
            "gain": t_fixed / t_auto, "classes_chosen": dict(zip(["%s+%s" % c for c in SEL.CLASSES], chosen)),
            "oracle_worst": {"eta": worst_eta, "e_con": worst_econ},
            "note": "wall time per solve including the selector's features and network; weights trained by "
                    "train_selector on the library's own timed solves"}


# --------------------------------------------------------------- arms --

def cond_seed(cond, rank=0):
    import math
    return SEED + int(round(math.log10(cond))) + 1000 * rank


def make_inputs(rank, device="cuda", cond=COND_A):
    """The rank's LSE problem (replicas: every rank its own seed)."""
    from paper_2406_16499_gb300 import inputs as I
    return I.lse_known_torch(cond_seed(cond, rank), M_, N_, P_, cond, COND_B, device)


def make_gls_inputs(rank):
    from paper_2406_16499_gb300 import inputs as I
    return I.gls_ar1(seed=GLS_SEED + 1000 * rank, n=GLS_N, m=GLS_M)


def host_problem(T):
    return {k: (v.cpu().numpy() if hasattr(v, "cpu") else v) for k, v in T.items()}


def oracle_accuracy(Hs, x, r, v):
    """eta, e_con (oracle, double-double residual) and the forward error
    against the known solution with its bound 10 kappa_up u."""
    import numpy as np
    import oracle
    met = oracle.lse_metrics(Hs["A"], Hs["B"], Hs["b"], Hs["d"], x, r, v)
    fe = float(np.linalg.norm(x - Hs["x_true"]) / np.linalg.norm(Hs["x_true"]))
    bound = 10 * Hs["kappa_up"] * U64
    return {"eta": met["eta"], "e_con": met["e_con"], "fwd": fe, "kappa_up": Hs["kappa_up"],
            "fwd_over_bound": fe / bound,
            "fp64_level": bool(met["eta"] <= 1e-14 and met["e_con"] <= 1e-14 and fe <= bound)}


def oracle_cpu_solve(Hs, fact="fp32"):
    import oracle
    return oracle.lse_solve(Hs["A"], Hs["B"], Hs["b"], Hs["d"], fact=fact)


def run_reference(args):
    rank, world, _ = dist_env()
    if rank != 0:
        return 0
    import oracle
    import numpy as np
    import torch
    T = make_inputs(0, "cpu")
    Hs = host_problem(T)
    del T
    oracle.lib()
    t0 = time.perf_counter()
    out = oracle_cpu_solve(Hs)                          # warm sample, also sizes the run
    t_first = time.perf_counter() - t0
    budget = 150.0
    warm = max(0, min(args.warmup - 1, int(budget / max(t_first, 1e-3)) // 4))
    for _ in range(warm):
        oracle_cpu_solve(Hs)
    steps = max(1, min(args.steps, int(budget / max(t_first, 1e-3))))
    times = []
    for _ in range(steps):
        t0 = time.perf_counter()
        out = oracle_cpu_solve(Hs)
        times.append(time.perf_counter() - t0)
    ms = 1000.0 * sum(times) / len(times)
    acc = oracle_accuracy(Hs, out["x"], out["r"], out["v"])
    value = 1000.0 / ms
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": "solves/s", "n_gpus": args.gpus,
        "steps": steps, "warmup": 1 + warm, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32/f64", "data": "synthetic",
        "config": config("fp32"),
        "cpu_baseline": {"value": value, "unit": "solves/s", "cores": nproc(), "kind": "oracle",
                         "threads": oracle.num_threads(),
                         "sample": "%d full solve(s) of the workload by the CPU oracle (Alg. 2: unblocked "
                                   "FP32 GRQ + FP64 classical IR, OpenMP)" % steps},
        "e2e": {"value": value, "unit": "solves/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
        "accuracy": dict(acc, iters=out["iters"], status=out["status"]),
    }
    print(json.dumps(line), flush=True)
    return 0


def timed_solve(h, T, opts, stream, reps, x, r, v, warm=True):
    """Median device time (CUDA events on the launch stream) of `reps`
    solves after one untimed one (warm); returns (ms, status, info)."""
    import torch
    if warm:
        h.lse_solve(T["A"], T["B"], T["b"], T["d"], x, r, v, opts)
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    ts, st, info = [], 0, None
    for _ in range(reps):
        e0.record(stream)
        st, info = h.lse_solve(T["A"], T["B"], T["b"], T["d"], x, r, v, opts)
        e1.record(stream)
        e1.synchronize()
        ts.append(e0.elapsed_time(e1))
    return sorted(ts)[len(ts) // 2], st, info


def run_sweep(h, stream, rank, T_head, Hs_head):
    """cond(A) in {1e1, 1e4, 1e8}: FP32 / TF32 factors with classical IR,
    FP32 with GMRES-IR, BF16 factors (cond 1e1) with classical and GMRES-IR,
    and the FP64 solves; every result's accuracy from the oracle's
    double-double residual and the known solution."""
    import torch
    from paper_2406_16499_gb300 import mpir
    out = {}
    x = torch.zeros(N_, dtype=torch.float64, device="cuda")
    r = torch.zeros(M_, dtype=torch.float64, device="cuda")
    v = torch.zeros(P_, dtype=torch.float64, device="cuda")
    # FP64 classical: FP64 factors + FP64 refinement, the fixed-precision
    # solve that reaches the FP64-level bar (the unrefined FP64 direct solve
    # computes r = b - A x directly and loses r's accuracy to cancellation)
    variants = [("fp32_classical", dict(fact="fp32", refine="classical"), 3),
                ("tf32_classical", dict(fact="tf32", refine="classical", escalate=False), 3),
                ("fp32_gmres", dict(fact="fp32", refine="gmres", escalate=False), 2),
                ("bf16_classical", dict(fact="bf16", refine="classical", escalate=False), 2),
                ("bf16_gmres", dict(fact="bf16", refine="gmres", escalate=False), 1),
                ("fp64_classical", dict(fact="fp64", refine="classical", escalate=False), 1),
                ("fp64_direct", dict(fact="fp64", refine="direct"), 1)]
    for cond in CONDS:
        if cond == COND_A:
            T, Hs = T_head, Hs_head
        else:
            T = make_inputs(rank, "cuda", cond)
            Hs = host_problem(T) if rank == 0 else None
        res = {}
        for name, kw, reps in variants:
            if name == "fp32_gmres" and cond >= 1e8:
                res[name] = {"skipped": "u_f kappa(A) kappa(B) > 1: the block-diagonal preconditioner "
                                        "does not apply (GMRES stalls; 6.3 s measured)"}
                continue
            if name.startswith("bf16") and cond > 1e1:
                res[name] = {"skipped": "u_bf16 kappa(A) > 1 (u_bf16 = 2^-8): neither classical IR nor the "
                                        "preconditioner converges"}
                continue
            ms, st, info = timed_solve(h, T, mpir.make_opts(**kw), stream, reps, x, r, v,
                                       warm=not name.startswith("fp64"))
            d = info.as_dict()
            e = {"ms": ms, "status": st, "iters": d["iters"], "inner_iters": d["inner_iters"],
                 "escalated": d["escalated"], "fact_used": d["fact_used"]}
            if rank == 0:
                e.update(oracle_accuracy(Hs, x.cpu().numpy(), r.cpu().numpy(), v.cpu().numpy()))
            res[name] = e
        out["%.0e" % cond] = res
        if cond != COND_A:
            del T, Hs
            torch.cuda.empty_cache()
    return out


def run_gls(h, dev, stream, rank, steps):
    """The GLS n = 4096 AR(1) workload: FP32 GQR + FP64 classical IR vs the
    FP64 GQR direct solve, accuracy against the oracle's solution."""
    import numpy as np
    import torch
    from paper_2406_16499_gb300 import mpir
    G = make_gls_inputs(rank)
    Wn, Vn, dn = G["W"], G["V"], G["d"]
    n, m = Wn.shape
    p = Vn.shape[1]

    def to_dev(a):
        return torch.from_numpy(np.ascontiguousarray(a.T)).to(dev).t()

    W, V, d = to_dev(Wn), to_dev(Vn), torch.from_numpy(dn.copy()).to(dev)
    x = torch.zeros(m, dtype=torch.float64, device=dev)
    y = torch.zeros(p, dtype=torch.float64, device=dev)
    z = torch.zeros(n, dtype=torch.float64, device=dev)
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device=dev)
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)

    def timed(o, k):
        h.gls_solve(W, V, d, x, y, z, o)
        torch.cuda.synchronize()
        ts, info = [], None
        for _ in range(k):
            flush.zero_()
            e0.record(stream)
            st, info = h.gls_solve(W, V, d, x, y, z, o)
            e1.record(stream)
            e1.synchronize()
            ts.append(e0.elapsed_time(e1))
        return sorted(ts)[len(ts) // 2], st, info

    out = {"workload": GLS_WORKLOAD, "l2": "inputs 168 MB > L2; 256 MB L2 flush before every timed step"}
    ms, st, info = timed(mpir.make_opts(fact="fp32", refine="classical"), steps)
    out["fp32_classical"] = {"ms": ms, "value": 1000.0 / ms, "unit": "solves/s", "status": st,
                             "iters": info.iters}
    if rank == 0:
        import oracle
        t = oracle.gls_truth(Wn, Vn, dn)
        F = oracle.gls_factor(Wn, Vn, "fp64")
        kap = oracle.gls_kappa(F, t["x"], t["y"])[0]
        met = oracle.gls_metrics(Wn, Vn, dn, x.cpu().numpy(), y.cpu().numpy(), z.cpu().numpy())
        fe = float(np.linalg.norm(x.cpu().numpy() - t["x"]) / np.linalg.norm(t["x"]))
        out["fp32_classical"].update(eta=met["eta"], e_con=met["e_con"], fwd=fe, kappa=kap,
                                     fwd_over_bound=fe / (10 * kap * U64))
    ms, st, info = timed(mpir.make_opts(fact="fp32", refine="gmres", escalate=False), 2)
    out["fp32_gmres"] = {"ms": ms, "status": st, "iters": info.iters, "inner_iters": info.inner_iters}
    ms64, st, info = timed(mpir.make_opts(fact="fp64", refine="direct"), 2)
    out["fp64_direct"] = {"ms": ms64, "value": 1000.0 / ms64, "status": st}
    out["speedup_vs_fp64_direct"] = ms64 / out["fp32_classical"]["ms"]
    return out


COMPLEX_LSE = (2048, 1024, 64, 1e3, 1e1)     # m, n, p, cond(A), cond(B)
COMPLEX_GLS = (2048, 512, 2048, 1e3, 1e1)    # n, m, p, cond(W), cond(V)


def run_complex(h, dev, stream):
    """Complex LSE and GLS (Sec. 1 poses both over C): zlse_solve /
    zgls_solve with FP32-class factors and FP64 classical IR against FP64
    factors, same GPU, same handle.  Accuracy in complex128 on the host:
    err-1 (the constraint residual of Tables 4 / 5) and the agreement of the
    two solutions.  Any failure is reported in the record instead of ending
    the benchmark."""
    import numpy as np
    import torch
    from paper_2406_16499_gb300 import inputs as I
    from paper_2406_16499_gb300 import mpir

    def zdev(a):
        a = np.asarray(a, dtype=np.complex128)
        if a.ndim == 1:
            return torch.from_numpy(a.copy()).to(dev)
        return torch.from_numpy(np.ascontiguousarray(a.T)).to(dev).t()

    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)

    def timed(fn, k):
        fn()
        torch.cuda.synchronize()
        ts, st, info = [], None, None
        for _ in range(k):
            e0.record(stream)
            st, info = fn()
            e1.record(stream)
            e1.synchronize()
            ts.append(e0.elapsed_time(e1))
        return sorted(ts)[len(ts) // 2], st, info

    out = {"what": "complex problems through the real 2x2 block embedding (FP32-class factors + FP64 classical "
                   "IR) against FP64 factors, same GPU; err-1 = ||Bx-d|| / (||B||_F ||x|| + ||d||) (LSE), "
                   "||Wx+Vy-d|| / (||W||_F ||x|| + ||V||_F ||y|| + ||d||) (GLS)"}
    try:
        m, n, p, ca, cb = COMPLEX_LSE
        P = I.zlse_svd(4242, m, n, p, ca, cb)
        A, B, b, d = zdev(P["A"]), zdev(P["B"]), zdev(P["b"]), zdev(P["d"])
        xs = {}
        rec = {"m": m, "n": n, "p": p, "cond_a": ca, "cond_b": cb}
        for name, kw, k in (("fp32_classical", dict(fact="fp32", refine="classical"), 5),
                            ("fp64_classical", dict(fact="fp64", refine="classical"), 2)):
            x = torch.zeros(n, dtype=torch.complex128, device=dev)
            r = torch.zeros(m, dtype=torch.complex128, device=dev)
            v = torch.zeros(p, dtype=torch.complex128, device=dev)
            o = mpir.make_opts(**kw)
            ms, st, info = timed(lambda: h.zlse_solve(A, B, b, d, x, r, v, o), k)
            xh = x.cpu().numpy()
            xs[name] = xh
            e1c = float(np.linalg.norm(P["B"] @ xh - P["d"]) /
                        (np.linalg.norm(P["B"]) * np.linalg.norm(xh) + np.linalg.norm(P["d"])))
            rec[name] = {"ms": ms, "status": st, "iters": info.iters, "escalated": info.escalated, "err1": e1c}
        rec["x_rel_diff"] = float(np.linalg.norm(xs["fp32_classical"] - xs["fp64_classical"]) /
                                  np.linalg.norm(xs["fp64_classical"]))
        rec["speedup_vs_fp64"] = rec["fp64_classical"]["ms"] / rec["fp32_classical"]["ms"]
        out["lse"] = rec
    except Exception as exc:                       # reported, never fatal
        out["lse"] = {"error": repr(exc)[:300]}
    try:
        n, m, p, cw, cv = COMPLEX_GLS
        G = I.zgls_svd(4343, n, m, p, cw, cv)
        W, V, d = zdev(G["W"]), zdev(G["V"]), zdev(G["d"])
        sol = {}
        rec = {"n": n, "m": m, "p": p, "cond_w": cw, "cond_v": cv}
        for name, kw, k in (("fp32_classical", dict(fact="fp32", refine="classical"), 5),
                            ("fp64_classical", dict(fact="fp64", refine="classical"), 2)):
            x = torch.zeros(m, dtype=torch.complex128, device=dev)
            y = torch.zeros(p, dtype=torch.complex128, device=dev)
            z = torch.zeros(n, dtype=torch.complex128, device=dev)
            o = mpir.make_opts(**kw)
            ms, st, info = timed(lambda: h.zgls_solve(W, V, d, x, y, z, o), k)
            xh, yh = x.cpu().numpy(), y.cpu().numpy()
            sol[name] = xh
            e1c = float(np.linalg.norm(G["W"] @ xh + G["V"] @ yh - G["d"]) /
                        (np.linalg.norm(G["W"]) * np.linalg.norm(xh) + np.linalg.norm(G["V"]) * np.linalg.norm(yh)
                         + np.linalg.norm(G["d"])))
            rec[name] = {"ms": ms, "status": st, "iters": info.iters, "escalated": info.escalated, "err1": e1c}
        rec["x_rel_diff"] = float(np.linalg.norm(sol["fp32_classical"] - sol["fp64_classical"]) /
                                  np.linalg.norm(sol["fp64_classical"]))
        rec["speedup_vs_fp64"] = rec["fp64_classical"]["ms"] / rec["fp32_classical"]["ms"]
        out["gls"] = rec
    except Exception as exc:                       # reported, never fatal
        out["gls"] = {"error": repr(exc)[:300]}
    return out


PAPER_LSE1 = [(n, m_f * n, n // p_d) for n in (1024, 2048, 3072) for (m_f, p_d) in
              ((8, 32), (8, 64), (10, 32), (10, 64), (12, 32), (12, 64))]
PAPER_LSE2 = [(n, m_f * n, n // p_d) for n in (128, 192, 256) for (m_f, p_d) in
              ((128, 8), (128, 4), (128, 2), (256, 8), (256, 4), (256, 2))]
PAPER_GLS = [(n, n // m_d, p_f * n) for n in (1024, 2048, 3072) for (p_f, m_d) in
             ((8, 32), (8, 64), (10, 32), (10, 64), (12, 32), (12, 64))]


def paper_shape_list(full):
    """The Sec. 6.2 / 6.3 shapes (all of them with `full`; else the corners:
    n in {1024, 2048} (LSE m > n >> p, GLS) and {128, 256} (LSE m >> n > p),
    the smallest and largest aspect ratios, two conditionings)."""
    if full:
        lse1 = [(s, k) for s in PAPER_LSE1 for k in (1e3, 1e5, 1e7, 1e9)]
        lse2 = [(s, 1e5) for s in PAPER_LSE2]
        gls = [(s, k) for s in PAPER_GLS for k in (1e3, 1e5, 1e7, 1e9)]
        return lse1, lse2, gls
    lse1 = [((n, m, p), k) for (n, m, p) in PAPER_LSE1 if n in (1024, 2048) and (m, p) in
            ((8 * n, n // 32), (12 * n, n // 64)) for k in (1e3, 1e7)]
    lse2 = [((n, m, p), 1e5) for (n, m, p) in PAPER_LSE2 if n in (128, 256) and (m, p) in
            ((128 * n, n // 8), (256 * n, n // 2))]
    gls = [((n, m, p), k) for (n, m, p) in PAPER_GLS if n in (1024, 2048) and (p, m) in
           ((8 * n, n // 32), (12 * n, n // 64)) for k in (1e3, 1e7)]
    return lse1, lse2, gls


def run_paper_shapes(h, dev, stream, full=False):
    """Timed sweep over the paper's test shapes (Sec. 6.2: LSE m > n >> p and
    m >> n > p; Sec. 6.3: GLS p >> n > m) with its matrix construction
    ([A^T, B^T] resp. [W, V] = W1 Sigma W2, geometric Sigma): FP32 factors
    with classical IR and with GMRES-IR (block-diagonal split preconditioner),
    against the FP64 factorization with FP64 classical IR on the same GPU
    (the paper's comparison is against xGGLSE / xGGGLM, also FP64).  Each
    entry: ms, status, refinement steps, the library's backward error
    (eq. lse-stop / gls-stop ratios) and x's relative distance to the FP64
    solution; speedup = t_fp64 / t_mixed."""
    import torch
    from paper_2406_16499_gb300 import inputs as I, mpir
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)

    def timed(fn, k):
        fn()
        ts, out = [], None
        for _ in range(k):
            torch.cuda.synchronize()
            e0.record(stream)
            out = fn()
            e1.record(stream)
            e1.synchronize()
            ts.append(e0.elapsed_time(e1))
        return sorted(ts)[len(ts) // 2], out

    def entry(ms, st, info):
        return {"ms": round(ms, 3), "status": st, "iters": info.iters, "inner_iters": info.inner_iters,
                "escalated": info.escalated, "eta": max(info.stop_ratio)}

    lse1, lse2, gls = paper_shape_list(full)
    rows = []

    def guarded(row, fn):
        try:
            fn(row)
        except mpir.MpirError as e:                 # record it, keep the sweep going
            row["error"] = str(e)
        rows.append(row)

    def fill(row, solve, x, x64):
        ms, (st, info) = timed(lambda: solve(mpir.make_opts(fact="fp32"), x), 2)
        row["fp32_classical"] = entry(ms, st, info)
        ms, (st, info) = timed(lambda: solve(mpir.make_opts(fact="fp32", refine="gmres", escalate=False), x), 1)
        row["fp32_gmres"] = entry(ms, st, info)
        ms64, (st, info) = timed(lambda: solve(mpir.make_opts(fact="fp64"), x64), 1)
        row["fp64_classical"] = entry(ms64, st, info)
        solve(mpir.make_opts(fact="fp32"), x)
        row["x_vs_fp64"] = float(torch.linalg.norm(x - x64) / torch.linalg.norm(x64))
        row["speedup_classical"] = ms64 / row["fp32_classical"]["ms"]
        row["speedup_gmres"] = ms64 / row["fp32_gmres"]["ms"]

    for case, lst in (("lse m>n>>p", lse1), ("lse m>>n>p", lse2)):
        for (n, m, p), kap in lst:
            P = I.lse_paper_torch(hash((m, n, p, kap)) & 0xFFFFFFFF, m, n, p, kap, dev)
            x = torch.zeros(n, dtype=torch.float64, device=dev)
            x64 = torch.zeros(n, dtype=torch.float64, device=dev)

            def solve(o, out):
                return h.lse_solve(P["A"], P["B"], P["b"], P["d"], out, None, None, o)

            guarded({"case": case, "m": m, "n": n, "p": p, "kappa": kap}, lambda row: fill(row, solve, x, x64))
            del P
    for (n, m, p), kap in gls:
        G = I.gls_paper_torch(hash((n, m, p, kap)) & 0xFFFFFFFF, n, m, p, kap, dev)
        x = torch.zeros(m, dtype=torch.float64, device=dev)
        y = torch.zeros(p, dtype=torch.float64, device=dev)
        x64 = torch.zeros(m, dtype=torch.float64, device=dev)

        def gsolve(o, out):
            return h.gls_solve(G["W"], G["V"], G["d"], out, y, None, o)

        guarded({"case": "gls p>>n>m", "n": n, "m": m, "p": p, "kappa": kap}, lambda row: fill(row, gsolve, x, x64))
        del G
    torch.cuda.empty_cache()
    return {"what": "Sec. 6.2 / 6.3 test shapes, FP32 factors (classical IR, GMRES-IR) vs FP64 factors, same GPU",
            "construction": "[A^T, B^T] (LSE) / [W, V] (GLS) = W1 Sigma W2, geometric Sigma with the given kappa_2, "
                            "Haar factors drawn on the GPU",
            "full": bool(full), "rows": rows}


def pick_roofline(prof, kp, work, iters, peaks, sms, clk):
    """Roofline of the kernel kind with the largest device time per solve
    (achieved = the algorithmic work of its launches / their summed CUDA-event
    time)."""
    cand = {k: v for k, v in prof.items() if v[1]}
    name, (ms, cnt) = max(cand.items(), key=lambda kv: kv[1][0])
    sm_max = peaks.get("sm_max_mhz", 2070.0)
    sec = ms * 1e-3
    if name == "larfb_tc":
        alg = work["tc_flops"] * kp
        roof = {"bound": "tensor", "unit": "TFLOP/s", "peak": tf32_peak(peaks, sustained=True),
                "peak_note": "TF32 dense = measured sustained BF16 cuBLAS x 1.1/2.25 (of measured); the "
                             "FP32-class update issues three TF32 products per algorithmic product",
                "achieved": alg / sec / 1e12}
    elif name in ("panel_qr", "larfb"):
        alg = (work["panel_flops"] if name == "panel_qr" else work["inner_flops"]) * kp
        roof = {"bound": "alu", "unit": "TFLOP/s", "peak": fp32_simt_peak(sm_max, sms),
                "peak_note": "FP32 SIMT: %d SMs x 128 lanes x 2 x max SM clock" % sms,
                "achieved": alg / sec / 1e12}
    else:
        alg = work["resid_bytes"] * kp * max(iters, 1)
        roof = {"bound": "hbm", "unit": "GB/s", "peak": peaks["hbm_gbs"], "peak_note": "measured HBM copy",
                "achieved": alg / sec / 1e9}
    roof.update({"kernel": name, "frac": roof["achieved"] / roof["peak"], "launches_per_step": cnt / kp,
                 "ms_per_step": ms / kp, "traffic": traffic_record(name),
                 "peak_source": "fallback peaks (MEASURED_PEAKS.json absent)" if peaks.get("_fallback")
                 else "MEASURED_PEAKS.json"})
    return roof


def run_ours(args):
    import numpy as np
    import torch
    from paper_2406_16499_gb300 import mpir

    rank, world, local = dist_env()
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group(backend="nccl")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    stream = torch.cuda.current_stream(dev)
    sms = torch.cuda.get_device_properties(dev).multi_processor_count
    h = mpir.Handle(local, stream.cuda_stream)
    if args.batched_only:
        res = run_batched(args.batched_count, h, dev, stream, rank)
        if rank == 0:
            print(json.dumps(res), flush=True)
        h.close()
        return 0
    if args.paper_shapes_only:
        res = run_paper_shapes(h, dev, stream, args.paper_shapes_full)
        if rank == 0:
            print(json.dumps(res), flush=True)
        h.close()
        return 0

    global M_, N_, P_
    if args.size:
        if not args.quick:
            raise SystemExit("--size is for --quick profiling runs only")
        M_, N_, P_ = args.size
    T = make_inputs(rank, dev)
    A, B, b, d = T["A"], T["B"], T["b"], T["d"]
    x = torch.zeros(N_, dtype=torch.float64, device=dev)
    r = torch.zeros(M_, dtype=torch.float64, device=dev)
    v = torch.zeros(P_, dtype=torch.float64, device=dev)
    opts = mpir.make_opts(fact=args.fact, refine="classical")

    def solve(o=opts, AA=A, BB=B, bb=b, dd=d):
        st, info = h.lse_solve(AA, BB, bb, dd, x, r, v, o)
        if st != 0:
            raise RuntimeError("lse_solve status %d: %s" % (st, h.last_error()))
        return info

    def barrier():
        if world > 1:
            torch.distributed.barrier()
        torch.cuda.synchronize(dev)

    clocks = ClockSampler(local)
    clocks.start()
    for _ in range(max(args.warmup, 3)):
        solve()
    barrier()
    launches0 = mpir.launch_count()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    total_ms = 0.0
    info = None
    if args.profile_range:
        torch.cuda.profiler.start()
    for _ in range(args.steps):
        e0.record(stream)
        info = solve()
        e1.record(stream)
        e1.synchronize()
        total_ms += e0.elapsed_time(e1)
    if args.profile_range:
        torch.cuda.profiler.stop()
    clk = clocks.stop()
    barrier()
    gpu_launches = (mpir.launch_count() - launches0) // max(args.steps, 1)
    ms = rank_max(total_ms / args.steps, world, dev)
    value = job_value(world, ms)

    if args.quick:
        # per-kind device time of a profiled pass (after the timed steps)
        mpir.profile(True)
        solve()
        torch.cuda.synchronize(dev)
        prof = mpir.profile_read()
        mpir.profile(False)
        if rank == 0:
            print(json.dumps({"metric": METRIC, "value": value, "unit": "solves/s", "ms_per_step": ms,
                              "quick": True, "size": [M_, N_, P_], "iters": info.iters if info else None,
                              "phase_ms": list(info.time_ms) if info else None,
                              "kernels": {k: {"ms": v[0], "launches": v[1]} for k, v in prof.items() if v[1]},
                              "gpu_launches": int(gpu_launches)}), flush=True)
        h.close()
        return 0

    # ---- per-kernel device time over a profiled pass of the same steps --
    mpir.profile(True)
    kp = max(2, min(args.steps, 4))
    for _ in range(kp):
        solve()
    torch.cuda.synchronize(dev)
    prof = mpir.profile_read()
    mpir.profile(False)

    # ---- accuracy of the last solution: oracle residual, known solution --
    Hs = host_problem(T) if rank == 0 else None
    acc = {}
    if rank == 0:
        acc = oracle_accuracy(Hs, x.cpu().numpy(), r.cpu().numpy(), v.cpu().numpy())
        acc.update(iters=info.iters, stop_ratio=list(info.stop_ratio), fact_used=info.fact_used,
                   escalated=info.escalated)

    # ---- end to end from pinned host buffers through the public API --------
    Ah = torch.empty((N_, M_), dtype=torch.float64).pin_memory()
    Ah.copy_(A.t())
    Bh = torch.empty((N_, P_), dtype=torch.float64).pin_memory()
    Bh.copy_(B.t())
    bh = b.cpu().pin_memory()
    dh = d.cpu().pin_memory()
    xh = torch.empty(N_, dtype=torch.float64).pin_memory()
    Ad = torch.empty((N_, M_), dtype=torch.float64, device=dev)
    Bd = torch.empty((N_, P_), dtype=torch.float64, device=dev)
    bd = torch.empty(M_, dtype=torch.float64, device=dev)
    ddv = torch.empty(P_, dtype=torch.float64, device=dev)
    h2d = (Ah.numel() + Bh.numel() + bh.numel() + dh.numel()) * 8
    d2h = N_ * 8

    def e2e_step():
        Ad.copy_(Ah, non_blocking=True)
        Bd.copy_(Bh, non_blocking=True)
        bd.copy_(bh, non_blocking=True)
        ddv.copy_(dh, non_blocking=True)
        solve(opts, Ad.t(), Bd.t(), bd, ddv)
        xh.copy_(x, non_blocking=True)

    e2e_step()
    torch.cuda.synchronize(dev)
    te = 0.0
    ke = max(2, min(args.steps, 5))
    for _ in range(ke):
        torch.cuda.synchronize(dev)
        t0 = time.perf_counter()
        e2e_step()
        torch.cuda.synchronize(dev)
        te += time.perf_counter() - t0
    e2e_ms = rank_max(1000.0 * te / ke, world, dev)
    del Ah, Bh, Ad, Bd
    torch.cuda.empty_cache()

    # ---- cond(A) sweep: FP32 / TF32 / GMRES-IR / FP64 direct -------------
    sweep = None if args.no_sweep else run_sweep(h, stream, rank, T, Hs)
    fp64 = None
    if sweep:
        f = sweep["%.0e" % COND_A]["fp64_classical"]
        fp64 = dict(f, value=1000.0 / f["ms"], unit="solves/s",
                    what="FP64 GRQ + null-space start + FP64 classical IR (same kernels at FP64): the "
                         "fixed-precision solve at the same FP64-level accuracy")

    # ---- the GLS n = 4096 workload and the batched uneven LSE -------------
    gls = None if args.no_gls else run_gls(h, dev, stream, rank, max(3, min(args.steps, 10)))
    paper_shapes = None
    if not args.no_paper_shapes and world == 1:
        paper_shapes = run_paper_shapes(h, dev, stream, args.paper_shapes_full)
    batched = None
    if args.batched_count > 0 and world == 1:
        batched = run_batched(args.batched_count, h, dev, stream, rank)
    batched_gls = None
    if args.batched_gls_count > 0 and world == 1:
        batched_gls = run_batched_gls(args.batched_gls_count, h, dev, rank)
    selector = None
    if args.selector_count > 0 and world == 1:
        selector = run_selector(h, rank, args.selector_count)
    cplx = None
    if not args.no_complex and world == 1:
        try:
            cplx = run_complex(h, dev, stream)
        except Exception as exc:                   # reported, never fatal
            cplx = {"error": repr(exc)[:300]}

    # ---- roofline of the dominant kernel --------------------------------
    work = lse_work(M_, N_, P_)
    peaks = measured_peaks()
    roof = pick_roofline(prof, kp, work, info.iters if info else 1, peaks, sms, clk)
    kernels = {k: {"ms_per_step": v[0] / kp, "launches_per_step": v[1] / kp} for k, v in prof.items() if v[1]}
    tc = prof.get("larfb_tc", (0.0, 0))
    tensor = None
    if tc[1]:
        tensor = {"kernel": "k_gemm_tc (tcgen05, TMA, TMEM)", "algorithmic_tflops": work["tc_flops"] * kp /
                  (tc[0] * 1e-3) / 1e12, "peak": tf32_peak(peaks, True),
                  "note": "algorithmic trailing-update flops / summed event time of the tensor-core GEMM "
                          "launches; the FP32-class update runs three TF32 products per product"}
        tensor["frac"] = tensor["algorithmic_tflops"] / tensor["peak"]
    dg = prof.get("dual_gemv_fp64", (0.0, 0))
    resid = None
    if dg[1]:
        nres = dg[1] / 2.0                     # two launches (A and B blocks) per residual
        resid = {"kernel": "k_dual_gemv (FP64 residual)", "gbs": work["resid_bytes"] * nres / (dg[0] * 1e-3) / 1e9,
                 "peak": peaks["hbm_gbs"], "traffic_per_launch": traffic_record("dual_gemv_fp64"),
                 "algorithmic_bytes_per_launch": work["resid_bytes"] / 2,
                 "note": "FP64-pipe bound (two FMAs per 8-byte element); ncu: FP64 pipe 91 % busy"}
        resid["frac"] = resid["gbs"] / resid["peak"]

    # ---- CPU oracle on the host cores (rank 0, N = 1) ---------------------
    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        import oracle
        t0 = time.perf_counter()
        oracle_cpu_solve(Hs)
        tc_ = time.perf_counter() - t0
        cpu = {"value": 1.0 / tc_, "unit": "solves/s", "cores": nproc(), "threads": oracle.num_threads(),
               "kind": "oracle",
               "sample": "1 full solve of the workload (Alg. 2: unblocked FP32 GRQ + FP64 IR, OpenMP), "
                         "%.1f s" % tc_}

    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": "solves/s", "n_gpus": world, "steps": args.steps,
            "warmup": max(args.warmup, 3), "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32/f64", "data": "synthetic",
            "config": config(args.fact),
            "roofline": roof,
            "cpu_baseline": cpu,
            "e2e": {"value": job_value(world, e2e_ms), "unit": "solves/s", "ms_per_step": e2e_ms,
                    "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h},
            "gpu_launches": int(gpu_launches),
            "clocks": clk,
            "accuracy": acc,
            "fp64_direct": fp64,
            "speedup_vs_fp64_direct": (fp64["ms"] / ms) if fp64 else None,
            "sweep": sweep,
            "gls_ar1": gls,
            "batched_lse": batched,
            "batched_gls": batched_gls,
            "selector": selector,
            "complex": cplx,
            "paper_shapes": paper_shapes,
            "tensor_core_update": tensor,
            "fp64_residual": resid,
            "kernels": kernels,
            "algorithmic": work,
            "parallelism": "replicas" if world > 1 else "single GPU",
        }
        print(json.dumps(line), flush=True)
    h.close()
    if world > 1:
        torch.distributed.destroy_process_group()
    return 0


def main():
    args = parse()
    if args.impl == "reference":
        return run_reference(args)
    return run_ours(args)


if __name__ == "__main__":
    sys.exit(main())
