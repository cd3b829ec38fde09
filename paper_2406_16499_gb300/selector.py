"""The learned precision / refinement selector: data, training and use.

Orchestration only.  The features (Golub-Kahan-Lanczos condition sketch and
norms), the labels (timed solves of the six classes), the training steps
(forward, backward, Adam) and the inference all run in libmpir's kernels;
this module moves arrays and keeps the trained parameters.

Classes (in the library's order): BF16 + classical, BF16 + GMRES,
FP32 + classical, FP32 + GMRES, FP64 + classical, FP64 + GMRES.
Label of a problem: the fastest class whose solve converged (status 0 from
the library's FP64 stop test); within 3 % of the fastest, the higher
factorization precision and then classical IR win, and a GMRES class gives
way to classical IR at the same precision unless it is faster by more than
25 % (GMRES-IR's time on small, latency-bound problems swings widely
between similar problems, classical IR's does not).
"""
import time

import numpy as np

from . import inputs as I
from . import mpir

CLASSES = [("bf16", "classical"), ("bf16", "gmres"), ("fp32", "classical"), ("fp32", "gmres"),
           ("fp64", "classical"), ("fp64", "gmres")]
NF, H1, H2, NC = 16, 64, 64, 6
PARAMS = H1 * NF + H1 + H2 * H1 + H2 + NC * H2 + NC


def _dev(a):
    import torch
    a = np.asarray(a, dtype=np.float64)
    if a.ndim == 1:
        return torch.from_numpy(a.copy()).cuda()
    if a.size == 0:
        return torch.zeros(a.shape, dtype=torch.float64, device="cuda")
    return torch.from_numpy(np.ascontiguousarray(a.T)).cuda().t()


def lse_features(h, P):
    """16 features of an LSE problem (dict of numpy or device arrays)."""
    import torch
    A, B, b, d = (P[k] if isinstance(P[k], torch.Tensor) else _dev(P[k]) for k in ("A", "B", "b", "d"))
    s = _dev(I.splitmix_vector(A.shape[1]))
    out = torch.zeros(16, dtype=torch.float32, device="cuda")
    h.lse_features(A, B, b, d, s, out)
    return out.cpu().numpy()


def gls_features(h, P):
    import torch
    W, V, d = (P[k] if isinstance(P[k], torch.Tensor) else _dev(P[k]) for k in ("W", "V", "d"))
    s = _dev(I.splitmix_vector(W.shape[1] + V.shape[1]))
    out = torch.zeros(16, dtype=torch.float32, device="cuda")
    h.gls_features(W, V, d, s, out)
    return out.cpu().numpy()


def time_lse_classes(h, P, **caps):
    """(times in ms, converged flags) of the six classes on one LSE problem
    (device solve time from the library's events; no escalation).  caps:
    optional maxit / inner_maxit limits of the timed solves."""
    import torch
    A, B, b, d = (_dev(P[k]) for k in ("A", "B", "b", "d"))
    m, n = A.shape
    p = B.shape[0]
    times, ok = [], []
    for fact, refine in CLASSES:
        x, r, v = (torch.zeros(k, dtype=torch.float64, device="cuda") for k in (n, m, max(p, 1)))
        try:
            st, info = h.lse_solve(A, B, b, d, x, r, v if p else None,
                                   mpir.make_opts(fact=fact, refine=refine, escalate=False, **caps))
            times.append(float(info.time_ms[5]))
            ok.append(st == 0)
        except mpir.MpirError:
            times.append(float("inf"))
            ok.append(False)
    return times, ok


def time_gls_classes(h, G, **caps):
    """(times in ms, converged flags) of the six classes on one GLS problem
    (device solve time from the library's events; no escalation).  caps:
    optional maxit / inner_maxit limits of the timed solves."""
    import torch
    W, V, d = (_dev(G[k]) for k in ("W", "V", "d"))
    n, m = W.shape
    p = V.shape[1]
    times, ok = [], []
    for fact, refine in CLASSES:
        x, y, z = (torch.zeros(k, dtype=torch.float64, device="cuda") for k in (m, p, n))
        try:
            st, info = h.gls_solve(W, V, d, x, y, z, mpir.make_opts(fact=fact, refine=refine, escalate=False,
                                                                     **caps))
            times.append(float(info.time_ms[5]))
            ok.append(st == 0)
        except mpir.MpirError:
            times.append(float("inf"))
            ok.append(False)
    return times, ok


def label(times, ok, tie=0.03, gmres_margin=0.25):
    cand = [i for i in range(NC) if ok[i]]
    if not cand:
        return -1
    best = min(times[i] for i in cand)
    near = [i for i in cand if times[i] <= best * (1 + tie)]
    prec = {"bf16": 0, "fp32": 1, "fp64": 2}
    lab = max(near, key=lambda i: (prec[CLASSES[i][0]], CLASSES[i][1] == "classical"))
    if CLASSES[lab][1] == "gmres":
        c = lab - 1                      # classical IR at the same precision
        if ok[c] and times[c] <= times[lab] * (1 + gmres_margin):
            lab = c
    return lab


def init_params(seed):
    """He initialization, flattened in the library's layout."""
    g = np.random.default_rng(seed)
    parts = [g.standard_normal((H1, NF)) * np.sqrt(2.0 / NF), np.zeros(H1),
             g.standard_normal((H2, H1)) * np.sqrt(2.0 / H1), np.zeros(H2),
             g.standard_normal((NC, H2)) * np.sqrt(2.0 / H2), np.zeros(NC)]
    return np.concatenate([p.reshape(-1) for p in parts]).astype(np.float32)


class Selector:
    """Trained parameters plus the feature standardization."""

    def __init__(self, params, mean, scale):
        self.params = np.asarray(params, dtype=np.float32)
        self.mean = np.asarray(mean, dtype=np.float32)
        self.scale = np.asarray(scale, dtype=np.float32)

    def install(self, h):
        h.selector_set(self.params, self.mean, self.scale)

    def save(self, path):
        np.savez(path, params=self.params, mean=self.mean, scale=self.scale)

    @staticmethod
    def load(path):
        z = np.load(path)
        return Selector(z["params"], z["mean"], z["scale"])

    def predict(self, h, X):
        import torch
        Xs = ((np.asarray(X, np.float32) - self.mean) / self.scale).astype(np.float32)
        P = torch.from_numpy(self.params).cuda()
        Xd = torch.from_numpy(np.ascontiguousarray(Xs)).cuda()
        prob = torch.zeros((len(Xs), NC), dtype=torch.float32, device="cuda")
        h.mlp_forward(P, Xd, prob)
        return prob.cpu().numpy()


def train(h, X, y, steps=600, lr=3e-3, seed=0, log_every=0):
    """Full-batch Adam on the mean cross-entropy with the library's kernels.
    Returns (Selector, losses)."""
    import torch
    X = np.asarray(X, np.float32)
    y = np.asarray(y, np.int32)
    mean = X.mean(axis=0)
    scale = X.std(axis=0)
    scale[scale < 1e-6] = 1.0
    Xs = ((X - mean) / scale).astype(np.float32)
    P = torch.from_numpy(init_params(seed)).cuda()
    M = torch.zeros_like(P)
    V = torch.zeros_like(P)
    Xd = torch.from_numpy(np.ascontiguousarray(Xs)).cuda()
    yd = torch.from_numpy(y).cuda()
    loss = torch.zeros(1, dtype=torch.float32, device="cuda")
    losses = []
    for t in range(1, steps + 1):
        lo = loss if (t == 1 or t == steps or (log_every and t % log_every == 0)) else None
        h.mlp_train_step(P, M, V, t, lr, Xd, yd, None, lo)
        if t == 1 or t == steps or (log_every and t % log_every == 0):
            losses.append((t, float(loss.item())))
    return Selector(P.cpu().numpy(), mean, scale), losses
