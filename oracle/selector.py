"""Selector oracle: problem features and the MLP, in FP64 numpy.

TEST INFRASTRUCTURE ONLY (see oracle/__init__.py).

The selector is not part of the paper; it chooses, per problem, the
factorization precision and the refinement variant (Sec. 3 classical IR,
Sec. 5 GMRES-IR) that the paper's method should use.

Features (16 per problem):
  0 log m, 1 log n, 2 log(p + 1), 3 n/m, 4 p/n, 5 kind (0 LSE, 1 GLS),
  6 complex flag (0), 7 log ||A||_F, 8 log ||B||_F, 9 log ||b||,
  10 log ||d||, 11 log(||A||_F / ||B||_F), 12 log kappa^(A),
  13 log kappa^(B), 14 log kappa^([A; B]), 15 log(flop estimate);
for GLS (n, m, p, W, V, d) the roles are (n, m, p) -> (m, n, p) read as
rows n of W, columns m, V n x p: 0 log n, 1 log m, 2 log(p + 1), 3 m/n,
4 n/p, 7 log ||W||_F, 8 log ||V||_F, 9 log ||d||, 10 0, 11 log(||W||/||V||),
12-14 kappa^ of W, V and [W, V].  Logs are natural, of x clamped to
[1e-300, 1e300].

kappa^(M) = sigma_max(B_k) / sigma_min(B_k) of the k x k bidiagonal of k
steps of Golub-Kahan-Lanczos bidiagonalization of M, in FP64, started from a
given vector, every new vector fully reorthogonalized against the previous
ones (two classical Gram-Schmidt passes), k = min(16, rows, columns) of M;
for a wide M the start vector is first mapped into range(M^T).  The Ritz
values interlace the nonzero singular values, so kappa^ <= sigma_max /
sigma_r (r = rank), with equality once k reaches the rank.  This is the
plain definition of the sketch; the GPU computes it in float32, and the
parity tests derive their tolerance from that rounding.

MLP: 16 -> 64 -> 64 -> 6, ReLU, softmax, cross-entropy; weights are used
as given (the GPU rounds them to bfloat16 before every forward; parity tests
hand the rounded weights to this oracle).
"""
import numpy as np

NF, H1, H2, NC = 16, 64, 64, 6
TINY = 1e-300


# ------------------------------------------------------------- features --

BREAKDOWN = 2.0 ** -40     # relative to the largest alpha / beta so far: far above FP64
                           # rounding (~1e-16 * sqrt(length)), far below any entry of the
                           # bidiagonal of a block with condition number up to 1e12


def gkl_bidiag(mv, rmv, s, k):
    """k steps of Golub-Kahan-Lanczos bidiagonalization: M V_k = U_k B_k with
    B_k upper bidiagonal (diag alpha, superdiag beta), v_1 = s / ||s||.
    mv(x) = M x, rmv(y) = M^T y; u and v are fully reorthogonalized against
    the earlier ones (two classical Gram-Schmidt passes).  Stops early when an
    alpha or beta falls to rounding level (below BREAKDOWN times the largest
    one so far): the Krylov space is exhausted (e.g. k exceeds the rank) and
    further steps would only add rounding noise."""
    v = s / np.linalg.norm(s)
    alphas, betas = [], []
    u_prev, beta = None, 0.0
    big = 0.0
    Us, Vs = [], [v]
    for j in range(k):
        u = mv(v) - (beta * u_prev if u_prev is not None else 0.0)
        if Us:                                 # reorthogonalize (two CGS passes)
            Um = np.column_stack(Us)
            for _ in range(2):
                u = u - Um @ (Um.T @ u)
        a = np.linalg.norm(u)
        if not a > BREAKDOWN * max(big, a if j == 0 else big):
            break
        big = max(big, a)
        u = u / a
        alphas.append(a)
        Us.append(u)
        if j == k - 1:
            break
        w = rmv(u) - a * v
        Vm = np.column_stack(Vs)                # reorthogonalize (two CGS passes)
        for _ in range(2):
            w = w - Vm @ (Vm.T @ w)
        beta = np.linalg.norm(w)
        if not beta > BREAKDOWN * big:
            break
        big = max(big, beta)
        betas.append(beta)
        v = w / beta
        Vs.append(v)
        u_prev = u
    kk = len(alphas)
    Bk = np.diag(alphas)
    for i in range(min(len(betas), kk - 1)):
        Bk[i, i + 1] = betas[i]
    return Bk


def kappa_hat(mv, rmv, s, k=16, wide=False):
    """sigma_max / sigma_min of the GKL bidiagonal.  For a wide M (fewer rows
    than columns) the start vector is first mapped into range(M^T)
    (s <- M^T M s), so that the Ritz values interlace the nonzero singular
    values instead of approaching the null space."""
    if wide:
        s = rmv(mv(s))
    Bk = gkl_bidiag(mv, rmv, s, k)
    if Bk.size == 0:
        return 1.0
    sv = np.linalg.svd(Bk, compute_uv=False)
    return sv[0] / sv[-1] if sv[-1] > 0 else np.inf


def kappa_of(M, s, k):
    """kappa^ of the dense FP64 matrix M (wide when it has fewer rows than
    columns) from start vector s."""
    M = np.asarray(M, np.float64)
    return kappa_hat(lambda x: M @ x, lambda y: M.T @ y, np.asarray(s, np.float64), k,
                     M.shape[0] < M.shape[1])


def _lg(x):
    return float(np.log(min(max(float(x), TINY), 1e300)))


def lse_flops(m, n, p):
    k = min(m, n)
    return 2.0 * n * p * p - 2.0 * p ** 3 / 3.0 + 4.0 * m * n * p + 2.0 * m * n * k - 2.0 * k ** 3 / 3.0


def gls_flops(n, m, p):
    k = min(n, p)
    return 2.0 * n * m * m - 2.0 * m ** 3 / 3.0 + 4.0 * n * m * p + 2.0 * p * n * k - 2.0 * k ** 3 / 3.0


def lse_features(A, B, b, d, s, k=16):
    """Features of LSE (A m x n, B p x n); s: start vector of length n."""
    A, B = np.asarray(A, float), np.asarray(B, float)
    m, n = A.shape
    p = B.shape[0]
    fA, fB = np.linalg.norm(A), np.linalg.norm(B)
    AB = np.vstack([A, B])
    kA = kappa_of(A, s, min(k, m, n))
    kB = kappa_of(B, s, min(k, p, n)) if p else 1.0
    kAB = kappa_of(AB, s, min(k, m + p, n))
    return np.array([_lg(m), _lg(n), np.log(p + 1.0), n / m, p / n, 0.0, 0.0, _lg(fA), _lg(fB),
                     _lg(np.linalg.norm(b)), _lg(np.linalg.norm(d)), _lg(fA) - _lg(fB),
                     _lg(kA), _lg(kB), _lg(kAB), _lg(lse_flops(m, n, p))])


def gls_features(W, V, d, s, k=16):
    """Features of GLS (W n x m, V n x p); s: start vector of length m + p
    (W uses s[:m], V uses s[m:], [W, V] uses s)."""
    W, V = np.asarray(W, float), np.asarray(V, float)
    n, m = W.shape
    p = V.shape[1]
    fW, fV = np.linalg.norm(W), np.linalg.norm(V)
    WV = np.hstack([W, V])
    kW = kappa_of(W, s[:m], min(k, n, m)) if m else 1.0
    kV = kappa_of(V, s[m:], min(k, n, p))
    kWV = kappa_of(WV, s, min(k, n, m + p))
    return np.array([_lg(n), _lg(m), np.log(p + 1.0), m / n, n / p, 1.0, 0.0, _lg(fW), _lg(fV),
                     _lg(np.linalg.norm(d)), 0.0, _lg(fW) - _lg(fV),
                     _lg(kW), _lg(kV), _lg(kWV), _lg(gls_flops(n, m, p))])


# ------------------------------------------------------------------ MLP --

def init_params(seed):
    """He-style initial weights (FP64), seeded."""
    g = np.random.default_rng(seed)
    return dict(W1=g.standard_normal((H1, NF)) * np.sqrt(2.0 / NF), b1=np.zeros(H1),
                W2=g.standard_normal((H2, H1)) * np.sqrt(2.0 / H1), b2=np.zeros(H2),
                W3=g.standard_normal((NC, H2)) * np.sqrt(2.0 / H2), b3=np.zeros(NC))


def forward(P, X):
    """X: (batch, 16) -> probabilities (batch, 6) and the cached activations."""
    X = np.asarray(X, float)
    z1 = X @ P["W1"].T + P["b1"]
    h1 = np.maximum(z1, 0.0)
    z2 = h1 @ P["W2"].T + P["b2"]
    h2 = np.maximum(z2, 0.0)
    z3 = h2 @ P["W3"].T + P["b3"]
    z3 = z3 - z3.max(axis=1, keepdims=True)
    e = np.exp(z3)
    prob = e / e.sum(axis=1, keepdims=True)
    return prob, (X, z1, h1, z2, h2)


def loss(P, X, y):
    prob, _ = forward(P, X)
    return float(-np.mean(np.log(prob[np.arange(len(y)), y])))


def backward(P, X, y):
    """Gradients of the mean cross-entropy with respect to every parameter."""
    prob, (X, z1, h1, z2, h2) = forward(P, X)
    nb = len(y)
    d3 = prob.copy()
    d3[np.arange(nb), y] -= 1.0
    d3 /= nb
    g = dict(W3=d3.T @ h2, b3=d3.sum(axis=0))
    d2 = (d3 @ P["W3"]) * (z2 > 0)
    g["W2"], g["b2"] = d2.T @ h1, d2.sum(axis=0)
    d1 = (d2 @ P["W2"]) * (z1 > 0)
    g["W1"], g["b1"] = d1.T @ X, d1.sum(axis=0)
    return g


def adam_step(P, g, state, lr=1e-3, b1=0.9, b2=0.999, eps=1e-8):
    """One Adam update (bias-corrected), in place; state: dict with t, m, v."""
    state["t"] = state.get("t", 0) + 1
    t = state["t"]
    for k in P:
        m = state.setdefault("m_" + k, np.zeros_like(P[k]))
        v = state.setdefault("v_" + k, np.zeros_like(P[k]))
        m[...] = b1 * m + (1 - b1) * g[k]
        v[...] = b2 * v + (1 - b2) * g[k] ** 2
        mh = m / (1 - b1 ** t)
        vh = v / (1 - b2 ** t)
        P[k] = P[k] - lr * mh / (np.sqrt(vh) + eps)
    return P


def bf16_round(x):
    """Round to the nearest bfloat16 (ties to even), returned as float64."""
    a = np.asarray(x, dtype=np.float32)
    u = a.view(np.uint32).astype(np.uint64)
    r = ((u + 0x7FFF + ((u >> 16) & 1)) >> 16) << 16
    return r.astype(np.uint32).view(np.float32).astype(np.float64)


CLASSES = [("bf16", "classical"), ("bf16", "gmres"), ("fp32", "classical"), ("fp32", "gmres"),
           ("fp64", "classical"), ("fp64", "gmres")]


def label(times, ok, tie=0.03):
    """Class of the fastest configuration among those that passed; within
    `tie` of the fastest, the higher factorization precision, then classical
    IR, wins.  times/ok indexed like CLASSES.  -1 if none passed."""
    cand = [i for i in range(len(CLASSES)) if ok[i]]
    if not cand:
        return -1
    best = min(times[i] for i in cand)
    near = [i for i in cand if times[i] <= best * (1 + tie)]
    prec = {"bf16": 0, "fp32": 1, "fp64": 2}
    return max(near, key=lambda i: (prec[CLASSES[i][0]], CLASSES[i][1] == "classical"))
