"""Seeded synthetic inputs shaped like the paper's test problems.

This module holds no arithmetic of the solver: it only draws matrices with a
prescribed singular spectrum, right-hand sides and batches.  The oracle and
the GPU path both consume exactly the arrays produced here.

Constructions
-------------
* Haar-distributed orthogonal factors: QR of a Gaussian matrix with the signs
  of diag(R) folded into Q (Mezzadri's correction), as the paper draws "the
  unitary factors from the QR factorization of randomly generated matrices"
  (Sec. 6.1).
* ``svd_matrix``: U diag(sigma) V^T with Haar U, V.
* ``lse_paper`` / ``gls_paper``: [A^T, B^T] = W1 Sigma W2 (resp. [W, V]) with a
  prescribed kappa_2, logarithmically spaced singular values (the paper uses
  xLATM1; the spacing mode is not stated, geometric spacing is used here).
* ``zlse_svd`` / ``zgls_svd``: the complex analogues (the paper defines both
  problems over C; Haar unitary factors from the QR of a complex Gaussian
  matrix with the phases of diag(R) folded into Q).
* ``lse_small`` (m=200, n=100, p=20), ``gls_ar1`` (W 4096x1024 with cond 1e3,
  V the Cholesky factor of an AR(1) covariance, rho=0.9), ``lse_large``
  (m=16384, n=8192, p=1024), ``lse_batch`` (uneven batch): the workloads the
  benchmark and the parity tests use.

Every generator takes an integer seed and returns float64 (complex128 for
the z-prefixed ones) arrays in column-major (Fortran) order.
"""
import numpy as np


def rng(seed):
    return np.random.Generator(np.random.PCG64(int(seed)))


def haar(g, rows, cols=None):
    """rows x cols matrix with orthonormal columns, Haar-distributed."""
    cols = rows if cols is None else cols
    X = g.standard_normal((rows, cols))
    Q, R = np.linalg.qr(X)
    s = np.sign(np.diag(R))
    s[s == 0] = 1.0
    return Q * s


def logspace_sigma(k, cond, top=1.0):
    """k singular values from top down to top/cond, geometrically spaced."""
    if k <= 1:
        return np.full(max(k, 0), top)
    return top * np.logspace(0.0, -np.log10(cond), k)


def latm1_sigma(k, cond, mode=3):
    """Singular values with condition number `cond` in the three xLATM1-style
    patterns the paper's generator can produce (the paper does not say which
    one it used): mode 1 one large value (1, 1/cond, ..., 1/cond), mode 2 one
    small value (1, ..., 1, 1/cond), mode 3 geometric spacing."""
    if k <= 1:
        return np.ones(max(k, 0))
    if mode == 1:
        s = np.full(k, 1.0 / cond)
        s[0] = 1.0
        return s
    if mode == 2:
        s = np.ones(k)
        s[-1] = 1.0 / cond
        return s
    return logspace_sigma(k, cond)


def svd_matrix(g, rows, cols, sigma):
    """U diag(sigma) V^T, U rows x r, V cols x r, r = len(sigma)."""
    r = len(sigma)
    U = haar(g, rows, r)
    V = haar(g, cols, r)
    return np.asfortranarray((U * sigma) @ V.T)


# ------------------------------------------------------------------ LSE --

def lse_paper(seed, m, n, p, kappa, mode=3):
    """[A^T, B^T] = W1 Sigma W2 with kappa_2([A; B]) = kappa (Sec. 6.2);
    `mode` selects the singular-value pattern (latm1_sigma)."""
    g = rng(seed)
    sigma = latm1_sigma(n, kappa, mode)
    AB = svd_matrix(g, m + p, n, sigma)
    A = np.asfortranarray(AB[:m])
    B = np.asfortranarray(AB[m:])
    x = g.standard_normal(n)
    b = A @ x + g.standard_normal(m)
    d = B @ x
    return dict(A=A, B=B, b=b, d=d)


def lse_svd(seed, m, n, p, cond_a, cond_b, noise=1.0):
    """A = U diag(logspace) V^T with cond(A) = cond_a, B likewise with
    cond_b; d = B x_true, b = A x_true + noise * N(0,1)."""
    g = rng(seed)
    A = svd_matrix(g, m, n, logspace_sigma(min(m, n), cond_a))
    B = svd_matrix(g, p, n, logspace_sigma(p, cond_b)) if p > 0 else np.zeros((0, n), order="F")
    x = g.standard_normal(n)
    d = B @ x
    b = A @ x + noise * g.standard_normal(m)
    return dict(A=A, B=np.asfortranarray(B), b=b, d=d, x_true=x)


def lse_small(seed=20241623):
    """LSE m=200, n=100, p=20: A = U diag(logspace(0,-2,100)) V^T,
    B = U' diag(logspace(0,-1,20)) V'^T, d = B x_true,
    b = A x_true + 1e-3 r with x_true, r ~ N(0,1)."""
    g = rng(seed)
    m, n, p = 200, 100, 20
    A = svd_matrix(g, m, n, np.logspace(0, -2, n))
    B = svd_matrix(g, p, n, np.logspace(0, -1, p))
    x = g.standard_normal(n)
    d = B @ x
    b = A @ x + 1e-3 * g.standard_normal(m)
    return dict(A=A, B=B, b=b, d=d, x_true=x)


def lse_large(seed=20243623, cond_a=1e4, cond_b=1e2, m=16384, n=8192, p=1024):
    """LSE m=16384, n=8192, p=1024 with cond(A) in {1e1, 1e4, 1e8} and
    cond(B) = 1e2 (same construction as lse_svd, b = A x + N(0,1))."""
    return lse_svd(seed, m, n, p, cond_a, cond_b)


def lse_batch_specs(seed=20244623, count=10000, m_lo=32, m_hi=512, cond_lo=1e1, cond_hi=1e6):
    """(seed, m, n, p, cond(A)) of each problem of the uneven batch:
    m ~ U[m_lo, m_hi], n ~ U[16, m/2], p ~ U[1, n/4], cond(A) log-uniform in
    [cond_lo, cond_hi]."""
    g = rng(seed)
    out = []
    for i in range(count):
        m = int(g.integers(m_lo, m_hi + 1))
        n = int(g.integers(16, max(16, m // 2) + 1))
        p = int(g.integers(1, max(1, n // 4) + 1))
        c = float(np.exp(g.uniform(np.log(cond_lo), np.log(cond_hi))))
        out.append((int(g.integers(1 << 62)), m, n, p, c))
    return out


def lse_batch(seed=20244623, count=10000, m_lo=32, m_hi=512, cond_lo=1e1, cond_hi=1e6, workers=1):
    """Uneven batch: m ~ U[m_lo, m_hi], n ~ U[16, m/2], p ~ U[1, n/4],
    cond(A) log-uniform in [cond_lo, cond_hi], cond(B) = 10 (lse_svd per
    problem with its own seed, so the result does not depend on workers)."""
    specs = lse_batch_specs(seed, count, m_lo, m_hi, cond_lo, cond_hi)

    def one(sp):
        s, m, n, p, c = sp
        return lse_svd(s, m, n, p, c, 10.0)

    if workers <= 1:
        return [one(sp) for sp in specs]
    from concurrent.futures import ThreadPoolExecutor
    with ThreadPoolExecutor(max_workers=workers) as ex:
        return list(ex.map(one, specs))


def lse_svd_torch(seed, m, n, p, cond_a, cond_b, device, noise=1.0):
    """lse_svd's construction drawn with torch's generator on `device` (for
    sizes whose Haar factors are slow to draw on the host): A = U diag(sigma)
    V^T with logspace spectra, d = B x, b = A x + noise N(0,1).  FP64
    column-major tensors (A, B, b, d, x_true)."""
    import torch
    g = torch.Generator(device=device)
    g.manual_seed(int(seed) & ((1 << 63) - 1))

    def haar(rows, cols):
        X = torch.randn(rows, cols, generator=g, device=device, dtype=torch.float64)
        Q, R = torch.linalg.qr(X)
        sg = torch.sign(torch.diagonal(R))
        sg[sg == 0] = 1.0
        return Q * sg

    def svd_m(rows, cols, sigma):
        U = haar(rows, len(sigma))
        V = haar(cols, len(sigma))
        return ((U * sigma) @ V.T).t().contiguous().t()

    sa = torch.from_numpy(logspace_sigma(min(m, n), cond_a)).to(device)
    sb = torch.from_numpy(logspace_sigma(p, cond_b)).to(device)
    A = svd_m(m, n, sa)
    B = svd_m(p, n, sb)
    x = torch.randn(n, generator=g, device=device, dtype=torch.float64)
    b = A @ x + noise * torch.randn(m, generator=g, device=device, dtype=torch.float64)
    return dict(A=A, B=B, b=b, d=B @ x, x_true=x)


def lse_known_torch(seed, m, n, p, cond_a, cond_b, device, resid=1e-3):
    """LSE with a known solution (the known-solution construction of the
    KKT system eq. aug-LSE), drawn with torch's generator on `device`:
    A = U_A diag(sigma) V_A^T (m >= n, logspace spectrum, cond_a),
    B = U_B diag(sigma_B) V_B^T (cond_b), x* ~ N(0,1), and
      r* = U_A Sigma^-1 V_A^T B^T v* + (I - U_A U_A^T) w,
    so that A^T r* = B^T v*; b = A x* + r*, d = B x*.  Then (x*, r*, v*) is
    the solution.  v* and w are scaled so that each part of r* has norm
    resid/2 * sigma_min(A) ||x*||: the rounding of the stored A perturbs the
    multiplier equation by ~u ||A|| ||r*||, which moves x by far less than
    kappa u.  Also returns kappa_up, an upper bound of the forward-error
    condition number kappa_N (1 + kappa_N ||r|| / (sigma_max(T11) ||x||)):
    kappa_N = kappa_2(A restricted to null(B)) <= cond_a (the singular
    values of A N with orthonormal N lie in [sigma_min(A), sigma_max(A)]),
    so kappa_up = cond_a (1 + cond_a ||r*|| / (sigma_max(A) ||x*||)).
    FP64 column-major tensors."""
    import torch
    assert m >= n
    g = torch.Generator(device=device)
    g.manual_seed(int(seed) & ((1 << 63) - 1))
    f64 = dict(generator=g, device=device, dtype=torch.float64)

    def haar(rows, cols):
        X = torch.randn(rows, cols, **f64)
        Q, R = torch.linalg.qr(X)
        sg = torch.sign(torch.diagonal(R))
        sg[sg == 0] = 1.0
        return Q * sg

    sa = torch.from_numpy(logspace_sigma(n, cond_a)).to(device)
    sb = torch.from_numpy(logspace_sigma(p, cond_b)).to(device)
    UA, VA = haar(m, n), haar(n, n)
    UB, VB = haar(p, p), haar(n, p)
    A = ((UA * sa) @ VA.T).t().contiguous().t()
    B = ((UB * sb) @ VB.T).t().contiguous().t()
    x = torch.randn(n, **f64)
    nx = torch.linalg.norm(x)
    tau = 0.5 * resid * float(sa[-1]) * float(nx)
    gv = torch.randn(p, **f64)
    r1 = UA @ ((VA.T @ (B.T @ gv)) / sa)
    s1 = tau / float(torch.linalg.norm(r1))
    v = gv * s1
    r1 = r1 * s1
    w = torch.randn(m, **f64)
    r2 = w - UA @ (UA.T @ w)
    r2 = r2 * (tau / float(torch.linalg.norm(r2)))
    r = r1 + r2
    b = A @ x + r
    d = B @ x
    kup = cond_a * (1.0 + cond_a * float(torch.linalg.norm(r)) / (float(sa[0]) * float(nx)))
    del UA, VA, UB, VB
    return dict(A=A, B=B, b=b, d=d, x_true=x, r_true=r, v_true=v, kappa_up=kup)


def _haar_torch(g, rows, cols, device):
    """rows x cols with orthonormal columns (QR of a Gaussian matrix, the
    signs of diag(R) folded in), drawn with generator g on `device`."""
    import torch
    X = torch.randn(rows, cols, generator=g, device=device, dtype=torch.float64)
    Q, R = torch.linalg.qr(X)
    sg = torch.sign(torch.diagonal(R))
    sg[sg == 0] = 1.0
    return Q * sg


def lse_paper_torch(seed, m, n, p, kappa, device, mode=3):
    """lse_paper drawn on `device` (the Sec. 6.2 shapes are too large for a
    host generator): [A^T, B^T] = W1 Sigma W2 with kappa_2([A; B]) = kappa,
    b = A x + N(0, 1) noise, d = B x.  FP64 column-major tensors."""
    import torch
    g = torch.Generator(device=device)
    g.manual_seed(int(seed) & ((1 << 63) - 1))
    sigma = torch.from_numpy(latm1_sigma(n, kappa, mode)).to(device)
    U = _haar_torch(g, m + p, n, device)
    V = _haar_torch(g, n, n, device)
    AB = (U * sigma) @ V.T
    A = AB[:m].t().contiguous().t()
    B = AB[m:].t().contiguous().t()
    x = torch.randn(n, generator=g, device=device, dtype=torch.float64)
    b = A @ x + torch.randn(m, generator=g, device=device, dtype=torch.float64)
    d = B @ x
    return dict(A=A, B=B, b=b, d=d)


def gls_paper_torch(seed, n, m, p, kappa, device, mode=3):
    """gls_paper drawn on `device`: [W, V] = W1 Sigma W2 with
    kappa_2([W, V]) = kappa (Sec. 6.3), d ~ N(0, 1)."""
    import torch
    g = torch.Generator(device=device)
    g.manual_seed(int(seed) & ((1 << 63) - 1))
    sigma = torch.from_numpy(latm1_sigma(n, kappa, mode)).to(device)
    U = _haar_torch(g, n, n, device)
    V = _haar_torch(g, m + p, n, device)
    WV = (U * sigma) @ V.T
    W = WV[:, :m].t().contiguous().t()
    Vm = WV[:, m:].t().contiguous().t()
    d = torch.randn(n, generator=g, device=device, dtype=torch.float64)
    return dict(W=W, V=Vm, d=d)


def lse_batch_torch(specs, device, cond_b=10.0):
    """The problems of lse_batch_specs drawn with torch's generator on
    `device` (same construction as lse_svd: Haar factors from the QR of
    Gaussian matrices with sign(diag R) folded in, logspace spectra, d = B x,
    b = A x + N(0,1)); fast enough for ten thousand problems.  Returns dicts
    of FP64 column-major tensors (A, B, b, d)."""
    import torch

    def haar(g, rows, cols):
        X = torch.randn(rows, cols, generator=g, device=device, dtype=torch.float64)
        Q, R = torch.linalg.qr(X)
        sg = torch.sign(torch.diagonal(R))
        sg[sg == 0] = 1.0
        return Q * sg

    def svd_m(g, rows, cols, sigma):
        U = haar(g, rows, len(sigma))
        V = haar(g, cols, len(sigma))
        M = (U * sigma) @ V.T
        return M.t().contiguous().t()

    out = []
    for s, m, n, p, c in specs:
        g = torch.Generator(device=device)
        g.manual_seed(s & ((1 << 63) - 1))
        sa = torch.from_numpy(logspace_sigma(min(m, n), c)).to(device)
        sb = torch.from_numpy(logspace_sigma(p, cond_b)).to(device)
        A = svd_m(g, m, n, sa)
        B = svd_m(g, p, n, sb)
        x = torch.randn(n, generator=g, device=device, dtype=torch.float64)
        out.append(dict(A=A, B=B, d=B @ x, b=A @ x + torch.randn(m, generator=g, device=device,
                                                                   dtype=torch.float64)))
    return out


def splitmix_vector(n, seed=0x5EED):
    """x_j = splitmix64(seed + j) (Steele, Lea, Flood 2014) mapped to
    [-1, 1): the start vector of the selector's condition sketch."""
    M = (1 << 64) - 1
    out = np.empty(n)
    for j in range(n):
        z = (seed + j + 0x9E3779B97F4A7C15) & M
        z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & M
        z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & M
        z ^= z >> 31
        out[j] = (z >> 11) * (1.0 / 9007199254740992.0) * 2.0 - 1.0
    return out


def selector_lse_problems(seed, count, m_lo=64, m_hi=400, cond_lo=1e0, cond_hi=1e12):
    """LSE problems for training / evaluating the selector: m ~ U[m_lo, m_hi],
    n ~ U[16, m/2], p ~ U[1, n/4], kappa_2([A; B]) log-uniform in
    [cond_lo, cond_hi] with a random xLATM1-style pattern (lse_paper)."""
    g = rng(seed)
    out = []
    for _ in range(count):
        m = int(g.integers(m_lo, m_hi + 1))
        n = int(g.integers(16, max(16, m // 2) + 1))
        p = int(g.integers(1, max(1, n // 4) + 1))
        c = float(np.exp(g.uniform(np.log(cond_lo), np.log(cond_hi))))
        mode = int(g.integers(1, 4))
        P = lse_paper(int(g.integers(1 << 62)), m, n, p, c, mode)
        P["kappa"] = c
        out.append(P)
    return out


def selector_gls_problems(seed, count, n_lo=64, n_hi=400, cond_lo=1e0, cond_hi=1e12):
    """GLS problems for training / evaluating the selector (xGGGLM
    convention): n ~ U[n_lo, n_hi], m ~ U[8, n/2], p ~ U[n, 5n/4],
    kappa_2([W, V]) log-uniform in [cond_lo, cond_hi] with a random
    xLATM1-style pattern (gls_paper)."""
    g = rng(seed)
    out = []
    for _ in range(count):
        n = int(g.integers(n_lo, n_hi + 1))
        m = int(g.integers(8, max(8, n // 2) + 1))
        p = int(g.integers(n, n + n // 4 + 1))
        c = float(np.exp(g.uniform(np.log(cond_lo), np.log(cond_hi))))
        mode = int(g.integers(1, 4))
        G = gls_paper(int(g.integers(1 << 62)), n, m, p, c, mode)
        G["kappa"] = c
        out.append(G)
    return out


# ------------------------------------------------------------------ GLS --

def ar1_cholesky(n, rho):
    """Lower-triangular Cholesky factor L of Sigma_ij = rho^|i-j| in closed
    form: L[i,0] = rho^i, L[i,j] = rho^(i-j) sqrt(1-rho^2) for 1 <= j <= i."""
    i = np.arange(n)[:, None]
    j = np.arange(n)[None, :]
    L = np.where(i >= j, rho ** np.clip(i - j, 0, None) * np.sqrt(1.0 - rho * rho), 0.0)
    L[:, 0] = rho ** np.arange(n)
    return np.asfortranarray(L)


def gls_ar1(seed=20242623, n=4096, m=1024, cond_w=1e3, rho=0.9):
    """GLS in the xGGGLM convention: W n x m with cond(W) = cond_w (SVD
    construction), V the n x n Cholesky factor of an AR(1) covariance,
    d = W x_true + V y_true with x_true, y_true ~ N(0,1)."""
    g = rng(seed)
    W = svd_matrix(g, n, m, logspace_sigma(m, cond_w))
    V = ar1_cholesky(n, rho)
    x = g.standard_normal(m)
    y = g.standard_normal(n)
    d = W @ x + V @ y
    return dict(W=W, V=V, d=d)


def gls_batch_specs(seed=20245623, count=1000, n_lo=32, n_hi=512, cond_lo=1e1, cond_hi=1e5):
    """(seed, n, m, p, cond(W)) of each problem of an uneven GLS batch in the
    xGGGLM convention: n ~ U[n_lo, n_hi], m ~ U[4, n/2], p ~ U[n, n + n/4]
    (so m <= n <= p), cond(W) log-uniform in [cond_lo, cond_hi]."""
    g = rng(seed)
    out = []
    for _ in range(count):
        n = int(g.integers(n_lo, n_hi + 1))
        m = int(g.integers(4, max(4, n // 2) + 1))
        p = int(g.integers(n, n + n // 4 + 1))
        c = float(np.exp(g.uniform(np.log(cond_lo), np.log(cond_hi))))
        out.append((int(g.integers(1 << 62)), n, m, p, c))
    return out


def gls_batch(seed=20245623, count=1000, **kw):
    """The problems of gls_batch_specs: W with cond(W) (SVD construction),
    V with cond(V) = 10, d = W x + V y (gls_svd per problem, own seed)."""
    return [gls_svd(s, n, m, p, c, 10.0) for s, n, m, p, c in gls_batch_specs(seed, count, **kw)]


def gls_batch_torch(specs, device, cond_v=10.0):
    """gls_batch_specs problems drawn with torch's generator on `device`
    (the construction of gls_svd): dicts of FP64 column-major W, V, d."""
    import torch

    def haar(g, rows, cols):
        X = torch.randn(rows, cols, generator=g, device=device, dtype=torch.float64)
        Q, R = torch.linalg.qr(X)
        sg = torch.sign(torch.diagonal(R))
        sg[sg == 0] = 1.0
        return Q * sg

    def svd_m(g, rows, cols, sigma):
        U = haar(g, rows, len(sigma))
        V = haar(g, cols, len(sigma))
        return ((U * sigma) @ V.T).t().contiguous().t()

    out = []
    for s, n, m, p, c in specs:
        g = torch.Generator(device=device)
        g.manual_seed(s & ((1 << 63) - 1))
        W = svd_m(g, n, m, torch.from_numpy(logspace_sigma(m, c)).to(device))
        V = svd_m(g, n, p, torch.from_numpy(logspace_sigma(min(n, p), cond_v)).to(device))
        x = torch.randn(m, generator=g, device=device, dtype=torch.float64)
        y = torch.randn(p, generator=g, device=device, dtype=torch.float64)
        out.append(dict(W=W, V=V, d=W @ x + V @ y))
    return out


def gls_paper(seed, n, m, p, kappa, mode=3):
    """[W, V] = W1 Sigma W2 with kappa_2([W, V]) = kappa (Sec. 6.3)."""
    g = rng(seed)
    sigma = latm1_sigma(n, kappa, mode)
    WV = svd_matrix(g, n, m + p, sigma)
    W = np.asfortranarray(WV[:, :m])
    V = np.asfortranarray(WV[:, m:])
    d = g.standard_normal(n)
    return dict(W=W, V=V, d=d)


def gls_svd(seed, n, m, p, cond_w, cond_v):
    """W n x m with cond_w, V n x p with cond_v, d = W x + V y."""
    g = rng(seed)
    W = svd_matrix(g, n, m, logspace_sigma(m, cond_w))
    V = svd_matrix(g, n, p, logspace_sigma(min(n, p), cond_v))
    x = g.standard_normal(m)
    y = g.standard_normal(p)
    d = W @ x + V @ y
    return dict(W=W, V=V, d=d)


# ---------------------------------------------------------------- complex --

def zhaar(g, rows, cols=None):
    """rows x cols matrix with orthonormal columns, Haar-distributed over C
    (QR of a complex Gaussian matrix, the phases of diag(R) folded into Q)."""
    cols = rows if cols is None else cols
    X = (g.standard_normal((rows, cols)) + 1j * g.standard_normal((rows, cols))) / np.sqrt(2.0)
    Q, R = np.linalg.qr(X)
    dg = np.diag(R)
    ph = np.where(np.abs(dg) > 0, dg / np.where(np.abs(dg) > 0, np.abs(dg), 1.0), 1.0)
    return Q * ph


def zsvd_matrix(g, rows, cols, sigma):
    """U diag(sigma) V^H with Haar unitary U (rows x r), V (cols x r)."""
    r = len(sigma)
    U = zhaar(g, rows, r)
    V = zhaar(g, cols, r)
    return np.asfortranarray((U * sigma) @ V.conj().T)


def zgauss(g, k):
    return (g.standard_normal(k) + 1j * g.standard_normal(k)) / np.sqrt(2.0)


def zlse_svd(seed, m, n, p, cond_a, cond_b, noise=1.0):
    """Complex LSE: A = U diag(logspace) V^H with cond(A) = cond_a, B
    likewise with cond_b; d = B x_true, b = A x_true + noise * CN(0,1)."""
    g = rng(seed)
    A = zsvd_matrix(g, m, n, logspace_sigma(min(m, n), cond_a))
    B = (zsvd_matrix(g, p, n, logspace_sigma(p, cond_b)) if p > 0
         else np.zeros((0, n), dtype=np.complex128, order="F"))
    x = zgauss(g, n)
    d = B @ x
    b = A @ x + noise * zgauss(g, m)
    return dict(A=A, B=np.asfortranarray(B), b=b, d=d, x_true=x)


def zgls_svd(seed, n, m, p, cond_w, cond_v):
    """Complex GLS: W n x m with cond_w, V n x p with cond_v, d = W x + V y."""
    g = rng(seed)
    W = zsvd_matrix(g, n, m, logspace_sigma(m, cond_w))
    V = zsvd_matrix(g, n, p, logspace_sigma(min(n, p), cond_v))
    x = zgauss(g, m)
    y = zgauss(g, p)
    d = W @ x + V @ y
    return dict(W=W, V=V, d=d)
