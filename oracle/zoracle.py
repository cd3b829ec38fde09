"""Complex LSE / GLS -- CPU oracle.

TEST INFRASTRUCTURE ONLY (see oracle/__init__.py): only ``tests/``,
``__graft_entry__.smoke()`` and ``bench.py``'s CPU legs may use it.

The paper states both problems over the complex field (Sec. 1: A in C^{m x n},
B in C^{p x n}; W in C^{n x m}, V in C^{n x p}) with conjugate transposes
throughout.  This module restates the method in complex arithmetic with plain
numpy: dense explicit unitary factors, matrix products and triangular solves
as library primitives, one Householder reflector at a time.

* ``zhouse``                -- one Householder reflector, H = I - tau v v^H,
                               H^H (alpha; x) = (beta; 0) with beta real,
                               beta = -sign(Re alpha) ||(alpha; x)|| (the
                               xLARFG convention of LAPACK's complex QR)
* ``zqr`` / ``zrq``         -- unblocked QR, and RQ as the QR of the reversed
                               conjugate transpose (C = T Z)
* ``zlse_factor``           -- GRQ (Lemma 4.5): B = [0, R] Q, A Q^H = Z T
* ``zgls_factor``           -- GQR (Lemma 4.6): W = Q [R; 0], Q^H V = T Z
* ``zlse_nullspace``        -- Sec. 2.1;  ``zgls_paige`` -- Sec. 2.2
* ``zlse_init_v`` / ``zgls_init_z`` -- the multipliers (Sec. 3.1 / 3.2,
                               z0 = Q [0; h] as in the real oracle)
* ``zlse_correction`` / ``zgls_correction`` -- Alg. 1 / Alg. 3, with the
                               readings used by the real path: Dz = -Q h and
                               T22 g2 = u2 in Alg. 3
* ``zlse_solve`` / ``zgls_solve`` -- Alg. 2 / Alg. 4 (complex128 residuals,
                               the eq. lse-stop / gls-stop test)
* ``zlse_truth`` / ``zgls_truth`` -- the plain definition: the KKT systems
                               (eq. aug-LSE / aug-GLS) solved in complex128 and
                               refined with extended-precision residuals
* ``zlse_metrics`` / ``zgls_metrics`` -- stop ratios and err-1 (Tables 4, 5)
* ``ZLseBD`` / ``ZGlsBD`` / ``zgmres`` / ``zlse_gmres_ir`` / ``zgls_gmres_ir``
                            -- GMRES-IR (Sec. 5) with the block-diagonal split
                               preconditioners, conjugate transposes throughout

Factors are computed in complex64 (fact='fp32') or complex128 ('fp64').
Pins: tests/test_oracle_complex.py.
"""
import numpy as np
from scipy.linalg import solve_triangular

_CT = {"fp32": np.complex64, "fp64": np.complex128}
_EXT = np.clongdouble                     # residual precision of the truth


def _h(M):
    return M.conj().T


def _flip(M):
    return M[::-1, ::-1]


# ------------------------------------------------------------ Householder --

def zhouse(alpha, x):
    """(tau, v, beta): v = (1; v_tail), H = I - tau v v^H, H^H (alpha; x) =
    (beta; 0), beta real.  tau = 0 (H = I) when x = 0 and alpha is real."""
    dt = np.result_type(alpha, x, np.complex64)
    xn = np.linalg.norm(x) if len(x) else 0.0
    if xn == 0 and np.imag(alpha) == 0:
        return dt.type(0), np.concatenate([[1], np.zeros(len(x))]).astype(dt), np.real(alpha)
    beta = -np.copysign(np.hypot(abs(alpha), xn), np.real(alpha))
    tau = (beta - alpha) / beta
    v = np.concatenate([[1], x / (alpha - beta)]).astype(dt)
    return dt.type(tau), v, beta


def zqr(A):
    """A (r x c) = Q [R; 0]: Q = H_1 ... H_k (r x r unitary), R upper
    trapezoidal (r x c), in A's precision."""
    R = np.array(A, copy=True)
    r, c = R.shape
    Q = np.eye(r, dtype=R.dtype)
    for j in range(min(r, c)):
        tau, v, beta = zhouse(R[j, j], R[j + 1:, j])
        # H^H applied to the remaining columns, H accumulated on the right of Q
        R[j:, j:] -= np.conj(tau) * np.outer(v, v.conj() @ R[j:, j:])
        R[j, j] = beta
        R[j + 1:, j] = 0
        Q[:, j:] -= tau * np.outer(Q[:, j:] @ v, v.conj())
    return Q, R


def zrq(C):
    """C (r x c, r <= c) = [0, T] Z with T upper triangular r x r and Z
    c x c unitary; for r > c, C = T Z with T upper trapezoidal.  Computed as
    the QR factorization of the reversed conjugate transpose:
    P C^H P = Q~ R~  gives  Z = P Q~^H P,  T = P R~^H P."""
    Qt, Rt = zqr(_flip(_h(C)))
    return _flip(_h(Rt)), _flip(_h(Qt))


# ------------------------------------------------------------------ LSE --

def zlse_factor(A, B, fact="fp32"):
    """GRQ (Lemma 4.5): B = [0, R] Q (R p x p upper triangular, Q n x n),
    A Q^H = Z T (Z m x m, T m x n upper trapezoidal)."""
    dt = _CT[fact]
    A, B = np.asarray(A, dt), np.asarray(B, dt)
    m, n = A.shape
    p = B.shape[0]
    if p:
        T0, Q = zrq(B)
        R = T0[:, n - p:]
    else:
        Q, R = np.eye(n, dtype=dt), np.zeros((0, 0), dt)
    Z, T = zqr(A @ _h(Q))
    return dict(kind="lse", m=m, n=n, p=p, Q=Q, R=R, Z=Z, T=T, dt=dt)


def zlse_nullspace(F, b, d):
    """Sec. 2.1: y = Q x, R y2 = d, T11 y1 = (Z^H b)_1 - T12 y2, x = Q^H y."""
    dt, m, n, p = F["dt"], F["m"], F["n"], F["p"]
    q = n - p
    T, R = F["T"], F["R"]
    c = _h(F["Z"]) @ np.asarray(b, dt)
    y2 = solve_triangular(R, np.asarray(d, dt)) if p else np.zeros(0, dt)
    y1 = solve_triangular(T[:q, :q], c[:q] - T[:q, q:] @ y2) if q else np.zeros(0, dt)
    return (_h(F["Q"]) @ np.concatenate([y1, y2])).astype(np.complex128)


def zlse_init_v(F, A, r):
    """R^H v = (Q A^H r)(n-p+1:n) (Sec. 3.1), A^H r in complex128."""
    dt, n, p = F["dt"], F["n"], F["p"]
    if not p:
        return np.zeros(0, np.complex128)
    t = F["Q"] @ (_h(np.asarray(A, np.complex128)) @ r).astype(dt)
    return solve_triangular(_h(F["R"]), t[n - p:], lower=True).astype(np.complex128)


def zlse_correction(F, f1, f2, f3):
    """Alg. 1 on  [I 0 A; 0 0 B; A^H B^H 0] [dr; -dv; dx] = [f1; f2; f3]:
    u = Q f3, w = Z^H f1, R y2 = f2, T11^H q1 = u1, T11 y1 = w1 - q1 - T12 y2,
    q2 = w2 - T22 y2, R^H dv = T12^H q1 + T22^H q2 - u2, dr = Z q, dx = Q^H y."""
    dt, m, n, p = F["dt"], F["m"], F["n"], F["p"]
    q = n - p
    T, R, Q, Z = F["T"], F["R"], F["Q"], F["Z"]
    u = Q @ np.asarray(f3, dt)
    w = _h(Z) @ np.asarray(f1, dt)
    y2 = solve_triangular(R, np.asarray(f2, dt)) if p else np.zeros(0, dt)
    q1 = solve_triangular(_h(T[:q, :q]), u[:q], lower=True) if q else np.zeros(0, dt)
    y1 = solve_triangular(T[:q, :q], w[:q] - q1 - T[:q, q:] @ y2) if q else np.zeros(0, dt)
    q2 = w[q:] - T[q:, q:] @ y2
    dv = (solve_triangular(_h(R), _h(T[:q, q:]) @ q1 + _h(T[q:, q:]) @ q2 - u[q:], lower=True)
          if p else np.zeros(0, dt))
    dr = Z @ np.concatenate([q1, q2])
    dx = _h(Q) @ np.concatenate([y1, y2])
    return dr.astype(np.complex128), dv.astype(np.complex128), dx.astype(np.complex128)


def zlse_residual(A, B, b, d, x, r, v, ext=False):
    """f1 = b - r - A x, f2 = d - B x, f3 = -A^H r + B^H v (eq. aug-LSE)."""
    t = _EXT if ext else np.complex128
    A, B = np.asarray(A, t), np.asarray(B, t)
    b, d, x, r, v = (np.asarray(z, t) for z in (b, d, x, r, v))
    return b - r - A @ x, d - B @ x, -_h(A) @ r + _h(B) @ v


def _lse_ratios(A, B, b, d, x, r, v, f):
    nA, nB = np.linalg.norm(A), np.linalg.norm(B)
    nr = lambda z: float(np.linalg.norm(np.asarray(z, np.complex128)))
    den = [nr(b) + nr(r) + nA * nr(x), nr(d) + nB * nr(x), nA * nr(r) + nB * nr(v)]
    return [nr(fi) / di if di else 0.0 for fi, di in zip(f, den)]


def zlse_solve(A, B, b, d, fact="fp32", tol=2e-15, maxit=40):
    """Alg. 2: factor once at fact, null-space start, multipliers, then
    classical IR with complex128 residuals and Alg. 1 corrections; stops on
    eq. lse-stop or after maxit steps (status 0 converged, 3 not)."""
    A, B = np.asarray(A, np.complex128), np.asarray(B, np.complex128)
    F = zlse_factor(A, B, fact)
    x = zlse_nullspace(F, b, d)
    r = np.asarray(b, np.complex128) - A @ x
    v = zlse_init_v(F, A, r)
    status, ratios, it = 3, [np.inf] * 3, 0
    for it in range(maxit):
        f = zlse_residual(A, B, b, d, x, r, v)
        ratios = _lse_ratios(A, B, b, d, x, r, v, f)
        if max(ratios) <= tol:
            status = 0
            break
        dr, dv, dx = zlse_correction(F, *f)
        r, v, x = r + dr, v + dv, x + dx
    return dict(x=x, r=r, v=v, status=status, iters=it, ratios=ratios)


def zlse_kkt(A, B):
    """The eq. aug-LSE matrix for the unknown [r; -v; x]."""
    A, B = np.asarray(A, np.complex128), np.asarray(B, np.complex128)
    m, n = A.shape
    p = B.shape[0]
    K = np.zeros((m + p + n, m + p + n), np.complex128)
    K[:m, :m] = np.eye(m)
    K[:m, m + p:] = A
    K[m:m + p, m + p:] = B
    K[m + p:, :m] = _h(A)
    K[m + p:, m:m + p] = _h(B)
    return K


def zlse_truth(A, B, b, d, steps=3):
    """The LSE solution (x, r, v) to about u: the KKT system solved in
    complex128 and refined with extended-precision residuals."""
    A, B = np.asarray(A, np.complex128), np.asarray(B, np.complex128)
    m, n = A.shape
    p = B.shape[0]
    K = zlse_kkt(A, B)
    rhs = np.concatenate([np.asarray(b, np.complex128), np.asarray(d, np.complex128), np.zeros(n)])
    s = np.linalg.solve(K, rhs)
    Ke, re = K.astype(_EXT), rhs.astype(_EXT)
    for _ in range(steps):
        s = s + np.linalg.solve(K, (re - Ke @ s.astype(_EXT)).astype(np.complex128))
    return dict(r=s[:m], v=-s[m:m + p], x=s[m + p:])


def zlse_metrics(A, B, b, d, x, r, v):
    """eq. lse-stop ratios from extended-precision residuals, and err-1 =
    ||B x - d|| / (||B||_F ||x|| + ||d||) (Table 4)."""
    f = zlse_residual(A, B, b, d, x, r, v, ext=True)
    ratios = _lse_ratios(A, B, b, d, x, r, v, f)
    nB = np.linalg.norm(B)
    e_con = float(np.linalg.norm(np.asarray(f[1], np.complex128))) / (
        nB * np.linalg.norm(x) + np.linalg.norm(d) or 1.0)
    return dict(eta=max(ratios), ratios=ratios, e_con=e_con)


# ------------------------------------------------------------------ GLS --

def zgls_factor(W, V, fact="fp32"):
    """GQR (Lemma 4.6): W = Q [R; 0] (Q n x n, R m x m upper triangular),
    Q^H V = T Z (T n x p upper trapezoidal, Z p x p)."""
    dt = _CT[fact]
    W, V = np.asarray(W, dt), np.asarray(V, dt)
    n, m = W.shape
    p = V.shape[1]
    Q, Rf = zqr(W)
    T, Z = zrq(_h(Q) @ V)
    return dict(kind="gls", n=n, m=m, p=p, Q=Q, R=Rf[:m, :m], T=T, Z=Z, dt=dt)


def _gls_blocks(F):
    n, m, p = F["n"], F["m"], F["p"]
    k = n - m                              # order of T22
    o = p - k                              # columns of T11
    T = F["T"]
    return k, o, T[:m, :o], T[:m, o:], T[m:, o:]


def zgls_paige(F, d):
    """Sec. 2.2: c = Q^H d, T22 s2 = c2, R x = c1 - T12 s2, y = Z^H [0; s2]
    (the minimum-norm y)."""
    dt, n, m, p = F["dt"], F["n"], F["m"], F["p"]
    k, o, T11, T12, T22 = _gls_blocks(F)
    c = _h(F["Q"]) @ np.asarray(d, dt)
    s2 = solve_triangular(T22, c[m:]) if k else np.zeros(0, dt)
    x = solve_triangular(F["R"], c[:m] - T12 @ s2) if m else np.zeros(0, dt)
    y = _h(F["Z"]) @ np.concatenate([np.zeros(o, dt), s2])
    return x.astype(np.complex128), y.astype(np.complex128)


def zgls_init_z(F, y):
    """z0 = Q [0; h], T22^H h = (Z y)(p-n+m+1:p) (Sec. 3.2)."""
    dt, n, m = F["dt"], F["n"], F["m"]
    k, o, T11, T12, T22 = _gls_blocks(F)
    t = F["Z"] @ np.asarray(y, dt)
    h = solve_triangular(_h(T22), t[o:], lower=True) if k else np.zeros(0, dt)
    return (F["Q"] @ np.concatenate([np.zeros(m, dt), h])).astype(np.complex128)


def zgls_correction(F, f1, f2, f3):
    """Alg. 3 on  [I V^H 0; V 0 W; 0 W^H 0] [dy; -dz; dx] = [f1; f2; f3]:
    u = Q^H f2, w = Z f1, R^H h1 = f3, T22 g2 = u2,
    T22^H h2 = w2 - g2 - T12^H h1, g1 = w1 - T11^H h1,
    R dx = u1 - T11 g1 - T12 g2, dy = Z^H g, dz = -Q h."""
    dt, n, m, p = F["dt"], F["n"], F["m"], F["p"]
    k, o, T11, T12, T22 = _gls_blocks(F)
    R, Q, Z = F["R"], F["Q"], F["Z"]
    u = _h(Q) @ np.asarray(f2, dt)
    w = Z @ np.asarray(f1, dt)
    h1 = solve_triangular(_h(R), np.asarray(f3, dt), lower=True) if m else np.zeros(0, dt)
    g2 = solve_triangular(T22, u[m:]) if k else np.zeros(0, dt)
    h2 = solve_triangular(_h(T22), w[o:] - g2 - _h(T12) @ h1, lower=True) if k else np.zeros(0, dt)
    g1 = w[:o] - _h(T11) @ h1
    dx = solve_triangular(R, u[:m] - T11 @ g1 - T12 @ g2) if m else np.zeros(0, dt)
    dy = _h(Z) @ np.concatenate([g1, g2])
    dz = -(Q @ np.concatenate([h1, h2]))
    return dy.astype(np.complex128), dz.astype(np.complex128), dx.astype(np.complex128)


def zgls_residual(W, V, d, x, y, z, ext=False):
    """f1 = -y + V^H z, f2 = d - W x - V y, f3 = W^H z (eq. aug-GLS)."""
    t = _EXT if ext else np.complex128
    W, V = np.asarray(W, t), np.asarray(V, t)
    d, x, y, z = (np.asarray(a, t) for a in (d, x, y, z))
    return -y + _h(V) @ z, d - W @ x - V @ y, _h(W) @ z


def _gls_ratios(W, V, d, x, y, z, f):
    nW, nV = np.linalg.norm(W), np.linalg.norm(V)
    nr = lambda a: float(np.linalg.norm(np.asarray(a, np.complex128)))
    den = [nr(y) + nV * nr(z), nr(d) + nW * nr(x) + nV * nr(y), nW * nr(z)]
    return [nr(fi) / di if di else 0.0 for fi, di in zip(f, den)]


def zgls_solve(W, V, d, fact="fp32", tol=2e-15, maxit=40):
    """Alg. 4: factor once at fact, Paige's start, z0, then classical IR
    with complex128 residuals and Alg. 3 corrections."""
    W, V = np.asarray(W, np.complex128), np.asarray(V, np.complex128)
    F = zgls_factor(W, V, fact)
    x, y = zgls_paige(F, d)
    z = zgls_init_z(F, y)
    status, ratios, it = 3, [np.inf] * 3, 0
    for it in range(maxit):
        f = zgls_residual(W, V, d, x, y, z)
        ratios = _gls_ratios(W, V, d, x, y, z, f)
        if max(ratios) <= tol:
            status = 0
            break
        dy, dz, dx = zgls_correction(F, *f)
        y, z, x = y + dy, z + dz, x + dx
    return dict(x=x, y=y, z=z, status=status, iters=it, ratios=ratios)


def zgls_kkt(W, V):
    """The eq. aug-GLS matrix for the unknown [y; -z; x]."""
    W, V = np.asarray(W, np.complex128), np.asarray(V, np.complex128)
    n, m = W.shape
    p = V.shape[1]
    K = np.zeros((p + n + m, p + n + m), np.complex128)
    K[:p, :p] = np.eye(p)
    K[:p, p:p + n] = _h(V)
    K[p:p + n, :p] = V
    K[p:p + n, p + n:] = W
    K[p + n:, p:p + n] = _h(W)
    return K


def zgls_truth(W, V, d, steps=3):
    """The GLS solution (x, minimum-norm y, z) to about u, as zlse_truth."""
    W, V = np.asarray(W, np.complex128), np.asarray(V, np.complex128)
    n, m = W.shape
    p = V.shape[1]
    K = zgls_kkt(W, V)
    rhs = np.concatenate([np.zeros(p), np.asarray(d, np.complex128), np.zeros(m)])
    s = np.linalg.solve(K, rhs)
    Ke, re = K.astype(_EXT), rhs.astype(_EXT)
    for _ in range(steps):
        s = s + np.linalg.solve(K, (re - Ke @ s.astype(_EXT)).astype(np.complex128))
    return dict(y=s[:p], z=-s[p:p + n], x=s[p + n:])


def zgls_metrics(W, V, d, x, y, z):
    """eq. gls-stop ratios from extended-precision residuals, and err-1 =
    ||W x + V y - d|| / (||W||_F ||x|| + ||V||_F ||y|| + ||d||) (Table 5)."""
    f = zgls_residual(W, V, d, x, y, z, ext=True)
    ratios = _gls_ratios(W, V, d, x, y, z, f)
    den = np.linalg.norm(W) * np.linalg.norm(x) + np.linalg.norm(V) * np.linalg.norm(y) + np.linalg.norm(d)
    e_con = float(np.linalg.norm(np.asarray(f[1], np.complex128))) / (den or 1.0)
    return dict(eta=max(ratios), ratios=ratios, e_con=e_con)


# ------------------------------------------------------------ GMRES-IR --
# Sec. 5 over C: the scaled augmented matrices F~(alpha, beta), the
# block-diagonal split preconditioners with conjugate transposes
# (eq. lse-bdpre-mlarge, m >= n; eq. gls-bdpre-plarge, n <= p), restarted
# GMRES in complex128, and the outer refinement loop.

class ZLseBD:
    """F~ = [a I 0 A; 0 0 b B; A^H b B^H 0],
    M_l = diag(a^-1/2 I, a^-1/2 b^-1 Y R^-1, a^1/2 T1^-H Q),
    M_r = diag(a^-1/2 I, a^-1/2 b^-1 R^-H Y^H, a^1/2 Q^H T1^-1),
    T1 the leading n x n block of T, Y = T1(n-p+1:n, n-p+1:n) (m >= n)."""

    def __init__(self, F, A, B, alpha, beta):
        m, n, p = F["m"], F["n"], F["p"]
        if m < n:
            raise ValueError("eq. lse-bdpre-mlarge needs m >= n")
        self.m, self.n, self.p = m, n, p
        self.A, self.B = np.asarray(A, np.complex128), np.asarray(B, np.complex128)
        self.Q = np.asarray(F["Q"], np.complex128)
        self.R = np.asarray(F["R"], np.complex128)
        self.T1 = np.asarray(F["T"], np.complex128)[:n, :n]
        self.Y = self.T1[n - p:, n - p:]
        self.a, self.b = alpha, beta

    def split(self, u):
        return u[:self.m], u[self.m:self.m + self.p], u[self.m + self.p:]

    def Fmul(self, u):
        u1, u2, u3 = self.split(u)
        return np.concatenate([self.a * u1 + self.A @ u3, self.b * (self.B @ u3),
                               _h(self.A) @ u1 + self.b * (_h(self.B) @ u2)])

    def Ml(self, u):
        u1, u2, u3 = self.split(u)
        a, b = self.a, self.b
        o2 = self.Y @ solve_triangular(self.R, u2) if self.p else u2
        o3 = solve_triangular(_h(self.T1), self.Q @ u3, lower=True)
        return np.concatenate([a ** -0.5 * u1, a ** -0.5 / b * o2, a ** 0.5 * o3])

    def Mr(self, t):
        t1, t2, t3 = self.split(t)
        a, b = self.a, self.b
        o2 = solve_triangular(_h(self.R), _h(self.Y) @ t2, lower=True) if self.p else t2
        o3 = _h(self.Q) @ solve_triangular(self.T1, t3)
        return np.concatenate([a ** -0.5 * t1, a ** -0.5 / b * o2, a ** 0.5 * o3])


class ZGlsBD:
    """F~ = [a I V^H 0; V 0 b W; 0 b W^H 0],
    M_l = diag(a^-1/2 I, a^1/2 T2^-1 Q^H, a^-1/2 b^-1 S^H R^-H),
    M_r = diag(a^-1/2 I, a^1/2 Q T2^-H, a^-1/2 b^-1 R^-1 S),
    T = [0, T2] (n <= p), S = T2(1:m, 1:m)."""

    def __init__(self, F, W, V, alpha, beta):
        n, m, p = F["n"], F["m"], F["p"]
        if n > p:
            raise ValueError("eq. gls-bdpre-plarge needs n <= p")
        self.n, self.m, self.p = n, m, p
        self.W, self.V = np.asarray(W, np.complex128), np.asarray(V, np.complex128)
        self.Q = np.asarray(F["Q"], np.complex128)
        self.R = np.asarray(F["R"], np.complex128)
        self.T2 = np.asarray(F["T"], np.complex128)[:, p - n:]
        self.S = self.T2[:m, :m]
        self.a, self.b = alpha, beta

    def split(self, u):
        return u[:self.p], u[self.p:self.p + self.n], u[self.p + self.n:]

    def Fmul(self, u):
        u1, u2, u3 = self.split(u)
        return np.concatenate([self.a * u1 + _h(self.V) @ u2, self.V @ u1 + self.b * (self.W @ u3),
                               self.b * (_h(self.W) @ u2)])

    def Ml(self, u):
        u1, u2, u3 = self.split(u)
        a, b = self.a, self.b
        o2 = solve_triangular(self.T2, _h(self.Q) @ u2)
        o3 = _h(self.S) @ solve_triangular(_h(self.R), u3, lower=True) if self.m else u3
        return np.concatenate([a ** -0.5 * u1, a ** 0.5 * o2, a ** -0.5 / b * o3])

    def Mr(self, t):
        t1, t2, t3 = self.split(t)
        a, b = self.a, self.b
        o2 = self.Q @ solve_triangular(_h(self.T2), t2, lower=True)
        o3 = solve_triangular(self.R, self.S @ t3) if self.m else t3
        return np.concatenate([a ** -0.5 * t1, a ** 0.5 * o2, a ** -0.5 / b * o3])


def zgmres(op, rhs, tol=1e-8, restart=30, maxit=300):
    """Restarted GMRES(restart) in complex128 from x0 = 0: modified
    Gram-Schmidt Arnoldi with Hermitian inner products; the small
    least-squares problem min ||beta e1 - H y|| by a library solve.
    Returns (x, iterations, relative residual)."""
    rhs = np.asarray(rhs, np.complex128)
    nb = np.linalg.norm(rhs)
    x = np.zeros_like(rhs)
    if nb == 0:
        return x, 0, 0.0
    total, rel = 0, 1.0
    r = rhs.copy()
    while total < maxit:
        beta0 = np.linalg.norm(r)
        if beta0 <= tol * nb:
            break
        Vb = [r / beta0]
        H = np.zeros((restart + 1, restart), np.complex128)
        e1 = np.zeros(restart + 1, np.complex128)
        e1[0] = beta0
        y = np.zeros(0, np.complex128)
        for j in range(restart):
            w = op(Vb[j])
            total += 1
            for i in range(j + 1):
                H[i, j] = np.vdot(Vb[i], w)
                w = w - H[i, j] * Vb[i]
            H[j + 1, j] = np.linalg.norm(w)
            Vb.append(w / H[j + 1, j] if H[j + 1, j] != 0 else w)
            y = np.linalg.lstsq(H[:j + 2, :j + 1], e1[:j + 2], rcond=None)[0]
            res = np.linalg.norm(e1[:j + 2] - H[:j + 2, :j + 1] @ y)
            if res <= tol * nb or total >= maxit:
                break
        x = x + np.column_stack(Vb[:len(y)]) @ y
        r = rhs - op(x)
        rel = np.linalg.norm(r) / nb
        if rel <= tol:
            break
    return x, total, rel


def zlse_gmres_ir(A, B, b, d, fact="fp32", tol=2e-15, maxit=40, restart=30, inner_tol=1e-8, inner_maxit=300,
                  beta=1.0):
    """Complex LSE GMRES-IR (m >= n), the readings of the real oracle:
    alpha = max(||r0||, sqrt(u) ||A||_F ||x0||), beta = 1."""
    A, B = np.asarray(A, np.complex128), np.asarray(B, np.complex128)
    b, d = np.asarray(b, np.complex128), np.asarray(d, np.complex128)
    F = zlse_factor(A, B, fact)
    x = zlse_nullspace(F, b, d)
    r = b - A @ x
    v = zlse_init_v(F, A, r)
    u = np.finfo(np.float64).eps / 2
    alpha = max(np.linalg.norm(r), np.sqrt(u) * np.linalg.norm(A) * np.linalg.norm(x)) or 1.0
    P = ZLseBD(F, A, B, alpha, beta)
    op = lambda t: P.Ml(P.Fmul(P.Mr(t)))
    status, inner, ratios, it = 3, 0, [np.inf] * 3, 0
    a, bb = alpha, beta
    for it in range(maxit):
        f = zlse_residual(A, B, b, d, x, r, v)
        ratios = _lse_ratios(A, B, b, d, x, r, v, f)
        if max(ratios) <= tol:
            status = 0
            break
        rhs = np.concatenate([a ** 0.5 * f[0], a ** 0.5 * bb * f[1], a ** -0.5 * f[2]])
        t, k, _ = zgmres(op, P.Ml(rhs), inner_tol, restart, inner_maxit)
        inner += k
        d1, d2, d3 = P.split(P.Mr(t))
        r, v, x = r + a ** 0.5 * d1, v - a ** 0.5 * bb * d2, x + a ** -0.5 * d3
    return dict(x=x, r=r, v=v, status=status, iters=it, inner_iters=inner, ratios=ratios, alpha=alpha)


def zgls_gmres_ir(W, V, d, fact="fp32", tol=2e-15, maxit=40, restart=30, inner_tol=1e-8, inner_maxit=300,
                  beta=1.0):
    """Complex GLS GMRES-IR (n <= p): alpha = max(||y0||, sqrt(u) ||V||_F ||z0||)."""
    W, V = np.asarray(W, np.complex128), np.asarray(V, np.complex128)
    d = np.asarray(d, np.complex128)
    F = zgls_factor(W, V, fact)
    x, y = zgls_paige(F, d)
    z = zgls_init_z(F, y)
    u = np.finfo(np.float64).eps / 2
    alpha = max(np.linalg.norm(y), np.sqrt(u) * np.linalg.norm(V) * np.linalg.norm(z)) or 1.0
    P = ZGlsBD(F, W, V, alpha, beta)
    op = lambda t: P.Ml(P.Fmul(P.Mr(t)))
    status, inner, ratios, it = 3, 0, [np.inf] * 3, 0
    a, bb = alpha, beta
    for it in range(maxit):
        f = zgls_residual(W, V, d, x, y, z)
        ratios = _gls_ratios(W, V, d, x, y, z, f)
        if max(ratios) <= tol:
            status = 0
            break
        rhs = np.concatenate([a ** 0.5 * f[0], a ** -0.5 * f[1], a ** 0.5 * bb * f[2]])
        t, k, _ = zgmres(op, P.Ml(rhs), inner_tol, restart, inner_maxit)
        inner += k
        d1, d2, d3 = P.split(P.Mr(t))
        y, z, x = y + a ** 0.5 * d1, z - a ** -0.5 * d2, x + a ** 0.5 * bb * d3
    return dict(x=x, y=y, z=z, status=status, iters=it, inner_iters=inner, ratios=ratios, alpha=alpha)
