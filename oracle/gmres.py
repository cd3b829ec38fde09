"""GMRES-based iterative refinement (Sec. 5) -- CPU oracle.

TEST INFRASTRUCTURE ONLY (see oracle/__init__.py).

Restates the paper's GMRES-IR for LSE and GLS:
* the scaled augmented matrices F~(alpha, beta) and the scaled correction
  unknowns / right-hand sides (eq. lse-limit-notation, eq. gls-limit-notation);
* the block-diagonal split preconditioners M_l, M_r built from the
  low-precision factors: LSE m >= n (eq. lse-bdpre-mlarge) and n > m
  (eq. lse-bdpre-nlarge), GLS n <= p (eq. gls-bdpre-plarge) and n > p
  (eq. gls-bdpre-nlarge); and the left preconditioners of Sec. 5.1
  (eq. lse-leftpre, eq. gls-leftpre), applied through Alg. 1 / Alg. 3;
* restarted GMRES in FP64 with modified Gram-Schmidt Arnoldi and Givens
  rotations (Sec. 6.1: GMRES runs entirely in double precision);
* the outer refinement loop of Alg. 2 / Alg. 4 with the correction system
  solved by that GMRES instead of Alg. 1 / Alg. 3.

Readings (the paper does not fix them): restart 30, inner relative residual
1e-8, at most 300 inner iterations per outer step, beta = 1,
alpha = max(||r0||, sqrt(u) ||A||_F ||x0||) for LSE and
alpha = max(||y0||, sqrt(u) ||V||_F ||z0||) for GLS (1 if both are zero).
Dense triangular solves use scipy (a library primitive); the orthogonal
factors are applied with the oracle's reflector routines.
"""
import numpy as np
from scipy.linalg import solve_triangular

from . import (R_T, apply, gls_correction, gls_factor, gls_init_z, gls_paige, gls_residual, lse_correction,
               lse_factor, lse_init_v, lse_nullspace, lse_residual)

U64 = np.finfo(np.float64).eps / 2


class LseBD:
    """F~ = [a I 0 A; 0 0 b B; A^T b B^T 0] and the split preconditioner
    M_l = diag(a^-1/2 I, a^-1/2 b^-1 S R^-1, a^1/2 T1^-T Q),
    M_r = diag(a^-1/2 I, a^-1/2 b^-1 R^-T S^T, a^1/2 Q^T T1^-1),
    S = T1(n-p+1:n, n-p+1:n).  T1 is the leading n x n block of T when
    m >= n (eq. lse-bdpre-mlarge); when n > m, T = [T^_1, T^_2] is m x n and
    T1 is the paper's U = [T^_1 T^_2; 0 I_{n-m}], whose trailing p x p block
    is its Y (eq. lse-bdpre-nlarge)."""

    def __init__(self, F, A, B, alpha, beta):
        m, n, p = F["m"], F["n"], F["p"]
        R, T = R_T(F)
        self.F, self.A, self.B = F, np.asarray(A), np.asarray(B)
        self.m, self.n, self.p = m, n, p
        if m >= n:
            self.T1 = T[:n, :n]
        else:
            self.T1 = np.vstack([T[:m, :n], np.hstack([np.zeros((n - m, m)), np.eye(n - m)])])
        self.S = self.T1[n - p:, n - p:]
        self.R = R
        self.a, self.b = alpha, beta

    def split(self, u):
        m, p = self.m, self.p
        return u[:m], u[m:m + p], u[m + p:]

    def Fmul(self, u):
        u1, u2, u3 = self.split(u)
        return np.concatenate([self.a * u1 + self.A @ u3, self.b * (self.B @ u3),
                               self.A.T @ u1 + self.b * (self.B.T @ u2)])

    def Ml(self, u):
        u1, u2, u3 = self.split(u)
        a, b = self.a, self.b
        o2 = self.S @ solve_triangular(self.R, u2, lower=False) if self.p else u2
        o3 = solve_triangular(self.T1, apply(self.F, "Q", u3), trans="T", lower=False)
        return np.concatenate([a ** -0.5 * u1, a ** -0.5 / b * o2, a ** 0.5 * o3])

    def Mr(self, t):
        t1, t2, t3 = self.split(t)
        a, b = self.a, self.b
        o2 = solve_triangular(self.R, self.S.T @ t2, trans="T", lower=False) if self.p else t2
        o3 = apply(self.F, "Q", solve_triangular(self.T1, t3, lower=False), trans=True)
        return np.concatenate([a ** -0.5 * t1, a ** -0.5 / b * o2, a ** 0.5 * o3])

    def scale_rhs(self, f1, f2, f3):
        a, b = self.a, self.b
        return np.concatenate([a ** 0.5 * f1, a ** 0.5 * b * f2, a ** -0.5 * f3])

    def unscale(self, du):
        """(dr, dv, dx) from the scaled correction [a^-1/2 dr; -a^-1/2 b^-1 dv; a^1/2 dx]."""
        d1, d2, d3 = self.split(du)
        a, b = self.a, self.b
        return a ** 0.5 * d1, -(a ** 0.5) * b * d2, a ** -0.5 * d3


class GlsBD:
    """F~ = [a I V^T 0; V 0 b W; 0 b W^T 0] and the split preconditioner
    M_l = diag(a^-1/2 I, a^1/2 T2^-1 Q^T, a^-1/2 b^-1 S^T R^-T),
    M_r = diag(a^-1/2 I, a^1/2 Q T2^-T, a^-1/2 b^-1 R^-1 S),
    S = T2(1:m, 1:m).  When n <= p, T = [0, T2] (eq. gls-bdpre-plarge); when
    n > p, T = [T^_1; T^_2] is n x p and T2 is the paper's
    U = [I_{n-p} T^_1; 0 T^_2], whose leading m x m block is its Y
    (eq. gls-bdpre-nlarge)."""

    def __init__(self, F, W, V, alpha, beta):
        n, m, p = F["n"], F["m"], F["p"]
        R, T = R_T(F)
        self.F, self.W, self.V = F, np.asarray(W), np.asarray(V)
        self.n, self.m, self.p = n, m, p
        if n <= p:
            self.T2 = T[:, p - n:]
        else:
            self.T2 = np.vstack([np.hstack([np.eye(n - p), T[:n - p, :p]]),
                                 np.hstack([np.zeros((p, n - p)), T[n - p:, :p]])])
        self.S = self.T2[:m, :m]
        self.R = R
        self.a, self.b = alpha, beta

    def split(self, u):
        p, n = self.p, self.n
        return u[:p], u[p:p + n], u[p + n:]

    def Fmul(self, u):
        u1, u2, u3 = self.split(u)
        return np.concatenate([self.a * u1 + self.V.T @ u2, self.V @ u1 + self.b * (self.W @ u3),
                               self.b * (self.W.T @ u2)])

    def Ml(self, u):
        u1, u2, u3 = self.split(u)
        a, b = self.a, self.b
        o2 = solve_triangular(self.T2, apply(self.F, "Q", u2, trans=True), lower=False)
        o3 = self.S.T @ solve_triangular(self.R, u3, trans="T", lower=False) if self.m else u3
        return np.concatenate([a ** -0.5 * u1, a ** 0.5 * o2, a ** -0.5 / b * o3])

    def Mr(self, t):
        t1, t2, t3 = self.split(t)
        a, b = self.a, self.b
        o2 = apply(self.F, "Q", solve_triangular(self.T2, t2, trans="T", lower=False))
        o3 = solve_triangular(self.R, self.S @ t3, lower=False) if self.m else t3
        return np.concatenate([a ** -0.5 * t1, a ** 0.5 * o2, a ** -0.5 / b * o3])

    def scale_rhs(self, f1, f2, f3):
        a, b = self.a, self.b
        return np.concatenate([a ** 0.5 * f1, a ** -0.5 * f2, a ** 0.5 * b * f3])

    def unscale(self, du):
        """(dy, dz, dx) from [a^-1/2 dy; -a^1/2 dz; a^-1/2 b^-1 dx]."""
        d1, d2, d3 = self.split(du)
        a, b = self.a, self.b
        return a ** 0.5 * d1, -(a ** -0.5) * d2, a ** 0.5 * b * d3


class LseLeft(LseBD):
    """The left preconditioner of Sec. 5.1 (eq. lse-leftpre): M ~ F~^{-1},
    applied, as the paper does, by the correction solver on the factors.
    F~ u = g is the correction system of Alg. 1 with f = (g1, g2 / b, a g3):
    (dr, dv, dx) -> u = (dr / a, -dv / (a b), dx).  M_r = I."""

    def __init__(self, F, A, B, alpha, beta):
        m, n, p = F["m"], F["n"], F["p"]
        self.F, self.A, self.B = F, np.asarray(A), np.asarray(B)
        self.m, self.n, self.p = m, n, p
        self.a, self.b = alpha, beta

    def Ml(self, g):
        g1, g2, g3 = self.split(g)
        a, b = self.a, self.b
        dr, dv, dx = lse_correction(self.F, g1, g2 / b, a * g3)
        return np.concatenate([dr / a, -dv / (a * b), dx])

    def Mr(self, t):
        return t


class GlsLeft(GlsBD):
    """The left preconditioner of Sec. 5.1 (eq. gls-leftpre), applied by
    Alg. 3: F~ u = g is the correction system with f = (g1, a g2, g3 / b):
    (dy, dz, dx) -> u = (dy / a, -dz, dx / (a b)).  M_r = I."""

    def __init__(self, F, W, V, alpha, beta):
        n, m, p = F["n"], F["m"], F["p"]
        self.F, self.W, self.V = F, np.asarray(W), np.asarray(V)
        self.n, self.m, self.p = n, m, p
        self.a, self.b = alpha, beta

    def Ml(self, g):
        g1, g2, g3 = self.split(g)
        a, b = self.a, self.b
        dy, dz, dx = gls_correction(self.F, g1, a * g2, g3 / b)
        return np.concatenate([dy / a, -dz, dx / (a * b)])

    def Mr(self, t):
        return t


def gmres(op, rhs, tol=1e-8, restart=30, maxit=300):
    """Restarted GMRES(restart) from x0 = 0, modified Gram-Schmidt Arnoldi,
    Givens rotations; stops when ||rhs - op(x)|| <= tol ||rhs||.
    Returns (x, iterations, relative residual)."""
    nb = np.linalg.norm(rhs)
    x = np.zeros_like(rhs)
    if nb == 0:
        return x, 0, 0.0
    total = 0
    r = rhs.copy()
    rel = 1.0
    while total < maxit:
        beta0 = np.linalg.norm(r)
        if beta0 <= tol * nb:
            break
        Vb = [r / beta0]
        H = np.zeros((restart + 1, restart))
        cs = np.zeros(restart)
        sn = np.zeros(restart)
        g = np.zeros(restart + 1)
        g[0] = beta0
        j_end = 0
        for j in range(restart):
            w = op(Vb[j])
            total += 1
            for i in range(j + 1):
                H[i, j] = Vb[i] @ w
                w = w - H[i, j] * Vb[i]
            H[j + 1, j] = np.linalg.norm(w)
            Vb.append(w / H[j + 1, j] if H[j + 1, j] > 0 else w)
            for i in range(j):
                t = cs[i] * H[i, j] + sn[i] * H[i + 1, j]
                H[i + 1, j] = -sn[i] * H[i, j] + cs[i] * H[i + 1, j]
                H[i, j] = t
            den = np.hypot(H[j, j], H[j + 1, j])
            cs[j] = H[j, j] / den if den else 1.0
            sn[j] = H[j + 1, j] / den if den else 0.0
            H[j, j] = den
            H[j + 1, j] = 0.0
            g[j + 1] = -sn[j] * g[j]
            g[j] = cs[j] * g[j]
            j_end = j + 1
            if abs(g[j + 1]) <= tol * nb or total >= maxit:
                break
        yk = solve_triangular(H[:j_end, :j_end], g[:j_end], lower=False)
        x = x + np.column_stack(Vb[:j_end]) @ yk
        r = rhs - op(x)
        rel = np.linalg.norm(r) / nb
        if rel <= tol:
            break
    return x, total, rel


def lse_gmres_ir(A, B, b, d, fact="fp32", tol=2e-15, maxit=40, restart=30, inner_tol=1e-8,
                 inner_maxit=300, beta=1.0, precond="bd"):
    """LSE GMRES-IR with the block-diagonal split preconditioner (precond
    'bd') or the left preconditioner of Sec. 5.1 ('left')."""
    A, B = np.asarray(A, dtype=np.float64), np.asarray(B, dtype=np.float64)
    b, d = np.asarray(b, dtype=np.float64), np.asarray(d, dtype=np.float64)
    F = lse_factor(A, B, fact)
    x = lse_nullspace(F, b, d)
    r = b - A @ x
    v = lse_init_v(F, A, r)
    nA, nB = np.linalg.norm(A), np.linalg.norm(B)
    alpha = max(np.linalg.norm(r), np.sqrt(U64) * nA * np.linalg.norm(x))
    alpha = alpha if alpha > 0 else 1.0
    P = (LseLeft if precond == "left" else LseBD)(F, A, B, alpha, beta)
    op = lambda t: P.Ml(P.Fmul(P.Mr(t)))
    status, inner, ratios = 3, 0, [0.0, 0.0, 0.0]
    it = 0
    for it in range(maxit):
        f1, f2, f3 = lse_residual(A, B, b, d, x, r, v, dd=False)
        den = [np.linalg.norm(b) + np.linalg.norm(r) + nA * np.linalg.norm(x), np.linalg.norm(d) + nB * np.linalg.norm(x),
               nA * np.linalg.norm(r) + nB * np.linalg.norm(v)]
        ratios = [np.linalg.norm(f) / dd if dd else 0.0 for f, dd in zip((f1, f2, f3), den)]
        if not np.all(np.isfinite(ratios)):
            status = 4
            break
        if max(ratios) <= tol:
            status = 0
            break
        t, k, _ = gmres(op, P.Ml(P.scale_rhs(f1, f2, f3)), inner_tol, restart, inner_maxit)
        inner += k
        dr, dv, dx = P.unscale(P.Mr(t))
        r, v, x = r + dr, v + dv, x + dx
    return dict(x=x, r=r, v=v, status=status, iters=it, inner_iters=inner, ratios=ratios, alpha=alpha)


def gls_gmres_ir(W, V, d, fact="fp32", tol=2e-15, maxit=40, restart=30, inner_tol=1e-8,
                 inner_maxit=300, beta=1.0, precond="bd"):
    """GLS GMRES-IR with the block-diagonal split preconditioner (precond
    'bd') or the left preconditioner of Sec. 5.1 ('left')."""
    W, V = np.asarray(W, dtype=np.float64), np.asarray(V, dtype=np.float64)
    d = np.asarray(d, dtype=np.float64)
    F = gls_factor(W, V, fact)
    x, y = gls_paige(F, d)
    z = gls_init_z(F, y)
    nW, nV = np.linalg.norm(W), np.linalg.norm(V)
    alpha = max(np.linalg.norm(y), np.sqrt(U64) * nV * np.linalg.norm(z))
    alpha = alpha if alpha > 0 else 1.0
    P = (GlsLeft if precond == "left" else GlsBD)(F, W, V, alpha, beta)
    op = lambda t: P.Ml(P.Fmul(P.Mr(t)))
    status, inner, ratios = 3, 0, [0.0, 0.0, 0.0]
    it = 0
    for it in range(maxit):
        f1, f2, f3 = gls_residual(W, V, d, x, y, z, dd=False)
        den = [np.linalg.norm(y) + nV * np.linalg.norm(z),
               np.linalg.norm(d) + nW * np.linalg.norm(x) + nV * np.linalg.norm(y), nW * np.linalg.norm(z)]
        ratios = [np.linalg.norm(f) / dd if dd else 0.0 for f, dd in zip((f1, f2, f3), den)]
        if not np.all(np.isfinite(ratios)):
            status = 4
            break
        if max(ratios) <= tol:
            status = 0
            break
        t, k, _ = gmres(op, P.Ml(P.scale_rhs(f1, f2, f3)), inner_tol, restart, inner_maxit)
        inner += k
        dy, dz, dx = P.unscale(P.Mr(t))
        y, z, x = y + dy, z + dz, x + dx
    return dict(x=x, y=y, z=z, status=status, iters=it, inner_iters=inner, ratios=ratios, alpha=alpha)
