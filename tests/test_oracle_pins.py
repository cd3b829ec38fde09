"""Pins that tie the CPU oracle to the paper and to independent mathematics.

Each test checks the oracle against something other than itself: LAPACK's
xGGLSE, textbook least squares, exact rational arithmetic, closed-form
identities of the factorizations (Lemma 4.5 / 4.6), the backward-stability
statement of Theorems 4.3 / 4.7, and the qualitative behaviour printed in
Tables 4 and 5.  A plausible slip in the oracle (a dropped term, a wrong sign
or index, a transposed operand) fails at least one of them.
"""
import json
import os
from fractions import Fraction

import numpy as np
import pytest
import scipy.linalg.lapack as lapack

from paper_2406_16499_gb300 import inputs as I

pytestmark = pytest.mark.filterwarnings("ignore::RuntimeWarning")
U = np.finfo(np.float64).eps / 2
GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "paper_tables.json")


# ------------------------------------------------------------ helpers --

def exact_solve(M, rhs):
    """Gaussian elimination with exact rationals (M, rhs given as floats)."""
    n = len(rhs)
    a = [[Fraction(float(M[i, j])) for j in range(n)] + [Fraction(float(rhs[i]))] for i in range(n)]
    for c in range(n):
        piv = next(r for r in range(c, n) if a[r][c] != 0)
        a[c], a[piv] = a[piv], a[c]
        for r in range(n):
            if r != c and a[r][c] != 0:
                f = a[r][c] / a[c][c]
                a[r] = [x - f * y for x, y in zip(a[r], a[c])]
    return [a[i][n] / a[i][i] for i in range(n)]


def lse_aug(A, B):
    m, n = A.shape
    p = B.shape[0]
    F = np.zeros((m + p + n, m + p + n))
    F[:m, :m] = np.eye(m)
    F[:m, m + p:] = A
    F[m:m + p, m + p:] = B
    F[m + p:, :m] = A.T
    F[m + p:, m:m + p] = B.T
    return F


def gls_aug(W, V):
    n, m = W.shape
    p = V.shape[1]
    F = np.zeros((p + n + m, p + n + m))
    F[:p, :p] = np.eye(p)
    F[:p, p:p + n] = V.T
    F[p:p + n, :p] = V
    F[p:p + n, p + n:] = W
    F[p + n:, p:p + n] = W.T
    return F


def rel(a, b):
    nb = np.linalg.norm(b)
    return np.linalg.norm(np.asarray(a) - np.asarray(b)) / (nb if nb else 1.0)


# ------------------------------------------- independent library / textbook --

@pytest.mark.parametrize("m,n,p,ca,cb", [(30, 12, 4, 1e3, 1e1), (40, 40, 8, 1e2, 1e1),
                                         (10, 14, 6, 1e2, 1e1), (25, 10, 10, 1e1, 1e1),
                                         (60, 33, 1, 1e5, 1.0)])
def test_lse_matches_lapack_dgglse(oracle_mod, m, n, p, ca, cb):
    """The oracle's LSE solution equals LAPACK DGGLSE's (the paper's
    fixed-precision reference algorithm, Sec. 6.1) to O(kappa u)."""
    P = I.lse_svd(100 + m + n + p, m, n, p, ca, cb)
    t = oracle_mod.lse_truth(P["A"], P["B"], P["b"], P["d"])
    xl = lapack.dgglse(P["A"].copy(order="F"), P["B"].copy(order="F"), P["b"].copy(), P["d"].copy())[3]
    assert rel(t["x"], xl) < 50 * max(ca, cb) * U


def test_lse_p0_is_ordinary_least_squares(oracle_mod):
    """p = 0: no constraint, the problem is ordinary least squares."""
    P = I.lse_svd(7, 40, 15, 0, 1e3, 1.0)
    t = oracle_mod.lse_truth(P["A"], P["B"], P["b"], P["d"])
    x_ls = np.linalg.lstsq(P["A"], P["b"], rcond=None)[0]
    assert rel(t["x"], x_ls) < 1e3 * 50 * U
    assert rel(t["r"], P["b"] - P["A"] @ x_ls) < 1e-12


def test_gls_square_v_is_weighted_least_squares(oracle_mod):
    """n = p, V nonsingular: min ||y|| s.t. Wx + Vy = d is the weighted LS
    min ||V^{-1}(d - W x)|| (the GLM motivation, Sec. 1)."""
    G = I.gls_svd(11, 24, 7, 24, 1e2, 1e1)
    W, V, d = G["W"], G["V"], G["d"]
    t = oracle_mod.gls_truth(W, V, d)
    VinvW = np.linalg.solve(V, W)
    x = np.linalg.lstsq(VinvW, np.linalg.solve(V, d), rcond=None)[0]
    y = np.linalg.solve(V, d - W @ x)
    assert rel(t["x"], x) < 1e-11
    assert rel(t["y"], y) < 1e-11


def test_gls_identity_v_is_least_squares(oracle_mod):
    """V = I: the GLS problem is min ||d - W x|| with y = d - W x (eq. link
    with the identity covariance)."""
    g = I.rng(5)
    W = I.svd_matrix(g, 30, 9, I.logspace_sigma(9, 1e3))
    d = g.standard_normal(30)
    t = oracle_mod.gls_truth(W, np.eye(30), d)
    x = np.linalg.lstsq(W, d, rcond=None)[0]
    assert rel(t["x"], x) < 1e-12
    assert rel(t["y"], d - W @ x) < 1e-12
    # z = y when V = I (row 1 of eq. aug-GLS: y = V^T z)
    assert rel(t["z"], t["y"]) < 1e-12


@pytest.mark.parametrize("m,n,p", [(9, 15, 6), (20, 21, 1), (1, 8, 7)])
def test_lse_square_stack_is_a_linear_solve(oracle_mod, m, n, p):
    """n = m + p: [A; B] is square and nonsingular (the rank conditions of
    the problem statement, Sec. 1), so the LSE solution solves [A; B] x =
    [b; d] and the least-squares residual r = b - A x vanishes."""
    P = I.lse_svd(300 + m + n, m, n, p, 1e2, 1e1)
    t = oracle_mod.lse_truth(P["A"], P["B"], P["b"], P["d"])
    x = np.linalg.solve(np.vstack([P["A"], P["B"]]), np.concatenate([P["b"], P["d"]]))
    kap = np.linalg.cond(np.vstack([P["A"], P["B"]]))
    assert rel(t["x"], x) < 50 * kap * U
    assert np.linalg.norm(t["r"]) < 50 * kap * U * np.linalg.norm(P["b"])


def test_lse_square_b_fixes_x(oracle_mod):
    """p = n: B x = d alone determines x (B nonsingular), whatever A and b
    are; r is then the plain residual b - A x."""
    P = I.lse_svd(41, 30, 12, 12, 1e3, 1e2)
    t = oracle_mod.lse_truth(P["A"], P["B"], P["b"], P["d"])
    x = np.linalg.solve(P["B"], P["d"])
    assert rel(t["x"], x) < 50 * 1e2 * U
    assert rel(t["r"], P["b"] - P["A"] @ x) < 1e-12


# ----------------------------------------------------- exact brute force --

@pytest.mark.parametrize("m,n,p", [(5, 4, 2), (4, 4, 1), (3, 4, 1), (4, 3, 3), (6, 3, 1)])
def test_lse_exact_rational_augmented_solve(oracle_mod, m, n, p):
    """The 3-block system eq. aug-LSE solved exactly in rationals gives
    [r; -v; x]; the oracle's refined solution agrees to ~u."""
    P = I.lse_svd(3 * m + 5 * n + p, m, n, p, 10.0, 3.0)
    A, B, b, d = P["A"], P["B"], P["b"], P["d"]
    sol = exact_solve(lse_aug(A, B), np.concatenate([b, d, np.zeros(n)]))
    r_ex = np.array([float(s) for s in sol[:m]])
    v_ex = -np.array([float(s) for s in sol[m:m + p]])
    x_ex = np.array([float(s) for s in sol[m + p:]])
    t = oracle_mod.lse_truth(A, B, b, d)
    assert rel(t["x"], x_ex) < 1e-14
    assert rel(t["r"], r_ex) < 1e-13
    assert rel(t["v"], v_ex) < 1e-13


@pytest.mark.parametrize("n,m,p", [(4, 2, 3), (5, 2, 3), (3, 3, 1), (4, 1, 4), (6, 2, 6)])
def test_gls_exact_rational_augmented_solve(oracle_mod, n, m, p):
    """eq. aug-GLS solved exactly in rationals gives [y; -z; x]."""
    G = I.gls_svd(7 * n + 3 * m + p, n, m, p, 10.0, 3.0)
    W, V, d = G["W"], G["V"], G["d"]
    sol = exact_solve(gls_aug(W, V), np.concatenate([np.zeros(p), d, np.zeros(m)]))
    y_ex = np.array([float(s) for s in sol[:p]])
    z_ex = -np.array([float(s) for s in sol[p:p + n]])
    x_ex = np.array([float(s) for s in sol[p + n:]])
    t = oracle_mod.gls_truth(W, V, d)
    assert rel(t["x"], x_ex) < 1e-14
    assert rel(t["y"], y_ex) < 1e-13
    assert rel(t["z"], z_ex) < 1e-13


def test_residual_double_double_is_exact(oracle_mod):
    """The double-double residual equals the exact rational residual to far
    below FP64 rounding; the plain FP64 residual obeys the gemv bound
    |err| <= gamma_{n+2} (|b| + |r| + |A||x|) (Assumption 4.1, Table 1)."""
    P = I.lse_svd(21, 7, 5, 2, 1e2, 1e1)
    A, B, b, d = P["A"], P["B"], P["b"], P["d"]
    g = I.rng(22)
    x, r, v = g.standard_normal(5), g.standard_normal(7), g.standard_normal(2)
    f1, f2, f3 = oracle_mod.lse_residual(A, B, b, d, x, r, v, dd=True)
    F = lse_aug(A, B)
    u = np.concatenate([r, -v, x])
    rhs = np.concatenate([b, d, np.zeros(5)])
    ex = [Fraction(float(rhs[i])) - sum(Fraction(float(F[i, j])) * Fraction(float(u[j]))
                                        for j in range(len(u))) for i in range(len(u))]
    got = np.concatenate([f1, f2, f3])
    for e, gv in zip(ex, got):
        assert abs(Fraction(float(gv)) - e) <= Fraction(U) * abs(e) + Fraction(1, 10 ** 30)
    p1, p2, p3 = oracle_mod.lse_residual(A, B, b, d, x, r, v, dd=False)
    bound = (len(u) + 2) * U * (np.abs(rhs) + np.abs(F) @ np.abs(u))
    assert np.all(np.abs(np.concatenate([p1, p2, p3]) - got) <= bound)


def test_gls_residual_double_double_is_exact(oracle_mod):
    G = I.gls_svd(23, 6, 2, 5, 1e2, 1e1)
    W, V, d = G["W"], G["V"], G["d"]
    g = I.rng(24)
    x, y, z = g.standard_normal(2), g.standard_normal(5), g.standard_normal(6)
    f1, f2, f3 = oracle_mod.gls_residual(W, V, d, x, y, z, dd=True)
    F = gls_aug(W, V)
    u = np.concatenate([y, -z, x])
    rhs = np.concatenate([np.zeros(5), d, np.zeros(2)])
    ex = [Fraction(float(rhs[i])) - sum(Fraction(float(F[i, j])) * Fraction(float(u[j]))
                                        for j in range(len(u))) for i in range(len(u))]
    got = np.concatenate([f1, f2, f3])
    for e, gv in zip(ex, got):
        assert abs(Fraction(float(gv)) - e) <= Fraction(U) * abs(e) + Fraction(1, 10 ** 30)


# ------------------------------------------- factorization identities --

@pytest.mark.parametrize("fact,tol", [("fp64", 1e-14), ("fp32", 1e-5)])
@pytest.mark.parametrize("m,n,p", [(20, 12, 5), (9, 12, 4), (15, 15, 15)])
def test_grq_backward_error_and_orthogonality(oracle_mod, fact, tol, m, n, p):
    """Lemma 4.5: B + dE1 = [0, R] Q, A + dE2 = Z T Q with ||dE|| = O(u_f)
    ||.||_F; Q and Z orthogonal; R upper triangular p x p; T upper
    trapezoidal m x n."""
    P = I.lse_svd(m * n + p, m, n, p, 1e2, 1e1)
    A, B = P["A"], P["B"]
    F = oracle_mod.lse_factor(A, B, fact)
    Q = oracle_mod.explicit(F, "Q")
    Z = oracle_mod.explicit(F, "Z")
    R, T = oracle_mod.R_T(F)
    RB = np.zeros((p, n))
    RB[:, n - p:] = R
    assert np.linalg.norm(B - RB @ Q) <= tol * np.linalg.norm(B)
    assert np.linalg.norm(A - Z @ T @ Q) <= tol * np.linalg.norm(A)
    assert np.linalg.norm(Q.T @ Q - np.eye(n)) <= tol * n
    assert np.linalg.norm(Z.T @ Z - np.eye(m)) <= tol * m
    assert np.allclose(T, np.triu(T))
    # the transposed applies are the inverses
    x = I.rng(1).standard_normal(n)
    assert rel(oracle_mod.apply(F, "Q", oracle_mod.apply(F, "Q", x), trans=True), x) < tol


@pytest.mark.parametrize("fact,tol", [("fp64", 1e-14), ("fp32", 1e-5)])
@pytest.mark.parametrize("n,m,p", [(12, 5, 20), (12, 5, 12), (12, 5, 8), (10, 10, 3)])
def test_gqr_backward_error_and_orthogonality(oracle_mod, fact, tol, n, m, p):
    """Lemma 4.6: W + dF1 = Q [R; 0], V + dF2 = Q T Z, T upper trapezoidal
    with T = [T11 T12; 0 T22], T22 (n-m) x (n-m) upper triangular."""
    G = I.gls_svd(n * m + p, n, m, p, 1e2, 1e1)
    W, V = G["W"], G["V"]
    F = oracle_mod.gls_factor(W, V, fact)
    Q = oracle_mod.explicit(F, "Q")
    Z = oracle_mod.explicit(F, "Z")
    R, T = oracle_mod.R_T(F)
    RW = np.zeros((n, m))
    RW[:m] = R
    assert np.linalg.norm(W - Q @ RW) <= tol * np.linalg.norm(W)
    assert np.linalg.norm(V - Q @ T @ Z) <= tol * np.linalg.norm(V)
    assert np.linalg.norm(Q.T @ Q - np.eye(n)) <= tol * n
    assert np.linalg.norm(Z.T @ Z - np.eye(p)) <= tol * p
    o = p - n + m
    assert np.allclose(T[m:, :o], 0.0)
    T22 = T[m:, o:]
    assert np.allclose(T22, np.triu(T22))


# ------------------------------------------------- correction solvers --

@pytest.mark.parametrize("m,n,p", [(20, 12, 5), (9, 12, 4), (30, 10, 10)])
def test_lse_correction_backward_stable(oracle_mod, m, n, p):
    """Theorem 4.3 with FP64 factors: the computed correction satisfies
    eq. correction-system-lse with a normwise backward error of O(u)."""
    P = I.lse_svd(m + 2 * n + 3 * p, m, n, p, 1e3, 1e1)
    A, B = P["A"], P["B"]
    F = oracle_mod.lse_factor(A, B, "fp64")
    g = I.rng(m)
    f1, f2, f3 = g.standard_normal(m), g.standard_normal(p), g.standard_normal(n)
    dr, dv, dx = oracle_mod.lse_correction(F, f1, f2, f3)
    Fa = lse_aug(A, B)
    sol = np.concatenate([dr, -dv, dx])
    f = np.concatenate([f1, f2, f3])
    eta = np.linalg.norm(Fa @ sol - f) / (np.linalg.norm(Fa) * np.linalg.norm(sol) + np.linalg.norm(f))
    assert eta < 100 * U


@pytest.mark.parametrize("n,m,p", [(12, 5, 20), (12, 5, 12), (12, 5, 8), (10, 10, 3)])
def test_gls_correction_backward_stable(oracle_mod, n, m, p):
    """Theorem 4.7 with FP64 factors, under the two readings of Alg. 3
    (T22 g2 = u2 and dz = -Q h)."""
    G = I.gls_svd(3 * n + m + 2 * p, n, m, p, 1e3, 1e1)
    W, V = G["W"], G["V"]
    F = oracle_mod.gls_factor(W, V, "fp64")
    g = I.rng(n + 77)
    f1, f2, f3 = g.standard_normal(p), g.standard_normal(n), g.standard_normal(m)
    dy, dz, dx = oracle_mod.gls_correction(F, f1, f2, f3)
    Fa = gls_aug(W, V)
    sol = np.concatenate([dy, -dz, dx])
    f = np.concatenate([f1, f2, f3])
    eta = np.linalg.norm(Fa @ sol - f) / (np.linalg.norm(Fa) * np.linalg.norm(sol) + np.linalg.norm(f))
    assert eta < 100 * U


def test_gls_correction_printed_literally_fails(oracle_mod):
    """Plants the printed Alg. 3 (T22^T g2 = u2 and x2 = Q h) in a numpy copy
    of the oracle's steps: it does NOT solve the correction system, while
    the oracle's reading does.  This documents both readings."""
    n, m, p = 7, 3, 9
    G = I.gls_svd(91, n, m, p, 1e2, 1e1)
    W, V = G["W"], G["V"]
    F = oracle_mod.gls_factor(W, V, "fp64")
    Q, Z = oracle_mod.explicit(F, "Q"), oracle_mod.explicit(F, "Z")
    R, T = oracle_mod.R_T(F)
    o = p - n + m
    T11, T12, T22 = T[:m, :o], T[:m, o:], T[m:, o:]
    g = I.rng(92)
    f1, f2, f3 = g.standard_normal(p), g.standard_normal(n), g.standard_normal(m)
    u, w = Q.T @ f2, Z @ f1
    h1 = np.linalg.solve(R.T, f3)
    g2 = np.linalg.solve(T22.T, u[m:])                 # as printed (Alg. 3 step 4)
    h2 = np.linalg.solve(T22.T, w[o:] - g2 - T12.T @ h1)
    g1 = w[:o] - T11.T @ h1
    dy = Z.T @ np.concatenate([g1, g2])
    dz = Q @ np.concatenate([h1, h2])                  # as printed (Alg. 3 step 7)
    dx = np.linalg.solve(R, u[:m] - T11 @ g1 - T12 @ g2)
    Fa = gls_aug(W, V)
    f = np.concatenate([f1, f2, f3])
    literal = np.linalg.norm(Fa @ np.concatenate([dy, -dz, dx]) - f) / np.linalg.norm(f)
    dy2, dz2, dx2 = oracle_mod.gls_correction(F, f1, f2, f3)
    ours = np.linalg.norm(Fa @ np.concatenate([dy2, -dz2, dx2]) - f) / np.linalg.norm(f)
    assert literal > 1e-3
    assert ours < 1e-13


def test_one_correction_step_with_exact_factors_lands_on_solution(oracle_mod):
    """With FP64 factors a single refinement step from a perturbed point
    reaches the solution (the correction system is solved exactly up to u)."""
    P = I.lse_svd(55, 25, 11, 3, 1e2, 1e1)
    A, B, b, d = P["A"], P["B"], P["b"], P["d"]
    t = oracle_mod.lse_truth(A, B, b, d)
    g = I.rng(56)
    x = t["x"] + 1e-3 * g.standard_normal(11)
    r = t["r"] + 1e-3 * g.standard_normal(25)
    v = t["v"] + 1e-3 * g.standard_normal(3)
    F = oracle_mod.lse_factor(A, B, "fp64")
    f1, f2, f3 = oracle_mod.lse_residual(A, B, b, d, x, r, v)
    dr, dv, dx = oracle_mod.lse_correction(F, f1, f2, f3)
    assert rel(x + dx, t["x"]) < 1e-12
    assert rel(v + dv, t["v"]) < 1e-12
    W, V, dvec = (lambda G: (G["W"], G["V"], G["d"]))(I.gls_svd(57, 7, 3, 9, 1e2, 1e1))
    tg = oracle_mod.gls_truth(W, V, dvec)
    x = tg["x"] + 1e-3 * g.standard_normal(3)
    y = tg["y"] + 1e-3 * g.standard_normal(9)
    z = tg["z"] + 1e-3 * g.standard_normal(7)
    Fg = oracle_mod.gls_factor(W, V, "fp64")
    f1, f2, f3 = oracle_mod.gls_residual(W, V, dvec, x, y, z)
    dy, dz, dx = oracle_mod.gls_correction(Fg, f1, f2, f3)
    assert rel(x + dx, tg["x"]) < 1e-12
    assert rel(y + dy, tg["y"]) < 1e-12
    assert rel(z + dz, tg["z"]) < 1e-12


def test_initial_multipliers_satisfy_kkt(oracle_mod):
    """LSE: R^T v0 = (Q A^T r0)(n-p+1:n) gives A^T r0 = B^T v0 when x0 is the
    null-space solution (Sec. 3.1).  GLS: z0 = Q [0; v] gives W^T z0 = 0 and
    y0 = V^T z0 (Sec. 3.2, read with Q in front of [0; v])."""
    P = I.lse_svd(61, 30, 12, 4, 1e2, 1e1)
    A, B, b, d = P["A"], P["B"], P["b"], P["d"]
    F = oracle_mod.lse_factor(A, B, "fp64")
    x0 = oracle_mod.lse_nullspace(F, b, d)
    r0 = b - A @ x0
    v0 = oracle_mod.lse_init_v(F, A, r0)
    assert rel(B.T @ v0, A.T @ r0) < 1e-12
    G = I.gls_svd(62, 10, 4, 12, 1e2, 1e1)
    W, V, dv = G["W"], G["V"], G["d"]
    Fg = oracle_mod.gls_factor(W, V, "fp64")
    x0, y0 = oracle_mod.gls_paige(Fg, dv)
    z0 = oracle_mod.gls_init_z(Fg, y0)
    assert np.linalg.norm(W.T @ z0) < 1e-13 * np.linalg.norm(W) * np.linalg.norm(z0)
    assert rel(V.T @ z0, y0) < 1e-12
    # Q^T [0; v] (the printed form) misses y0 = V^T z0
    Q = oracle_mod.explicit(Fg, "Q")
    zq = Q.T @ (Q.T @ z0)
    assert rel(V.T @ zq, y0) > 1e-3


# ---------------------------------------- refinement: Tables 4 and 5 --

def _golden():
    with open(GOLDEN) as f:
        return json.load(f)


@pytest.mark.parametrize("ki", [0, 1, 2, 3])
def test_mplse_convergence_matches_table4(oracle_mod, ki):
    """Table 4 (MPLSE, u_f = single): converges in a few steps for kappa up
    to 1e7 with err-1 at FP64 level; does not converge at kappa = 1e9."""
    gold = _golden()["table4_mplse"]
    kappa = gold["kappa"][ki]
    n = 64
    P = I.lse_paper(400 + ki, 8 * n, n, n // 32, kappa)
    out = oracle_mod.lse_solve(P["A"], P["B"], P["b"], P["d"], fact="fp32", tol=1e-13)
    met = oracle_mod.lse_metrics(P["A"], P["B"], P["b"], P["d"], out["x"], out["r"], out["v"])
    if gold["diverged"][ki]:
        assert out["status"] != 0 or met["eta"] > 1e-10
    else:
        assert out["status"] == 0
        assert out["iters"] <= 3 * gold["iters"][ki] + 2
        assert met["eta"] < 2e-13
        # the tighter FP64-level target: backward error and err-1 <= 1e-14
        out = oracle_mod.lse_solve(P["A"], P["B"], P["b"], P["d"], fact="fp32", tol=2e-15)
        met = oracle_mod.lse_metrics(P["A"], P["B"], P["b"], P["d"], out["x"], out["r"], out["v"])
        assert out["status"] == 0
        assert met["e_con"] < 1e-14 and met["eta"] < 1e-14


@pytest.mark.parametrize("ki", [0, 1, 2, 3])
def test_mpgls_convergence_matches_table5(oracle_mod, ki):
    """Table 5 (MPGLS, u_f = single): converges for kappa up to 1e7, fails at
    1e9."""
    gold = _golden()["table5_mpgls"]
    kappa = gold["kappa"][ki]
    n = 64
    G = I.gls_paper(500 + ki, n, n // 32, 8 * n, kappa)
    out = oracle_mod.gls_solve(G["W"], G["V"], G["d"], fact="fp32", tol=1e-13)
    met = oracle_mod.gls_metrics(G["W"], G["V"], G["d"], out["x"], out["y"], out["z"])
    if gold["diverged"][ki]:
        assert out["status"] != 0 or met["eta"] > 1e-10
    else:
        assert out["status"] == 0
        assert out["iters"] <= 3 * gold["iters"][ki] + 2
        assert met["eta"] < 2e-13
        out = oracle_mod.gls_solve(G["W"], G["V"], G["d"], fact="fp32", tol=2e-15)
        met = oracle_mod.gls_metrics(G["W"], G["V"], G["d"], out["x"], out["y"], out["z"])
        assert out["status"] == 0
        assert met["e_con"] < 1e-14 and met["eta"] < 1e-14


def test_fp64_refinement_reaches_truth(oracle_mod):
    """With FP64 factors and FP64 residuals, refinement reaches the
    double-double-refined solution within O(kappa u) (Table 2, row 2)."""
    P = I.lse_small()
    A, B, b, d = P["A"], P["B"], P["b"], P["d"]
    t = oracle_mod.lse_truth(A, B, b, d)
    mp = oracle_mod.lse_solve(A, B, b, d, fact="fp32")
    F = oracle_mod.lse_factor(A, B, "fp64")
    kap = oracle_mod.lse_kappa(F, t["x"], t["r"])[0]
    assert mp["status"] == 0
    assert rel(mp["x"], t["x"]) < 10 * kap * 1.1e-16


# ------------------------------------------------ condition estimates --

def test_kappa_estimates_match_svd(oracle_mod):
    """The power-iteration estimates equal numpy's SVD-based condition
    numbers of T11, R (LSE) and S^{-1} R (GLS) to a few percent."""
    P = I.lse_svd(71, 40, 20, 5, 1e3, 1e1)
    F = oracle_mod.lse_factor(P["A"], P["B"], "fp64")
    R, T = oracle_mod.R_T(F)
    t = oracle_mod.lse_truth(P["A"], P["B"], P["b"], P["d"])
    k = oracle_mod.lse_kappa(F, t["x"], t["r"], iters=200)
    assert abs(k[1] / np.linalg.cond(T[:15, :15]) - 1) < 0.05
    assert abs(k[2] / np.linalg.cond(R) - 1) < 0.05
    G = I.gls_svd(72, 16, 5, 20, 1e3, 1e1)
    Fg = oracle_mod.gls_factor(G["W"], G["V"], "fp64")
    Rg, Tg = oracle_mod.R_T(Fg)
    S = Tg[:5, 4:9]
    tg = oracle_mod.gls_truth(G["W"], G["V"], G["d"])
    kg = oracle_mod.gls_kappa(Fg, tg["x"], tg["y"], iters=200)
    assert abs(kg[1] / np.linalg.cond(np.linalg.solve(S, Rg)) - 1) < 0.05


# ------------------------------------------------------------ inputs --

def test_input_generators_spectra():
    """The generators realise the requested singular spectra and the AR(1)
    Cholesky closed form reproduces Sigma_ij = rho^|i-j|."""
    P = I.lse_svd(1, 50, 20, 5, 1e4, 1e2)
    s = np.linalg.svd(P["A"], compute_uv=False)
    assert abs(s[0] / s[-1] / 1e4 - 1) < 1e-8
    L = I.ar1_cholesky(40, 0.9)
    S = 0.9 ** np.abs(np.subtract.outer(np.arange(40), np.arange(40)))
    assert np.allclose(L @ L.T, S, atol=1e-13)
    G = I.gls_paper(3, 20, 4, 30, 1e5)
    s = np.linalg.svd(np.hstack([G["W"], G["V"]]), compute_uv=False)
    assert abs(s[0] / s[-1] / 1e5 - 1) < 1e-6
    a = I.lse_small(9)["A"]
    b = I.lse_small(9)["A"]
    assert np.array_equal(a, b)


@pytest.mark.parametrize("cond", [1e2, 1e6])
def test_known_solution_construction(oracle_mod, cond):
    """The known-solution LSE construction used at full size: the oracle's
    FP64 solution equals (x*, r*) to within the forward-error bound, and
    kappa_up bounds the oracle's condition number (reading C13) from above."""
    torch = pytest.importorskip("torch")
    T = I.lse_known_torch(5, 90, 40, 7, cond, 1e1, "cpu")
    A, B, b, d = (T[k].numpy() for k in ("A", "B", "b", "d"))
    xs, rs = T["x_true"].numpy(), T["r_true"].numpy()
    t = oracle_mod.lse_truth(A, B, b, d)
    F = oracle_mod.lse_factor(A, B, "fp64")
    kap = oracle_mod.lse_kappa(F, t["x"], t["r"])[0]
    assert kap <= T["kappa_up"] * (1 + 1e-6), (kap, T["kappa_up"])
    fe = np.linalg.norm(t["x"] - xs) / np.linalg.norm(xs)
    assert fe <= 10 * T["kappa_up"] * 1.1e-16, (fe, T["kappa_up"])
    assert np.linalg.norm(t["r"] - rs) <= 1e-6 * np.linalg.norm(rs)
    # the multiplier equation of the construction
    assert np.linalg.norm(A.T @ rs - B.T @ T["v_true"].numpy()) <= 1e-12 * np.linalg.norm(A) * np.linalg.norm(rs)
