"""Pins of the complex oracle (oracle/zoracle.py) against LAPACK, exact
arithmetic, textbook special cases, the real oracle and the paper's lemmas.

The paper defines LSE and GLS over C (Sec. 1).  Each test checks the complex
oracle against something other than itself, chosen so that a plausible slip
(a missing conjugate, a wrong sign in Alg. 1 / Alg. 3, a transposed factor)
fails at least one of them.
"""
from fractions import Fraction

import numpy as np
import pytest
import scipy.linalg.lapack as lapack

from paper_2406_16499_gb300 import inputs as I

U = np.finfo(np.float64).eps / 2


def rel(a, b):
    nb = np.linalg.norm(b)
    return np.linalg.norm(np.asarray(a) - np.asarray(b)) / (nb if nb else 1.0)


def exact_complex_solve(K, rhs):
    """K s = rhs in exact rationals, through the real embedding
    [Re K, -Im K; Im K, Re K] [Re s; Im s] = [Re rhs; Im rhs]."""
    N = len(rhs)
    M = np.block([[K.real, -K.imag], [K.imag, K.real]])
    r = np.concatenate([rhs.real, rhs.imag])
    n2 = 2 * N
    a = [[Fraction(float(M[i, j])) for j in range(n2)] + [Fraction(float(r[i]))] for i in range(n2)]
    for c in range(n2):
        piv = next(k for k in range(c, n2) if a[k][c] != 0)
        a[c], a[piv] = a[piv], a[c]
        for k in range(n2):
            if k != c and a[k][c] != 0:
                f = a[k][c] / a[c][c]
                a[k] = [x - f * y for x, y in zip(a[k], a[c])]
    s = [float(a[i][n2] / a[i][i]) for i in range(n2)]
    return np.array(s[:N]) + 1j * np.array(s[N:])


# ------------------------------------------------------------ Householder --

@pytest.mark.parametrize("k,seed", [(1, 0), (5, 1), (17, 2)])
def test_reflector_maps_onto_a_real_multiple_of_e1(k, seed):
    """xLARFG convention: H = I - tau v v^H is unitary, H^H (alpha; x) =
    (beta; 0), beta real with the sign opposite to Re alpha."""
    from oracle import zoracle as Z
    g = np.random.default_rng(seed)
    a = g.standard_normal(k + 1) + 1j * g.standard_normal(k + 1)
    tau, v, beta = Z.zhouse(a[0], a[1:])
    H = np.eye(k + 1) - tau * np.outer(v, v.conj())
    assert np.abs(H.conj().T @ H - np.eye(k + 1)).max() < 1e-14
    out = H.conj().T @ a
    assert abs(out[0] - beta) < 1e-13 and np.abs(out[1:]).max() < 1e-13
    assert np.isreal(beta) and np.sign(beta) == -np.sign(a[0].real)
    assert abs(abs(beta) - np.linalg.norm(a)) < 1e-13


# -------------------------------------------------------------- LAPACK --

@pytest.mark.parametrize("m,n,p,ca,cb", [(30, 12, 4, 1e3, 1e1), (20, 20, 5, 1e2, 1e1),
                                         (9, 14, 6, 1e2, 1e1), (25, 10, 10, 1e1, 1e1)])
def test_complex_lse_truth_matches_lapack_zgglse(m, n, p, ca, cb):
    from oracle import zoracle as Z
    P = I.zlse_svd(700 + m + n + p, m, n, p, ca, cb)
    t = Z.zlse_truth(P["A"], P["B"], P["b"], P["d"])
    xl = lapack.zgglse(P["A"].copy(order="F"), P["B"].copy(order="F"), P["b"].copy(), P["d"].copy())[3]
    assert rel(t["x"], xl) < 50 * max(ca, cb) * U


def test_complex_gls_identity_v_is_least_squares():
    """V = I: min ||d - W x|| with y = d - W x and z = y (eq. link)."""
    from oracle import zoracle as Z
    g = I.rng(9)
    W = I.zsvd_matrix(g, 24, 7, I.logspace_sigma(7, 1e2))
    d = I.zgauss(g, 24)
    t = Z.zgls_truth(W, np.eye(24), d)
    x = np.linalg.lstsq(W, d, rcond=None)[0]
    assert rel(t["x"], x) < 1e-12
    assert rel(t["y"], d - W @ x) < 1e-12
    assert rel(t["z"], t["y"]) < 1e-12


def test_complex_gls_square_v_is_weighted_least_squares():
    """n = p, V nonsingular: min ||V^{-1}(d - W x)||, y = V^{-1}(d - W x)."""
    from oracle import zoracle as Z
    G = I.zgls_svd(13, 18, 5, 18, 1e2, 1e1)
    W, V, d = G["W"], G["V"], G["d"]
    t = Z.zgls_truth(W, V, d)
    x = np.linalg.lstsq(np.linalg.solve(V, W), np.linalg.solve(V, d), rcond=None)[0]
    assert rel(t["x"], x) < 1e-11
    assert rel(t["y"], np.linalg.solve(V, d - W @ x)) < 1e-11


# --------------------------------------------------------------- exact --

@pytest.mark.parametrize("m,n,p", [(4, 3, 1), (3, 4, 2), (5, 3, 3)])
def test_complex_lse_exact_rational_kkt(m, n, p):
    from oracle import zoracle as Z
    P = I.zlse_svd(40 + m + n + p, m, n, p, 1e1, 1e1)
    K = Z.zlse_kkt(P["A"], P["B"])
    s = exact_complex_solve(K, np.concatenate([P["b"], P["d"], np.zeros(n)]))
    t = Z.zlse_truth(P["A"], P["B"], P["b"], P["d"])
    assert rel(t["x"], s[m + p:]) < 1e-14
    assert rel(t["r"], s[:m]) < 1e-13
    assert rel(t["v"], -s[m:m + p]) < 1e-13


@pytest.mark.parametrize("n,m,p", [(4, 2, 3), (3, 3, 3), (5, 2, 4)])
def test_complex_gls_exact_rational_kkt(n, m, p):
    from oracle import zoracle as Z
    G = I.zgls_svd(50 + n + m + p, n, m, p, 1e1, 1e1)
    K = Z.zgls_kkt(G["W"], G["V"])
    s = exact_complex_solve(K, np.concatenate([np.zeros(p), G["d"], np.zeros(m)]))
    t = Z.zgls_truth(G["W"], G["V"], G["d"])
    assert rel(t["x"], s[p + n:]) < 1e-13
    assert rel(t["y"], s[:p]) < 1e-13
    assert rel(t["z"], -s[p:p + n]) < 1e-13


# --------------------------------------------------- real special case --

def test_complex_oracle_on_real_data_matches_the_real_oracle(oracle_mod):
    """Real inputs: the complex restatement and the independent real oracle
    (plain C, Alg. 1-4 in reversed coordinates) reach the same solutions."""
    from oracle import zoracle as Z
    P = I.lse_svd(61, 40, 18, 5, 1e3, 1e1)
    zr = Z.zlse_solve(P["A"], P["B"], P["b"], P["d"], fact="fp32")
    tr = oracle_mod.lse_truth(P["A"], P["B"], P["b"], P["d"])
    assert zr["status"] == 0 and rel(zr["x"], tr["x"]) < 1e-12
    assert np.abs(np.asarray(zr["x"]).imag).max() == 0.0
    G = I.gls_svd(62, 30, 8, 35, 1e3, 1e1)
    zg = Z.zgls_solve(G["W"], G["V"], G["d"], fact="fp32")
    tg = oracle_mod.gls_truth(G["W"], G["V"], G["d"])
    assert zg["status"] == 0 and rel(zg["x"], tg["x"]) < 1e-12 and rel(zg["y"], tg["y"]) < 1e-12


# ------------------------------------------------ factorization lemmas --

@pytest.mark.parametrize("fact,tol", [("fp64", 1e-13), ("fp32", 2e-5)])
def test_complex_grq_and_gqr_invariants(fact, tol):
    """Lemma 4.5 / 4.6: backward error and unitarity of the factors at u_f."""
    from oracle import zoracle as Z
    P = I.zlse_svd(71, 50, 30, 8, 1e3, 1e1)
    F = Z.zlse_factor(P["A"], P["B"], fact)
    Q, R, Zm, T = (np.asarray(F[k], np.complex128) for k in ("Q", "R", "Z", "T"))
    m, n, p = 50, 30, 8
    B0 = np.hstack([np.zeros((p, n - p)), R]) @ Q
    assert np.linalg.norm(P["B"] - B0) / np.linalg.norm(P["B"]) < tol
    assert np.linalg.norm(P["A"] - Zm @ T @ Q) / np.linalg.norm(P["A"]) < tol
    for U_ in (Q, Zm):
        assert np.linalg.norm(U_.conj().T @ U_ - np.eye(len(U_))) < tol * 10
    assert np.allclose(np.tril(R, -1), 0) and np.allclose(np.tril(T, -1), 0)
    G = I.zgls_svd(72, 40, 10, 45, 1e3, 1e1)
    F = Z.zgls_factor(G["W"], G["V"], fact)
    Q, R, Zm, T = (np.asarray(F[k], np.complex128) for k in ("Q", "R", "Z", "T"))
    W0 = Q @ np.vstack([R, np.zeros((30, 10))])
    assert np.linalg.norm(G["W"] - W0) / np.linalg.norm(G["W"]) < tol
    assert np.linalg.norm(G["V"] - Q @ T @ Zm) / np.linalg.norm(G["V"]) < tol
    assert np.allclose(T[:, :45 - 40], 0)                     # T = [0, T^] for n <= p


# ------------------------------------------------- Alg. 1-4 over C --

def test_complex_one_correction_with_exact_factors_lands_on_the_solution():
    """With FP64 factors one Alg. 1 / Alg. 3 step from a perturbed point
    solves the correction system, so the next iterate is the solution (this
    pins the conjugates and the readings Dz = -Q h, T22 g2 = u2 over C)."""
    from oracle import zoracle as Z
    g = np.random.default_rng(4)
    P = I.zlse_svd(81, 26, 14, 5, 1e2, 1e1)
    A, B, b, d = P["A"], P["B"], P["b"], P["d"]
    t = Z.zlse_truth(A, B, b, d)
    F = Z.zlse_factor(A, B, "fp64")
    x, r, v = (t[k] + 1e-3 * I.zgauss(g, len(t[k])) for k in ("x", "r", "v"))
    dr, dv, dx = Z.zlse_correction(F, *Z.zlse_residual(A, B, b, d, x, r, v))
    assert rel(x + dx, t["x"]) < 1e-12 and rel(r + dr, t["r"]) < 1e-11 and rel(v + dv, t["v"]) < 1e-11
    G = I.zgls_svd(82, 20, 6, 24, 1e2, 1e1)
    W, V, dd = G["W"], G["V"], G["d"]
    t = Z.zgls_truth(W, V, dd)
    F = Z.zgls_factor(W, V, "fp64")
    x, y, z = (t[k] + 1e-3 * I.zgauss(g, len(t[k])) for k in ("x", "y", "z"))
    dy, dz, dx = Z.zgls_correction(F, *Z.zgls_residual(W, V, dd, x, y, z))
    assert rel(x + dx, t["x"]) < 1e-12 and rel(y + dy, t["y"]) < 1e-11 and rel(z + dz, t["z"]) < 1e-11


def test_complex_initial_multipliers_satisfy_the_kkt_rows():
    """Sec. 3.1 / 3.2: A^H r0 = B^H v0 and W^H z0 = 0, y0 = V^H z0 up to the
    factor precision (FP32 factors)."""
    from oracle import zoracle as Z
    P = I.zlse_svd(91, 40, 20, 6, 1e2, 1e1)
    A, B, b, d = P["A"], P["B"], P["b"], P["d"]
    F = Z.zlse_factor(A, B, "fp32")
    x = Z.zlse_nullspace(F, b, d)
    r = b - A @ x
    v = Z.zlse_init_v(F, A, r)
    assert rel(B.conj().T @ v, A.conj().T @ r) < 1e-4
    G = I.zgls_svd(92, 30, 8, 36, 1e2, 1e1)
    F = Z.zgls_factor(G["W"], G["V"], "fp32")
    x, y = Z.zgls_paige(F, G["d"])
    z = Z.zgls_init_z(F, y)
    assert np.linalg.norm(G["W"].conj().T @ z) / (np.linalg.norm(G["W"]) * np.linalg.norm(z)) < 1e-5
    assert rel(G["V"].conj().T @ z, y) < 1e-4


@pytest.mark.parametrize("kappa", [1e3, 1e5])
def test_complex_mixed_precision_refinement_reaches_fp64_accuracy(kappa):
    """Alg. 2 / Alg. 4 with complex64 factors and complex128 residuals meet
    the eq. lse-stop / gls-stop bar and the forward-error bar of the real
    path (Table 4 / 5 behaviour below kappa ~ 1/u_f)."""
    from oracle import zoracle as Z
    P = I.zlse_svd(101, 60, 30, 6, kappa, 1e1)
    out = Z.zlse_solve(P["A"], P["B"], P["b"], P["d"], fact="fp32")
    met = Z.zlse_metrics(P["A"], P["B"], P["b"], P["d"], out["x"], out["r"], out["v"])
    t = Z.zlse_truth(P["A"], P["B"], P["b"], P["d"])
    assert out["status"] == 0 and met["eta"] < 1e-14 and met["e_con"] < 1e-14
    assert rel(out["x"], t["x"]) < 10 * kappa * 1.1e-16 * 10
    G = I.zgls_svd(102, 40, 10, 48, kappa, 1e1)
    out = Z.zgls_solve(G["W"], G["V"], G["d"], fact="fp32")
    met = Z.zgls_metrics(G["W"], G["V"], G["d"], out["x"], out["y"], out["z"])
    assert out["status"] == 0 and met["eta"] < 1e-14 and met["e_con"] < 1e-14


def test_complex_refinement_fails_beyond_the_single_precision_limit():
    """Table 4: with u_f = single, classical IR stops converging once
    kappa is well beyond 1/u_f."""
    from oracle import zoracle as Z
    P = I.zlse_svd(111, 60, 30, 6, 1e10, 1e1)
    out = Z.zlse_solve(P["A"], P["B"], P["b"], P["d"], fact="fp32", maxit=15)
    assert out["status"] != 0


def test_complex_generators_realise_the_requested_spectra():
    """zhaar gives orthonormal columns over C, zsvd_matrix the requested
    singular values, the problem generators consistent right-hand sides, and
    a seed always the same arrays."""
    g = I.rng(5)
    Q = I.zhaar(g, 30, 12)
    assert np.iscomplexobj(Q) and np.abs(Q.conj().T @ Q - np.eye(12)).max() < 1e-13
    sig = I.logspace_sigma(12, 1e4)
    M = I.zsvd_matrix(g, 30, 12, sig)
    assert np.allclose(np.linalg.svd(M, compute_uv=False), sig, rtol=1e-10)
    P = I.zlse_svd(4, 20, 10, 3, 1e2, 1e1)
    assert np.linalg.norm(P["B"] @ P["x_true"] - P["d"]) < 1e-13 * np.linalg.norm(P["d"])
    G = I.zgls_svd(6, 15, 5, 18, 1e2, 1e1)
    assert np.iscomplexobj(G["W"]) and np.iscomplexobj(G["d"])
    assert np.array_equal(I.zlse_svd(4, 20, 10, 3, 1e2, 1e1)["A"], P["A"])


# ----------------------------------------------------- GMRES-IR over C --

def _dense(op, N):
    return np.column_stack([op(e) for e in np.eye(N, dtype=np.complex128)])


def _bd_roots():
    return np.sort(np.roots([1, -1, -2, 1]).real), np.array([(1 - 5 ** 0.5) / 2, (1 + 5 ** 0.5) / 2])


@pytest.mark.parametrize("m,n,p,a,b", [(14, 9, 4, 0.7, 1.3), (12, 12, 5, 1.0, 1.0)])
def test_complex_lse_preconditioned_matrix_spectrum(m, n, p, a, b):
    """Sec. 5.2 over C: with exact factors M_l F~ M_r is Hermitian with the
    eigenvalues 1, (1 +- sqrt 5)/2 and the roots of x^3 - x^2 - 2x + 1
    (multiplicities m-n, n-p, p), so kappa_2 < 9.0985."""
    from oracle import zoracle as Z
    P = I.zlse_svd(121 + m, m, n, p, 1e3, 1e1)
    bd = Z.ZLseBD(Z.zlse_factor(P["A"], P["B"], "fp64"), P["A"], P["B"], a, b)
    M = _dense(lambda t: bd.Ml(bd.Fmul(bd.Mr(t))), m + n + p)
    assert np.abs(M - M.conj().T).max() < 1e-12
    cubic, gold = _bd_roots()
    want = np.sort(np.concatenate([np.repeat(cubic, p), np.repeat(gold, n - p), np.ones(m - n)]))
    assert np.abs(np.sort(np.linalg.eigvalsh(M)) - want).max() < 1e-10
    assert np.linalg.cond(M) <= 9.0985


@pytest.mark.parametrize("n,m,p,a,b", [(9, 3, 12, 0.6, 1.7), (10, 4, 10, 1.0, 1.0)])
def test_complex_gls_preconditioned_matrix_spectrum(n, m, p, a, b):
    """Sec. 5.3 over C: multiplicities m, n-m, p-n."""
    from oracle import zoracle as Z
    G = I.zgls_svd(131 + n, n, m, p, 1e3, 1e1)
    bd = Z.ZGlsBD(Z.zgls_factor(G["W"], G["V"], "fp64"), G["W"], G["V"], a, b)
    M = _dense(lambda t: bd.Ml(bd.Fmul(bd.Mr(t))), m + n + p)
    cubic, gold = _bd_roots()
    want = np.sort(np.concatenate([np.repeat(cubic, m), np.repeat(gold, n - m), np.ones(p - n)]))
    assert np.abs(np.sort(np.linalg.eigvalsh(M)) - want).max() < 1e-10


def test_complex_gmres_full_restart_is_exact():
    from oracle import zoracle as Z
    g = np.random.default_rng(8)
    K = g.standard_normal((30, 30)) + 1j * g.standard_normal((30, 30)) + 8 * np.eye(30)
    rhs = g.standard_normal(30) + 1j * g.standard_normal(30)
    x, k, rel_ = Z.zgmres(lambda v: K @ v, rhs, tol=1e-13, restart=30, maxit=30)
    assert rel_ < 1e-12 and rel(x, np.linalg.solve(K, rhs)) < 1e-10


def test_complex_gmres_ir_beyond_the_classical_limit():
    """Table 4 over C: at kappa = 1e9 classical IR with complex64 factors
    does not converge, GMRES-IR with the split preconditioner does."""
    from oracle import zoracle as Z
    P = I.zlse_svd(5, 120, 40, 6, 1e9, 1e1)
    A, B, b, d = P["A"], P["B"], P["b"], P["d"]
    assert Z.zlse_solve(A, B, b, d, maxit=15)["status"] != 0
    out = Z.zlse_gmres_ir(A, B, b, d)
    met = Z.zlse_metrics(A, B, b, d, out["x"], out["r"], out["v"])
    assert out["status"] == 0 and met["eta"] < 1e-14
    G = I.zgls_svd(6, 40, 10, 48, 1e3, 1e1)
    out = Z.zgls_gmres_ir(G["W"], G["V"], G["d"])
    met = Z.zgls_metrics(G["W"], G["V"], G["d"], out["x"], out["y"], out["z"])
    assert out["status"] == 0 and met["eta"] < 1e-14


# --------------------------------------------------------- real embedding --

def _embed(Z):
    Z = np.asarray(Z)
    return np.block([[Z.real, -Z.imag], [Z.imag, Z.real]])


@pytest.mark.parametrize("m,n,p", [(30, 12, 4), (20, 20, 6), (9, 10, 5)])
def test_lse_real_embedding_has_the_complex_solution(m, n, p):
    """The GPU solves a complex LSE as the real LSE of E(Z) = [Re Z, -Im Z;
    Im Z, Re Z]: the real oracle's solution of the embedded problem is
    [Re x; Im x], [Re r; Im r], [Re v; Im v] of the complex oracle's (both
    plain KKT definitions), and E keeps the singular values (each twice)."""
    import oracle
    from oracle import zoracle as Z
    P = I.zlse_svd(m + n + p, m, n, p, 1e3, 1e1)
    A, B, b, d = P["A"], P["B"], P["b"], P["d"]
    t = Z.zlse_truth(A, B, b, d)
    e = oracle.lse_truth(_embed(A), _embed(B), np.concatenate([b.real, b.imag]), np.concatenate([d.real, d.imag]))
    assert rel(e["x"], np.concatenate([t["x"].real, t["x"].imag])) < 1e-12
    assert rel(e["r"], np.concatenate([t["r"].real, t["r"].imag])) < 1e-12
    assert rel(e["v"], np.concatenate([t["v"].real, t["v"].imag])) < 1e-12
    sv = np.linalg.svd(A, compute_uv=False)
    assert np.allclose(np.linalg.svd(_embed(A), compute_uv=False), np.repeat(sv, 2), rtol=1e-12)


@pytest.mark.parametrize("n,m,p", [(20, 8, 25), (12, 12, 12), (15, 9, 10)])
def test_gls_real_embedding_has_the_complex_solution(n, m, p):
    import oracle
    from oracle import zoracle as Z
    G = I.zgls_svd(n + m + p, n, m, p, 1e2, 1e1)
    W, V, d = G["W"], G["V"], G["d"]
    t = Z.zgls_truth(W, V, d)
    e = oracle.gls_truth(_embed(W), _embed(V), np.concatenate([d.real, d.imag]))
    assert rel(e["x"], np.concatenate([t["x"].real, t["x"].imag])) < 1e-12
    ty = np.concatenate([t["y"].real, t["y"].imag])
    # (m = n: y = 0 up to rounding, so measure against the size of the solution)
    assert np.linalg.norm(e["y"] - ty) <= 1e-12 * max(np.linalg.norm(ty), np.linalg.norm(t["x"]))
