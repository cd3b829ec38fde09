"""Pins of the GMRES-IR oracle (Sec. 5) against the paper's closed forms and
its reported behaviour.

* With exact (FP64) factors the preconditioned matrix M_l F~ M_r has the
  eigenvalues 1, (1 +- sqrt 5)/2 and the roots of x^3 - x^2 - 2x + 1 with
  multiplicities m-n, n-p, p (LSE) and p-n, n-m, m (GLS) (Sec. 5.2, App. C);
  its 2-norm condition number is below C = 1 + 2 lambda3/lambda2 ~ 9.0984.
  This pins F~, both preconditioners and their scalings at any alpha, beta.
* For the wide shapes (LSE n > m, GLS n > p) the same product equals the
  block matrices the paper gives for those preconditioners.
* GMRES with full restart solves small systems exactly (numpy solve).
* Table 4 / Table 5: with u_f = single, GMRES-IR reaches FP64-level accuracy
  where classical IR does not (kappa = 1e9, one small singular value).
"""
import json
import os

import numpy as np
import pytest

from paper_2406_16499_gb300 import inputs as I

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "paper_tables.json")


def _roots():
    cubic = np.sort(np.roots([1, -1, -2, 1]).real)
    return cubic, np.array([(1 - 5 ** 0.5) / 2, (1 + 5 ** 0.5) / 2])


def _dense(op, N):
    return np.column_stack([op(e) for e in np.eye(N)])


@pytest.mark.parametrize("m,n,p,a,b", [(14, 9, 4, 0.7, 1.3), (20, 12, 12, 2.0, 0.5), (11, 11, 3, 1.0, 1.0)])
def test_lse_preconditioned_spectrum(oracle_mod, m, n, p, a, b):
    from oracle import gmres as G
    gold = json.load(open(GOLDEN))["bd_spectrum"]
    P = I.lse_svd(m * n + p, m, n, p, 1e3, 1e1)
    F = oracle_mod.lse_factor(P["A"], P["B"], "fp64")
    bd = G.LseBD(F, P["A"], P["B"], a, b)
    M = _dense(lambda t: bd.Ml(bd.Fmul(bd.Mr(t))), m + n + p)
    ev = np.sort(np.linalg.eigvals(M).real)
    cubic, gold_r = _roots()
    assert np.allclose(cubic, gold["cubic_roots"], atol=1e-4)
    want = np.sort(np.concatenate([np.repeat(cubic, p), np.repeat(gold_r, n - p), np.ones(m - n)]))
    assert np.allclose(ev, want, atol=1e-8)
    assert np.linalg.cond(M) <= gold["C"] + 1e-3


@pytest.mark.parametrize("n,m,p,a,b", [(9, 3, 12, 0.6, 1.7), (10, 4, 10, 1.0, 1.0), (12, 5, 20, 3.0, 0.25)])
def test_gls_preconditioned_spectrum(oracle_mod, n, m, p, a, b):
    from oracle import gmres as G
    G_ = I.gls_svd(n * m + p, n, m, p, 1e3, 1e1)
    F = oracle_mod.gls_factor(G_["W"], G_["V"], "fp64")
    bd = G.GlsBD(F, G_["W"], G_["V"], a, b)
    M = _dense(lambda t: bd.Ml(bd.Fmul(bd.Mr(t))), m + n + p)
    ev = np.sort(np.linalg.eigvals(M).real)
    cubic, gold_r = _roots()
    want = np.sort(np.concatenate([np.repeat(cubic, m), np.repeat(gold_r, n - m), np.ones(p - n)]))
    assert np.allclose(ev, want, atol=1e-8)
    assert np.linalg.cond(M) <= 9.0985


@pytest.mark.parametrize("m,n,p,a,b", [(8, 12, 6, 0.7, 1.3), (10, 14, 4, 1.0, 1.0), (5, 9, 9, 2.0, 0.5)])
def test_lse_wide_preconditioned_matrix(oracle_mod, m, n, p, a, b):
    """n > m (eq. lse-bdpre-nlarge): with exact (FP64) factors M_l F~ M_r is
    [I_m 0 Zb; 0 0 Ib; Zb^T Ib^T 0], Zb = [Z, 0] (m x n), Ib = [0, I_p]
    (Sec. 5.2), and its 2-norm condition number stays below C = 9.0984."""
    from oracle import gmres as G
    P = I.lse_svd(m * n + p + 7, m, n, p, 1e3, 1e1)
    F = oracle_mod.lse_factor(P["A"], P["B"], "fp64")
    bd = G.LseBD(F, P["A"], P["B"], a, b)
    M = _dense(lambda t: bd.Ml(bd.Fmul(bd.Mr(t))), m + n + p)
    Zb = np.hstack([oracle_mod.explicit(F, "Z"), np.zeros((m, n - m))])
    Ib = np.hstack([np.zeros((p, n - p)), np.eye(p)])
    X = np.zeros((m + p + n, m + p + n))
    X[:m, :m] = np.eye(m)
    X[:m, m + p:], X[m + p:, :m] = Zb, Zb.T
    X[m:m + p, m + p:], X[m + p:, m:m + p] = Ib, Ib.T
    assert np.abs(M - X).max() < 1e-10
    assert np.linalg.cond(M) <= 9.0985


@pytest.mark.parametrize("n,m,p,a,b", [(12, 4, 8, 0.6, 1.7), (10, 6, 5, 1.0, 1.0), (9, 3, 6, 3.0, 0.25)])
def test_gls_wide_preconditioned_matrix(oracle_mod, n, m, p, a, b):
    """n > p (eq. gls-bdpre-nlarge): with exact factors M_l F~ M_r is
    [I_p Zc^T 0; Zc 0 Ic; 0 Ic^T 0], Zc = [0; Z] (n x p), Ic = [I_m; 0]
    (Sec. 5.3), condition number below C."""
    from oracle import gmres as G
    G_ = I.gls_svd(n * m + p + 7, n, m, p, 1e3, 1e1)
    F = oracle_mod.gls_factor(G_["W"], G_["V"], "fp64")
    bd = G.GlsBD(F, G_["W"], G_["V"], a, b)
    M = _dense(lambda t: bd.Ml(bd.Fmul(bd.Mr(t))), m + n + p)
    Zc = np.vstack([np.zeros((n - p, p)), oracle_mod.explicit(F, "Z")])
    Ic = np.vstack([np.eye(m), np.zeros((n - m, m))])
    X = np.zeros((p + n + m, p + n + m))
    X[:p, :p] = np.eye(p)
    X[:p, p:p + n], X[p:p + n, :p] = Zc.T, Zc
    X[p:p + n, p + n:], X[p + n:, p:p + n] = Ic, Ic.T
    assert np.abs(M - X).max() < 1e-10
    assert np.linalg.cond(M) <= 9.0985


@pytest.mark.parametrize("kappa", [1e3, 1e6])
def test_gmres_ir_wide_shapes_converge(oracle_mod, kappa):
    """GMRES-IR with the wide-shape preconditioners (LSE n > m, GLS n > p)
    reaches FP64-level accuracy with u_f = single while u_f kappa(A)
    kappa(B) stays below one (the condition of Sec. 5.2 / 5.3)."""
    from oracle import gmres as G
    P = I.lse_paper(401, 40, 64, 32, kappa)
    out = G.lse_gmres_ir(P["A"], P["B"], P["b"], P["d"])
    met = oracle_mod.lse_metrics(P["A"], P["B"], P["b"], P["d"], out["x"], out["r"], out["v"])
    assert out["status"] == 0 and met["eta"] < 1e-14 and met["e_con"] < 1e-14
    Gp = I.gls_paper(501, 48, 16, 40, kappa)
    out = G.gls_gmres_ir(Gp["W"], Gp["V"], Gp["d"])
    met = oracle_mod.gls_metrics(Gp["W"], Gp["V"], Gp["d"], out["x"], out["y"], out["z"])
    assert out["status"] == 0 and met["eta"] < 1e-14


def test_gmres_full_restart_is_exact():
    from oracle import gmres as G
    g = np.random.default_rng(3)
    Mat = g.standard_normal((40, 40)) + 8 * np.eye(40)
    rhs = g.standard_normal(40)
    x, k, rel = G.gmres(lambda v: Mat @ v, rhs, tol=1e-13, restart=40, maxit=40)
    assert rel < 1e-12 and k <= 40
    assert np.linalg.norm(x - np.linalg.solve(Mat, rhs)) < 1e-10 * np.linalg.norm(x)


def test_preconditioned_correction_solves_the_system(oracle_mod):
    """M_r t with t from GMRES on M_l F~ M_r t = M_l s~ solves F~ du = s~,
    and unscaling gives the correction of eq. correction-system-lse."""
    from oracle import gmres as G
    P = I.lse_svd(31, 60, 30, 6, 1e3, 1e1)
    A, B = P["A"], P["B"]
    F = oracle_mod.lse_factor(A, B, "fp32")
    bd = G.LseBD(F, A, B, 0.9, 1.0)
    g = np.random.default_rng(5)
    f1, f2, f3 = g.standard_normal(60), g.standard_normal(6), g.standard_normal(30)
    t, k, rel = G.gmres(lambda v: bd.Ml(bd.Fmul(bd.Mr(v))), bd.Ml(bd.scale_rhs(f1, f2, f3)), tol=1e-12,
                        restart=30, maxit=300)
    dr, dv, dx = bd.unscale(bd.Mr(t))
    assert np.linalg.norm(dr + A @ dx - f1) < 1e-9 * np.linalg.norm(f1)
    assert np.linalg.norm(B @ dx - f2) < 1e-9 * np.linalg.norm(f2) + 1e-9
    assert np.linalg.norm(A.T @ dr - B.T @ dv - f3) < 1e-9 * np.linalg.norm(f3)


@pytest.mark.parametrize("kappa", [1e3, 1e7])
def test_gmres_ir_converges_geometric(oracle_mod, kappa):
    """Table 4 / 5 (GMRES-BD rows): converges to FP64-level accuracy for
    kappa up to 1e7 (geometric singular values)."""
    from oracle import gmres as G
    P = I.lse_paper(400, 512, 64, 2, kappa)
    out = G.lse_gmres_ir(P["A"], P["B"], P["b"], P["d"])
    met = oracle_mod.lse_metrics(P["A"], P["B"], P["b"], P["d"], out["x"], out["r"], out["v"])
    assert out["status"] == 0 and met["eta"] < 1e-14 and met["e_con"] < 1e-14
    Gp = I.gls_paper(500, 64, 2, 512, kappa)
    out = G.gls_gmres_ir(Gp["W"], Gp["V"], Gp["d"])
    met = oracle_mod.gls_metrics(Gp["W"], Gp["V"], Gp["d"], out["x"], out["y"], out["z"])
    assert out["status"] == 0 and met["eta"] < 1e-14


def test_gmres_ir_beyond_classical_limit(oracle_mod):
    """Table 4: at kappa = 1e9 classical IR with u_f = single does not
    converge while GMRES-IR with the block-diagonal split preconditioner does
    (shown with one small singular value, xLATM1 mode-2 pattern)."""
    from oracle import gmres as G
    P = I.lse_paper(7, 512, 64, 2, 1e9, mode=2)
    A, B, b, d = P["A"], P["B"], P["b"], P["d"]
    cl = oracle_mod.lse_solve(A, B, b, d, fact="fp32", tol=1e-13)
    assert cl["status"] != 0
    out = G.lse_gmres_ir(A, B, b, d)
    met = oracle_mod.lse_metrics(A, B, b, d, out["x"], out["r"], out["v"])
    assert out["status"] == 0 and met["eta"] < 1e-14 and met["e_con"] < 1e-14


@pytest.mark.parametrize("a,b", [(0.7, 1.3), (2.0, 0.5)])
def test_left_preconditioner_inverts_ftilde_with_exact_factors(oracle_mod, a, b):
    """Sec. 5.1: the left preconditioner is F~^{-1} applied through the
    correction solvers (Alg. 1 / Alg. 3); with FP64 factors M F~ = I."""
    from oracle import gmres as G
    g = np.random.default_rng(11)
    P = I.lse_svd(201, 40, 20, 6, 1e3, 1e1)
    L = G.LseLeft(oracle_mod.lse_factor(P["A"], P["B"], "fp64"), P["A"], P["B"], a, b)
    u = g.standard_normal(40 + 6 + 20)
    assert np.linalg.norm(L.Ml(L.Fmul(u)) - u) <= 1e-10 * np.linalg.norm(u)
    Gp = I.gls_svd(202, 30, 8, 35, 1e3, 1e1)
    L = G.GlsLeft(oracle_mod.gls_factor(Gp["W"], Gp["V"], "fp64"), Gp["W"], Gp["V"], a, b)
    u = g.standard_normal(35 + 30 + 8)
    assert np.linalg.norm(L.Ml(L.Fmul(u)) - u) <= 1e-10 * np.linalg.norm(u)


def test_gmres_left_converges_beyond_the_classical_limit(oracle_mod):
    """Table 4, GMRES-Left column: converges at kappa = 1e9 where classical IR
    with u_f = single does not."""
    from oracle import gmres as G
    P = I.lse_paper(7, 512, 64, 2, 1e9, mode=2)
    A, B, b, d = P["A"], P["B"], P["b"], P["d"]
    out = G.lse_gmres_ir(A, B, b, d, precond="left")
    met = oracle_mod.lse_metrics(A, B, b, d, out["x"], out["r"], out["v"])
    assert out["status"] == 0 and met["eta"] < 1e-14 and met["e_con"] < 1e-14
