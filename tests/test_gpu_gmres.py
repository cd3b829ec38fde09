"""GMRES-IR on the GPU (Sec. 5) against the oracle.

* The building blocks through the C ABI -- F~(alpha, beta), the
  block-diagonal split preconditioners M_l, M_r and M_l F~ M_r -- element by
  element against oracle/gmres.py (LseBD, GlsBD) on the same factors' class:
  with FP64 factors on both sides the results agree to rounding (scaled by
  the conditioning of the triangular factors); with FP32 factors to the
  factor precision.
* Full solves with refine = GMRES reach the same FP64-level bar as the
  classical path (eq. lse-stop / gls-stop ratios <= 1e-14, constraint
  residual, forward error against the oracle's solution).
* Table 4's behaviour: at kappa = 1e9 (one small singular value) classical
  IR with FP32 factors does not converge and GMRES-IR does.
* The wide shapes (LSE n > m, GLS n > p) with the split preconditioners of
  eq. lse-bdpre-nlarge / gls-bdpre-nlarge: pieces against the oracle and
  full solves at the FP64 bar.
* The left preconditioner of Sec. 5.1 (M ~ F~^-1 applied by the correction
  solver): M and M F~ against the oracle's LseLeft / GlsLeft, M F~ = I with
  FP64 factors, and full solves on every shape, wide ones included.
"""
import numpy as np
import pytest

from paper_2406_16499_gb300 import inputs as I
from gpu_util import dev, host, rel, zeros
from test_gpu_solve import check_gls, check_lse, run_gls, run_lse

pytestmark = pytest.mark.gpu
U32 = 2.0 ** -24


@pytest.fixture(scope="module")
def h():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2406_16499_gb300 import mpir
    hd = mpir.Handle()
    yield hd
    hd.close()


def _pieces(bd):
    return {"F": bd.Fmul, "Ml": bd.Ml, "Mr": bd.Mr, "op": lambda t: bd.Ml(bd.Fmul(bd.Mr(t)))}


LSE_SHAPES = [(300, 200, 37), (257, 130, 0), (160, 160, 40), (700, 333, 129)]
GLS_SHAPES = [(200, 70, 333), (150, 150, 150), (129, 1, 300), (333, 129, 700)]
# wide shapes: LSE n > m (eq. lse-bdpre-nlarge), GLS n > p (eq. gls-bdpre-nlarge)
LSE_WIDE = [(90, 100, 45), (60, 100, 70), (129, 200, 100)]
GLS_WIDE = [(200, 120, 100), (150, 100, 60), (300, 250, 97)]


@pytest.mark.parametrize("m,n,p", LSE_SHAPES + LSE_WIDE)
@pytest.mark.parametrize("fact,tol", [("fp64", 1e-11), ("fp32", 5e-4)])
def test_lse_bd_pieces_match_oracle(h, oracle_mod, m, n, p, fact, tol):
    from oracle import gmres as G
    P = I.lse_svd(11 * m + n + p, m, n, p, 1e2, 1e1)
    A, B = P["A"], P["B"]
    a, b = 0.37, 1.7
    F = oracle_mod.lse_factor(A, B, fact)
    bd = G.LseBD(F, A, B, a, b)
    dA, dB = dev(A), dev(B)
    h.lse_factor(dA, dB, fact=fact)
    g = np.random.default_rng(m + n + p)
    N = m + p + n
    if fact == "fp32":
        # two independent FP32 factorizations: each inverse of T1 is off by
        # about u_single kappa(T1), and the wide T1 = [T; 0, I] can be far
        # worse conditioned than A (the identity block is not scaled to T)
        tol = max(tol, U32 * np.linalg.cond(G.LseBD(oracle_mod.lse_factor(A, B, "fp64"), A, B, a, b).T1))
    for which, fn in _pieces(bd).items():
        u = g.standard_normal(N)
        out = zeros(N)
        h.lse_bd_apply(dA, dB, a, b, which, dev(u), out)
        want = fn(u)
        t = 1e-13 if which == "F" else tol
        assert rel(host(out), want) <= t, (which, rel(host(out), want))


@pytest.mark.parametrize("n,m,p", GLS_SHAPES + GLS_WIDE)
@pytest.mark.parametrize("fact,tol", [("fp64", 1e-11), ("fp32", 5e-4)])
def test_gls_bd_pieces_match_oracle(h, oracle_mod, n, m, p, fact, tol):
    from oracle import gmres as G
    Gp = I.gls_svd(13 * n + m + p, n, m, p, 1e2, 1e1)
    W, V = Gp["W"], Gp["V"]
    a, b = 2.5, 0.6
    F = oracle_mod.gls_factor(W, V, fact)
    bd = G.GlsBD(F, W, V, a, b)
    dW, dV = dev(W), dev(V)
    h.gls_factor(dW, dV, fact=fact)
    g = np.random.default_rng(n + m + p)
    N = p + n + m
    if fact == "fp32":
        tol = max(tol, U32 * np.linalg.cond(G.GlsBD(oracle_mod.gls_factor(W, V, "fp64"), W, V, a, b).T2))
    for which, fn in _pieces(bd).items():
        u = g.standard_normal(N)
        out = zeros(N)
        h.gls_bd_apply(dW, dV, a, b, which, dev(u), out)
        want = fn(u)
        t = 1e-13 if which == "F" else tol
        assert rel(host(out), want) <= t, (which, rel(host(out), want))


LSE_LEFT_SHAPES = LSE_SHAPES + [(90, 100, 45), (60, 100, 70)]        # the last two wide (m < n)
GLS_LEFT_SHAPES = GLS_SHAPES + [(200, 120, 100), (150, 100, 60)]     # the last two with n > p


@pytest.mark.parametrize("m,n,p", LSE_LEFT_SHAPES)
@pytest.mark.parametrize("fact,tol", [("fp64", 1e-11), ("fp32", 5e-4)])
def test_lse_left_pieces_match_oracle(h, oracle_mod, m, n, p, fact, tol):
    """The left preconditioner of Sec. 5.1 (M ~ F~^-1 through Alg. 1) and
    M F~ against oracle/gmres.py's LseLeft; with FP64 factors M F~ u = u to
    rounding (M is F~^-1 up to the factorization's backward error)."""
    from oracle import gmres as G
    P = I.lse_svd(17 * m + n + p, m, n, p, 1e2, 1e1)
    A, B = P["A"], P["B"]
    a, b = 0.37, 1.7
    F = oracle_mod.lse_factor(A, B, fact)
    lp = G.LseLeft(F, A, B, a, b)
    dA, dB = dev(A), dev(B)
    h.lse_factor(dA, dB, fact=fact)
    g = np.random.default_rng(m * n + p)
    N = m + p + n
    for which, fn in (("M", lp.Ml), ("left_op", lambda t: lp.Ml(lp.Fmul(t)))):
        u = g.standard_normal(N)
        out = zeros(N)
        h.lse_bd_apply(dA, dB, a, b, which, dev(u), out)
        assert rel(host(out), fn(u)) <= tol, (which, rel(host(out), fn(u)))
        if which == "left_op" and fact == "fp64":
            assert rel(host(out), u) <= 1e-10


@pytest.mark.parametrize("n,m,p", GLS_LEFT_SHAPES)
@pytest.mark.parametrize("fact,tol", [("fp64", 1e-11), ("fp32", 5e-4)])
def test_gls_left_pieces_match_oracle(h, oracle_mod, n, m, p, fact, tol):
    """As above for GLS (M through Alg. 3, oracle GlsLeft)."""
    from oracle import gmres as G
    Gp = I.gls_svd(19 * n + m + p, n, m, p, 1e2, 1e1)
    W, V = Gp["W"], Gp["V"]
    a, b = 2.5, 0.6
    F = oracle_mod.gls_factor(W, V, fact)
    lp = G.GlsLeft(F, W, V, a, b)
    dW, dV = dev(W), dev(V)
    h.gls_factor(dW, dV, fact=fact)
    g = np.random.default_rng(n * m + p)
    N = p + n + m
    for which, fn in (("M", lp.Ml), ("left_op", lambda t: lp.Ml(lp.Fmul(t)))):
        u = g.standard_normal(N)
        out = zeros(N)
        h.gls_bd_apply(dW, dV, a, b, which, dev(u), out)
        assert rel(host(out), fn(u)) <= tol, (which, rel(host(out), fn(u)))
        if which == "left_op" and fact == "fp64":
            assert rel(host(out), u) <= 1e-10


def test_preconditioned_operator_spectrum_on_gpu(h):
    """With FP64 factors the GPU's M_l F~ M_r, assembled column by column,
    has the closed-form spectrum of Sec. 5.2 / App. C: 1 (m - n times),
    (1 +- sqrt 5)/2 (n - p times each) and the roots of x^3 - x^2 - 2x + 1
    (p times each)."""
    import torch
    m, n, p = 40, 24, 9
    P = I.lse_svd(99, m, n, p, 1e3, 1e1)
    dA, dB = dev(P["A"]), dev(P["B"])
    h.lse_factor(dA, dB, fact="fp64")
    N = m + p + n
    cols = []
    for k in range(N):
        e = torch.zeros(N, dtype=torch.float64, device="cuda")
        e[k] = 1.0
        out = zeros(N)
        h.lse_bd_apply(dA, dB, 0.8, 1.4, "op", e, out)
        cols.append(host(out))
    ev = np.sort(np.linalg.eigvals(np.column_stack(cols)).real)
    cubic = np.sort(np.roots([1, -1, -2, 1]).real)
    gold = np.array([(1 - 5 ** 0.5) / 2, (1 + 5 ** 0.5) / 2])
    want = np.sort(np.concatenate([np.repeat(cubic, p), np.repeat(gold, n - p), np.ones(m - n)]))
    assert np.allclose(ev, want, atol=1e-8)


def test_lse_gmres_small_config(h, oracle_mod):
    """LSE m=200, n=100, p=20 solved with GMRES-IR (FP32 factors)."""
    P = I.lse_small()
    st, info, x, r, v = run_lse(h, P, refine="gmres")
    assert st == 0 and info.status == 0 and info.refine_used == 1 and info.escalated == 0
    assert info.inner_iters >= 1
    check_lse(oracle_mod, P, x, r, v)


@pytest.mark.parametrize("m,n,p,ca", [(333, 290, 77, 1e3), (1000, 513, 1, 1e4), (257, 129, 31, 1e5),
                                      (300, 120, 0, 1e3)])
def test_lse_gmres_shapes(h, oracle_mod, m, n, p, ca):
    P = I.lse_svd(m + 7 * n + p, m, n, p, ca, 1e1)
    st, info, x, r, v = run_lse(h, P, refine="gmres", escalate=False)
    assert st == 0 and info.inner_iters >= 1
    check_lse(oracle_mod, P, x, r, v)


@pytest.mark.parametrize("n,m,p,cw", [(300, 77, 300, 1e3), (257, 100, 400, 1e4), (129, 100, 140, 1e2)])
def test_gls_gmres_shapes(h, oracle_mod, n, m, p, cw):
    G = I.gls_svd(3 * n + m + p, n, m, p, cw, 1e1)
    st, info, x, y, z = run_gls(h, G, refine="gmres", escalate=False)
    assert st == 0 and info.inner_iters >= 1
    check_gls(oracle_mod, G, x, y, z)


def test_gls_gmres_square_w_matches_oracle(h, oracle_mod):
    """m = n: W is square, so y = 0 and z = 0 exactly and the f1, f3 bounds of
    eq. gls-stop vanish; GMRES-IR then cannot meet the relative stop test
    (the oracle's GMRES-IR reports the same), while x is accurate."""
    from oracle import gmres as Gm
    G = I.gls_svd(3 * 129 + 129 + 140, 129, 129, 140, 1e2, 1e1)
    ref = Gm.gls_gmres_ir(G["W"], G["V"], G["d"])
    st, info, x, y, z = run_gls(h, G, refine="gmres", escalate=False)
    assert st == ref["status"] == 3
    t = oracle_mod.gls_truth(G["W"], G["V"], G["d"])
    assert rel(x, t["x"]) <= 1e-12 and rel(ref["x"], t["x"]) <= 1e-12


def test_gls_gmres_ar1_reduced(h, oracle_mod):
    G = I.gls_ar1(seed=78, n=1024, m=256)
    st, info, x, y, z = run_gls(h, G, refine="gmres", escalate=False)
    assert st == 0
    check_gls(oracle_mod, G, x, y, z)


def test_gmres_ir_beyond_classical_limit(h, oracle_mod):
    """Table 4: kappa = 1e9 with one small singular value (xLATM1 mode-2
    pattern).  FP32 classical IR fails (no escalation allowed); GMRES-IR with
    the same FP32 factors reaches FP64-level accuracy, as the oracle's
    GMRES-IR does."""
    from oracle import gmres as G
    P = I.lse_paper(7, 512, 64, 2, 1e9, mode=2)
    st, info, x, r, v = run_lse(h, P, escalate=False)
    assert st != 0
    st, info, x, r, v = run_lse(h, P, refine="gmres", escalate=False)
    assert st == 0 and info.fact_used == 2
    # eta, e_con <= 1e-14 and forward error <= 10 kappa u against the
    # oracle's solution (kappa ~ 8e10 here, so x itself is only accurate to
    # ~1e-6 in any FP64 method)
    check_lse(oracle_mod, P, x, r, v)
    ref = G.lse_gmres_ir(P["A"], P["B"], P["b"], P["d"])
    assert ref["status"] == 0


@pytest.mark.parametrize("m,n,p,ca", [(333, 290, 77, 1e3), (257, 129, 31, 1e5), (300, 120, 0, 1e3),
                                      (90, 100, 45, 1e3), (60, 100, 70, 1e4)])
def test_lse_gmres_left_shapes(h, oracle_mod, m, n, p, ca):
    """GMRES-IR with the left preconditioner (Sec. 5.1), wide shapes
    included: the FP64 bar, and the oracle's left GMRES-IR converges too."""
    from oracle import gmres as Gm
    P = I.lse_svd(m + 5 * n + p, m, n, p, ca, 1e1)
    st, info, x, r, v = run_lse(h, P, refine="gmres_left", escalate=False)
    assert st == 0 and info.refine_used == 3 and info.inner_iters >= 1
    check_lse(oracle_mod, P, x, r, v)
    assert Gm.lse_gmres_ir(P["A"], P["B"], P["b"], P["d"], precond="left")["status"] == 0


@pytest.mark.parametrize("n,m,p,cw", [(300, 77, 300, 1e3), (257, 100, 400, 1e4), (200, 120, 100, 1e2),
                                      (150, 100, 60, 1e3)])
def test_gls_gmres_left_shapes(h, oracle_mod, n, m, p, cw):
    from oracle import gmres as Gm
    G = I.gls_svd(5 * n + m + p, n, m, p, cw, 1e1)
    st, info, x, y, z = run_gls(h, G, refine="gmres_left", escalate=False)
    assert st == 0 and info.refine_used == 3 and info.inner_iters >= 1
    check_gls(oracle_mod, G, x, y, z)
    assert Gm.gls_gmres_ir(G["W"], G["V"], G["d"], precond="left")["status"] == 0


def test_gmres_left_beyond_classical_limit(h, oracle_mod):
    """Table 4's kappa = 1e9 case with the left preconditioner: FP32 factors,
    no escalation, FP64-level result."""
    P = I.lse_paper(7, 512, 64, 2, 1e9, mode=2)
    st, info, x, r, v = run_lse(h, P, refine="gmres_left", escalate=False)
    assert st == 0 and info.fact_used == 2
    check_lse(oracle_mod, P, x, r, v)


@pytest.mark.parametrize("kappa", [1e3, 1e7])
def test_gls_gmres_paper_spectrum(h, oracle_mod, kappa):
    """GLS [W, V] with kappa_2 = kappa (Sec. 6.3, geometric spectrum)."""
    Gp = I.gls_paper(500, 64, 2, 512, kappa)
    st, info, x, y, z = run_gls(h, Gp, refine="gmres", escalate=False)
    assert st == 0
    met = oracle_mod.gls_metrics(Gp["W"], Gp["V"], Gp["d"], x, y, z)
    assert met["eta"] <= 1e-14


def test_gmres_is_deterministic(h):
    P = I.lse_svd(4242, 400, 200, 30, 1e4, 1e1)
    a = run_lse(h, P, refine="gmres", escalate=False)
    b = run_lse(h, P, refine="gmres", escalate=False)
    assert a[0] == 0 and np.array_equal(a[2], b[2]) and a[1].inner_iters == b[1].inner_iters


@pytest.mark.parametrize("m,n,p,ca", [(90, 100, 45, 1e3), (60, 100, 70, 1e4), (129, 200, 100, 1e3)])
def test_lse_gmres_wide_shapes(h, oracle_mod, m, n, p, ca):
    """n > m: the split preconditioner with T1 = [T; 0, I] (eq.
    lse-bdpre-nlarge) reaches the FP64 bar, as the oracle's GMRES-IR does."""
    from oracle import gmres as Gm
    P = I.lse_svd(m + 11 * n + p, m, n, p, ca, 1e1)
    st, info, x, r, v = run_lse(h, P, refine="gmres", escalate=False)
    assert st == 0 and info.refine_used == 1 and info.inner_iters >= 1
    check_lse(oracle_mod, P, x, r, v)
    assert Gm.lse_gmres_ir(P["A"], P["B"], P["b"], P["d"])["status"] == 0


@pytest.mark.parametrize("n,m,p,cw", [(200, 120, 100, 1e2), (150, 100, 60, 1e3), (300, 250, 97, 1e3)])
def test_gls_gmres_wide_shapes(h, oracle_mod, n, m, p, cw):
    """n > p: T2 = [I, T^1; 0, T^2] (eq. gls-bdpre-nlarge)."""
    from oracle import gmres as Gm
    G = I.gls_svd(7 * n + m + p, n, m, p, cw, 1e1)
    st, info, x, y, z = run_gls(h, G, refine="gmres", escalate=False)
    assert st == 0 and info.refine_used == 1 and info.inner_iters >= 1
    check_gls(oracle_mod, G, x, y, z)
    assert Gm.gls_gmres_ir(G["W"], G["V"], G["d"])["status"] == 0


def test_gls_gmres_full_size_ar1(h, oracle_mod):
    """The GLS AR(1) workload at full size (n = p = 4096, m = 1024) with
    GMRES-IR: backward error and constraint residual from the oracle's
    double-double residual."""
    G = I.gls_ar1()
    st, info, x, y, z = run_gls(h, G, refine="gmres", escalate=False)
    assert st == 0
    met = oracle_mod.gls_metrics(G["W"], G["V"], G["d"], x, y, z)
    assert met["eta"] <= 1e-14 and met["e_con"] <= 1e-14
