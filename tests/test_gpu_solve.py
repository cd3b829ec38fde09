"""End-to-end GPU solves (lse_solve / gls_solve through the C ABI) against the
CPU oracle's solution.  The bar: normwise augmented backward error (eq.
lse-stop / gls-stop ratios, double-double residual) <= 1e-14, constraint
residual ||Bx-d|| / (||B|| ||x|| + ||d||) <= 1e-14, and forward error
<= 10 kappa 1.1e-16 with kappa the oracle's condition estimate."""
import numpy as np
import pytest

from paper_2406_16499_gb300 import inputs as I
from gpu_util import dev, host, rel, zeros

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def h():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2406_16499_gb300 import mpir
    hd = mpir.Handle()
    yield hd
    hd.close()


def run_lse(h, P, fact="fp32", refine="classical", **kw):
    from paper_2406_16499_gb300 import mpir
    A, B, b, d = P["A"], P["B"], P["b"], P["d"]
    m, n = A.shape
    p = B.shape[0]
    x, r, v = zeros(n), zeros(m), zeros(p)
    st, info = h.lse_solve(dev(A), dev(B), dev(b), dev(d), x, r, v if p else None,
                           mpir.make_opts(fact=fact, refine=refine, **kw))
    return st, info, host(x), host(r), host(v)[:p]


def run_gls(h, G, fact="fp32", refine="classical", **kw):
    from paper_2406_16499_gb300 import mpir
    W, V, d = G["W"], G["V"], G["d"]
    n, m = W.shape
    p = V.shape[1]
    x, y, z = zeros(m), zeros(p), zeros(n)
    st, info = h.gls_solve(dev(W), dev(V), dev(d), x, y, z, mpir.make_opts(fact=fact, refine=refine, **kw))
    return st, info, host(x), host(y), host(z)


def check_lse(oracle_mod, P, x, r, v, tight=True):
    A, B, b, d = P["A"], P["B"], P["b"], P["d"]
    t = oracle_mod.lse_truth(A, B, b, d)
    met = oracle_mod.lse_metrics(A, B, b, d, x, r, v)
    F = oracle_mod.lse_factor(A, B, "fp64")
    kap = oracle_mod.lse_kappa(F, t["x"], t["r"])[0]
    fe = rel(x, t["x"])
    assert met["eta"] <= 1e-14, met
    assert met["e_con"] <= 1e-14, met
    assert fe <= 10 * kap * 1.1e-16, (fe, kap)
    return met, fe, kap


def check_gls(oracle_mod, G, x, y, z):
    W, V, d = G["W"], G["V"], G["d"]
    t = oracle_mod.gls_truth(W, V, d)
    met = oracle_mod.gls_metrics(W, V, d, x, y, z)
    n, m = W.shape
    p = V.shape[1]
    if n <= p:
        F = oracle_mod.gls_factor(W, V, "fp64")
        kap = oracle_mod.gls_kappa(F, t["x"], t["y"])[0]
    else:
        kap = 1e4
    fe = rel(x, t["x"])
    assert met["eta"] <= 1e-14, met
    assert met["e_con"] <= 1e-14, met
    assert fe <= 10 * kap * 1.1e-16, (fe, kap)
    assert rel(y, t["y"]) <= 10 * kap * 1.1e-16
    return met, fe, kap


def test_lse_small_config_fp32_classical(h, oracle_mod):
    """LSE m=200, n=100, p=20 (logspace spectra), FP32 GRQ + FP64
    classical IR."""
    P = I.lse_small()
    st, info, x, r, v = run_lse(h, P)
    assert st == 0 and info.status == 0 and info.escalated == 0
    assert 1 <= info.iters <= 6
    check_lse(oracle_mod, P, x, r, v)


@pytest.mark.parametrize("m,n,p,ca", [(333, 290, 77, 1e3), (1000, 513, 1, 1e4), (64, 64, 64, 1e2),
                                      (90, 100, 45, 1e3), (257, 129, 31, 1e5)])
def test_lse_ragged_shapes(h, oracle_mod, m, n, p, ca):
    P = I.lse_svd(m + 7 * n + p, m, n, p, ca, 1e1)
    st, info, x, r, v = run_lse(h, P)
    assert st == 0
    check_lse(oracle_mod, P, x, r, v)


def test_lse_no_constraint_is_least_squares(h, oracle_mod):
    """p = 0: ordinary least squares."""
    P = I.lse_svd(5, 300, 120, 0, 1e3, 1.0)
    st, info, x, r, v = run_lse(h, P)
    assert st == 0
    x_ls = np.linalg.lstsq(P["A"], P["b"], rcond=None)[0]
    assert rel(x, x_ls) < 1e-11


@pytest.mark.parametrize("n,m,p,cw", [(300, 77, 300, 1e3), (257, 100, 400, 1e4), (200, 120, 100, 1e2),
                                      (129, 129, 40, 1e2)])
def test_gls_shapes_fp32_classical(h, oracle_mod, n, m, p, cw):
    G = I.gls_svd(3 * n + m + p, n, m, p, cw, 1e1)
    st, info, x, y, z = run_gls(h, G)
    assert st == 0 and info.escalated == 0
    check_gls(oracle_mod, G, x, y, z)


def test_gls_ar1_reduced(h, oracle_mod):
    """The AR(1) covariance workload at a reduced size (n = p = 1024,
    m = 256): FP32 GQR + FP64 classical IR."""
    G = I.gls_ar1(seed=77, n=1024, m=256)
    st, info, x, y, z = run_gls(h, G)
    assert st == 0 and info.escalated == 0 and info.iters <= 8
    check_gls(oracle_mod, G, x, y, z)


def test_gls_ar1_full_size_classical(h, oracle_mod):
    """The benchmarked workload itself (n = p = 4096, m = 1024, the same
    seed and the same FP32 GQR + FP64 classical IR launch path): eq.
    gls-stop ratios and the constraint residual from the oracle's
    double-double residual, and the forward error of x and y against the
    oracle's solution, FP32 factors without escalation."""
    G = I.gls_ar1()
    st, info, x, y, z = run_gls(h, G, escalate=False)
    assert st == 0 and info.escalated == 0 and info.fact_used == 2
    # the oracle's FP64 GQR and double-double refinement at full size give
    # the solution and the forward-error condition number (reading C13)
    met, fe, kap = check_gls(oracle_mod, G, x, y, z)
    print("GLS n=4096: eta %.2e e_con %.2e fwd %.2e kappa %.3e fwd/(10 kappa u) %.3f"
          % (met["eta"], met["e_con"], fe, kap, fe / (10 * kap * 1.1e-16)))


def test_fp64_direct_matches_oracle(h, oracle_mod):
    """The fixed-precision FP64 path (GQR + Paige, no refinement) is the
    comparator the mixed-precision solve is timed against."""
    G = I.gls_svd(17, 300, 77, 300, 1e3, 1e1)
    st, info, x, y, z = run_gls(h, G, fact="fp64", refine="direct")
    assert st == 0
    t = oracle_mod.gls_truth(G["W"], G["V"], G["d"])
    assert rel(x, t["x"]) < 1e-10
    P = I.lse_small()
    st, info, x, r, v = run_lse(h, P, fact="fp64", refine="direct")
    assert st == 0
    t = oracle_mod.lse_truth(P["A"], P["B"], P["b"], P["d"])
    assert rel(x, t["x"]) < 1e-12


def test_escalation_on_ill_conditioned(h, oracle_mod):
    """kappa ~ 1e9 exceeds what FP32 classical IR can refine (Table 2,
    Table 4): the solver reports non-convergence at FP32 and escalates to an
    FP64 factorization, which converges."""
    P = I.lse_paper(404, 512, 64, 2, 1e9)
    st, info, x, r, v = run_lse(h, P)
    assert st == 0
    assert info.escalated >= 1 and info.fact_used == 3
    met = oracle_mod.lse_metrics(P["A"], P["B"], P["b"], P["d"], x, r, v)
    assert met["eta"] <= 1e-14
    st, info, x, r, v = run_lse(h, P, escalate=False)
    assert st == 3


def test_power_of_two_scaling(h, oracle_mod):
    """Data far outside the FP32 range still factors in FP32: A, B are
    scaled by powers of two before down-conversion (Sec. 6.1)."""
    P = I.lse_svd(9, 150, 80, 10, 1e2, 1e1)
    P = dict(A=P["A"] * 2.0 ** 200, B=P["B"] * 2.0 ** -180, b=P["b"] * 2.0 ** 200, d=P["d"] * 2.0 ** -180)
    st, info, x, r, v = run_lse(h, P, escalate=False)
    assert st == 0
    met = oracle_mod.lse_metrics(P["A"], P["B"], P["b"], P["d"], x, r, v)
    assert met["eta"] <= 1e-14


@pytest.mark.parametrize("kind", ["lse", "gls"])
def test_double_double_residual_reaches_u(h, oracle_mod, kind):
    """The u_r < u variant (resid_dd, Table 2's third row): residuals in
    double-double and refinement until the corrections stop shrinking give a
    forward error of a few u even at cond = 1e6, where the FP64 residual
    leaves it near kappa u (checked against the oracle's solution, itself
    refined with double-double residuals)."""
    U = 1.1102230246251565e-16
    if kind == "lse":
        P = I.lse_svd(4711, 300, 150, 20, 1e6, 1e1)
        t = oracle_mod.lse_truth(P["A"], P["B"], P["b"], P["d"])
        st, info, x, r, v = run_lse(h, P, fact="fp64", resid_dd=1, escalate=False)
        st0, _, x0, _, _ = run_lse(h, P, fact="fp64", escalate=False)
        met = oracle_mod.lse_metrics(P["A"], P["B"], P["b"], P["d"], x, r, v)
    else:
        G = I.gls_svd(4712, 300, 80, 320, 1e6, 1e1)
        t = oracle_mod.gls_truth(G["W"], G["V"], G["d"])
        st, info, x, y, z = run_gls(h, G, fact="fp64", resid_dd=1, escalate=False)
        st0, _, x0, _, _ = run_gls(h, G, fact="fp64", escalate=False)
        met = oracle_mod.gls_metrics(G["W"], G["V"], G["d"], x, y, z)
    assert st == 0 and st0 == 0
    assert met["eta"] <= 1e-14 and met["e_con"] <= 1e-14, met
    fe, fe0 = rel(x, t["x"]), rel(x0, t["x"])
    print("%s: forward error %.2e with double-double residuals, %.2e with FP64 residuals" % (kind, fe, fe0))
    assert fe <= 20 * U, (fe, fe0)
