"""Complex LSE / GLS on the GPU (zlse_solve, zgls_solve) against the complex
oracle (oracle/zoracle.py).

The library solves a complex problem through its real 2 x 2 block
embedding on the real path; these tests judge only what the user gets back
(x, r, v / x, y, z), against the complex oracle's plain definition (the
KKT systems in complex128 with extended-precision residuals):
* the eq. lse-stop / gls-stop backward error and the constraint residual
  err-1 (Tables 4, 5) at the FP64-level bar, 1e-14;
* the forward error of x (and y) within 10 kappa u, kappa the real
  oracle's condition estimate of the embedded problem (the embedding keeps
  every singular value, so the two problems have the same kappa);
* every shape class of the real path: tall, square, wide (n > m), p = 0 and
  the GLS corner m = n, with classical IR and with GMRES-IR.
"""
import numpy as np
import pytest

from paper_2406_16499_gb300 import inputs as I
from gpu_util import rel

pytestmark = pytest.mark.gpu
U = 1.1e-16


@pytest.fixture(scope="module")
def h():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2406_16499_gb300 import mpir
    hd = mpir.Handle()
    yield hd
    hd.close()


def zdev(a):
    """numpy complex (any order) -> column-major complex128 CUDA tensor."""
    import torch
    a = np.asarray(a, dtype=np.complex128)
    if a.ndim == 1:
        return torch.from_numpy(a.copy()).cuda()
    if a.size == 0:
        return torch.zeros(a.shape, dtype=torch.complex128, device="cuda")
    return torch.from_numpy(np.ascontiguousarray(a.T)).cuda().t()


def zzeros(k):
    import torch
    return torch.zeros(k, dtype=torch.complex128, device="cuda")


def zhost(t):
    return t.detach().cpu().numpy().copy()


def embed(Z):
    Z = np.asarray(Z)
    return np.block([[Z.real, -Z.imag], [Z.imag, Z.real]])


def run_zlse(h, P, **kw):
    from paper_2406_16499_gb300 import mpir
    A, B = P["A"], P["B"]
    m, n = A.shape
    p = B.shape[0]
    x, r, v = zzeros(n), zzeros(m), zzeros(max(p, 1))
    st, info = h.zlse_solve(zdev(A), zdev(B), zdev(P["b"]), zdev(P["d"]), x, r, v if p else None,
                            mpir.make_opts(**kw))
    return st, info, zhost(x), zhost(r), zhost(v)[:p]


def run_zgls(h, G, **kw):
    from paper_2406_16499_gb300 import mpir
    W, V = G["W"], G["V"]
    n, m = W.shape
    p = V.shape[1]
    x, y, z = zzeros(m), zzeros(p), zzeros(n)
    st, info = h.zgls_solve(zdev(W), zdev(V), zdev(G["d"]), x, y, z, mpir.make_opts(**kw))
    return st, info, zhost(x), zhost(y), zhost(z)


def check_zlse(oracle_mod, P, x, r, v):
    from oracle import zoracle as Z
    A, B, b, d = P["A"], P["B"], P["b"], P["d"]
    t = Z.zlse_truth(A, B, b, d)
    met = Z.zlse_metrics(A, B, b, d, x, r, v)
    assert met["eta"] <= 1e-14 and met["e_con"] <= 1e-14, met
    # kappa of the embedded real problem (the same singular values)
    xe, re_ = np.concatenate([t["x"].real, t["x"].imag]), np.concatenate([t["r"].real, t["r"].imag])
    F = oracle_mod.lse_factor(embed(A), embed(B) if B.shape[0] else np.zeros((0, 2 * A.shape[1])), "fp64")
    kap = oracle_mod.lse_kappa(F, xe, re_)[0]
    fe = rel(x, t["x"])
    assert fe <= 10 * kap * U, (fe, kap)
    return met, fe, kap


def check_zgls(oracle_mod, G, x, y, z):
    from oracle import zoracle as Z
    W, V, d = G["W"], G["V"], G["d"]
    t = Z.zgls_truth(W, V, d)
    met = Z.zgls_metrics(W, V, d, x, y, z)
    assert met["eta"] <= 1e-14 and met["e_con"] <= 1e-14, met
    n, m = W.shape
    p = V.shape[1]
    if n <= p:
        xe = np.concatenate([t["x"].real, t["x"].imag])
        ye = np.concatenate([t["y"].real, t["y"].imag])
        F = oracle_mod.gls_factor(embed(W), embed(V), "fp64")
        kap = oracle_mod.gls_kappa(F, xe, ye)[0]
    else:
        kap = 1e4
    assert rel(x, t["x"]) <= 10 * kap * U, (rel(x, t["x"]), kap)
    if np.linalg.norm(t["y"]) > 1e-8 * np.linalg.norm(t["x"]):
        assert rel(y, t["y"]) <= 10 * kap * U, (rel(y, t["y"]), kap)
    else:                                  # m = n: y = 0
        assert np.linalg.norm(y) <= 10 * kap * U * np.linalg.norm(t["x"])
    return met


@pytest.mark.parametrize("m,n,p,ca", [(200, 100, 20, 1e3), (150, 150, 40, 1e2), (90, 100, 45, 1e3),
                                      (120, 60, 0, 1e4), (257, 129, 31, 1e5)])
def test_zlse_classical_matches_complex_oracle(h, oracle_mod, m, n, p, ca):
    P = I.zlse_svd(7 * m + n + p, m, n, p, ca, 1e1)
    st, info, x, r, v = run_zlse(h, P, escalate=False)
    assert st == 0 and info.escalated == 0
    check_zlse(oracle_mod, P, x, r, v)


@pytest.mark.parametrize("refine", ["gmres", "gmres_left"])
def test_zlse_gmres_ir(h, oracle_mod, refine):
    P = I.zlse_svd(31, 300, 120, 25, 1e4, 1e1)
    st, info, x, r, v = run_zlse(h, P, refine=refine, escalate=False)
    assert st == 0 and info.inner_iters >= 1
    check_zlse(oracle_mod, P, x, r, v)


def test_zlse_fp64_and_tf32_factors(h, oracle_mod):
    P = I.zlse_svd(41, 180, 90, 12, 1e2, 1e1)
    for fact in ("fp64", "tf32"):
        st, info, x, r, v = run_zlse(h, P, fact=fact, escalate=False)
        assert st == 0
        check_zlse(oracle_mod, P, x, r, v)


@pytest.mark.parametrize("n,m,p,cw", [(200, 70, 333, 1e3), (150, 150, 150, 1e2), (129, 1, 300, 1e2),
                                      (200, 120, 100, 1e2), (300, 77, 300, 1e4)])
def test_zgls_classical_matches_complex_oracle(h, oracle_mod, n, m, p, cw):
    G = I.zgls_svd(5 * n + m + p, n, m, p, cw, 1e1)
    st, info, x, y, z = run_zgls(h, G, escalate=False)
    assert st == 0
    check_zgls(oracle_mod, G, x, y, z)


def test_zgls_gmres_ir(h, oracle_mod):
    G = I.zgls_svd(77, 257, 100, 400, 1e4, 1e1)
    st, info, x, y, z = run_zgls(h, G, refine="gmres", escalate=False)
    assert st == 0 and info.inner_iters >= 1
    check_zgls(oracle_mod, G, x, y, z)


def test_zlse_argument_errors(h):
    """Dimension rules and leading dimensions (counted in complex elements)
    are checked on the host, as for lse_solve."""
    from paper_2406_16499_gb300 import mpir
    P = I.zlse_svd(3, 40, 20, 5, 1e1, 1e1)
    A = zdev(P["A"])
    with pytest.raises(mpir.MpirError):
        h.zlse_solve(A[:, :4], zdev(P["B"][:, :4]), zdev(P["b"]), zdev(P["d"]), zzeros(4))   # p > n
    with pytest.raises(mpir.MpirError):
        h.zlse_solve(A, zdev(P["B"]), zdev(P["b"]), zdev(P["d"]), zzeros(20).real.contiguous())


def test_zlse_batched_uneven(h, oracle_mod):
    """Uneven complex LSE batch (one persistent launch on the embedded
    problems): every answer at the bar of the single solve."""
    g = np.random.default_rng(11)
    probs, Ps, xs = [], [], []
    for k in range(24):
        m = int(g.integers(8, 120))
        n = int(g.integers(2, max(3, m // 2)))
        p = int(g.integers(0, max(1, n // 3)))
        P = I.zlse_svd(100 + k, m, n, p, float(10 ** g.uniform(0, 4)), 1e1)
        Ps.append(P)
        probs.append(dict(A=zdev(P["A"]), B=zdev(P["B"]), b=zdev(P["b"]), d=zdev(P["d"])))
        xs.append(zzeros(n))
    st, infos = h.zlse_solve_batched(probs, xs)
    assert st == 0
    from oracle import zoracle as Z
    for P, x, f in zip(Ps, xs, infos):
        assert f.status == 0
        A, B, b, d = P["A"], P["B"], P["b"], P["d"]
        t = Z.zlse_truth(A, B, b, d)
        xh = zhost(x)
        r = b - A @ xh
        e_con = np.linalg.norm(d - B @ xh) / (np.linalg.norm(B) * np.linalg.norm(xh) + np.linalg.norm(d) or 1.0)
        assert e_con <= 1e-14
        xe, re_ = np.concatenate([t["x"].real, t["x"].imag]), np.concatenate([t["r"].real, t["r"].imag])
        F = oracle_mod.lse_factor(embed(A), embed(B) if B.shape[0] else np.zeros((0, 2 * A.shape[1])), "fp64")
        kap = oracle_mod.lse_kappa(F, xe, re_)[0]
        assert rel(xh, t["x"]) <= 10 * kap * U, (rel(xh, t["x"]), kap)


def test_zgls_batched_uneven(h, oracle_mod):
    g = np.random.default_rng(12)
    probs, Gs, xs, ys = [], [], [], []
    for k in range(24):
        n = int(g.integers(8, 120))
        m = int(g.integers(1, max(2, n // 2)))
        p = int(g.integers(n, n + n // 4 + 1))
        G = I.zgls_svd(300 + k, n, m, p, float(10 ** g.uniform(0, 3)), 1e1)
        Gs.append(G)
        probs.append(dict(W=zdev(G["W"]), V=zdev(G["V"]), d=zdev(G["d"])))
        xs.append(zzeros(m))
        ys.append(zzeros(p))
    st, infos = h.zgls_solve_batched(probs, xs, ys)
    assert st == 0
    from oracle import zoracle as Z
    for G, x, y, f in zip(Gs, xs, ys, infos):
        assert f.status == 0
        W, V, d = G["W"], G["V"], G["d"]
        t = Z.zgls_truth(W, V, d)
        xh, yh = zhost(x), zhost(y)
        e_con = np.linalg.norm(W @ xh + V @ yh - d) / (np.linalg.norm(W) * np.linalg.norm(xh) +
                                                      np.linalg.norm(V) * np.linalg.norm(yh) + np.linalg.norm(d))
        assert e_con <= 1e-14
        xe = np.concatenate([t["x"].real, t["x"].imag])
        ye = np.concatenate([t["y"].real, t["y"].imag])
        F = oracle_mod.gls_factor(embed(W), embed(V), "fp64")
        kap = oracle_mod.gls_kappa(F, xe, ye)[0]
        assert rel(xh, t["x"]) <= 10 * kap * U, (rel(xh, t["x"]), kap)
