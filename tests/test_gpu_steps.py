"""GPU parity of each stage of the method against the CPU oracle, through the
C ABI: FP64 residuals (Alg. 2 step 6 / Alg. 4 step 5), the GRQ / GQR
factorizations (Lemma 4.5 / 4.6 invariants), the initial solutions and
multipliers (Sec. 2, Sec. 3), and the correction solves (Alg. 1 / Alg. 3,
Theorems 4.3 / 4.7).  Sizes span several 32-wide panels and ragged tails."""
import numpy as np
import pytest

from paper_2406_16499_gb300 import inputs as I
from gpu_util import U64, dev, host, rel, zeros

pytestmark = pytest.mark.gpu

U32 = np.finfo(np.float32).eps / 2


@pytest.fixture(scope="module")
def h():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2406_16499_gb300 import mpir
    hd = mpir.Handle()
    yield hd
    hd.close()


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


# ------------------------------------------------------------- residuals --

@pytest.mark.parametrize("m,n,p", [(200, 100, 20), (333, 290, 77), (1000, 513, 1), (64, 64, 64)])
def test_lse_residual_matches_double_double(h, oracle_mod, m, n, p):
    """Every entry of the GPU FP64 residual is within the FP64 gemv bound
    gamma_{n+2} (|b| + |r| + |A||x| ...) of the double-double residual."""
    P = I.lse_svd(m + n + p, m, n, p, 1e3, 1e1)
    A, B, b, d = P["A"], P["B"], P["b"], P["d"]
    g = I.rng(7)
    x, r, v = g.standard_normal(n), g.standard_normal(m), g.standard_normal(p)
    f1, f2, f3 = zeros(m), zeros(p), zeros(n)
    norms = h.lse_residual(dev(A), dev(B), dev(b), dev(d), dev(x), dev(r), dev(v), f1, f2, f3)
    e1, e2, e3 = oracle_mod.lse_residual(A, B, b, d, x, r, v, dd=True)
    got = np.concatenate([host(f1), host(f2)[:p], host(f3)])
    ref = np.concatenate([e1, e2, e3])
    F = lse_aug(A, B)
    u = np.concatenate([r, -v, x])
    rhs = np.concatenate([b, d, np.zeros(n)])
    bound = (m + n + p + 2) * U64 * (np.abs(rhs) + np.abs(F) @ np.abs(u))
    assert np.all(np.abs(got - ref) <= bound)
    assert abs(norms[0] / np.linalg.norm(e1) - 1) < 1e-10
    assert abs(norms[3] / np.linalg.norm(x) - 1) < 1e-14
    assert abs(norms[6] / np.linalg.norm(A) - 1) < 1e-14
    assert abs(norms[7] / max(np.linalg.norm(B), 1e-300) - 1) < 1e-14


@pytest.mark.parametrize("n,m,p", [(300, 77, 300), (257, 100, 400), (200, 120, 100)])
def test_gls_residual_matches_double_double(h, oracle_mod, n, m, p):
    G = I.gls_svd(n + 2 * m + p, n, m, p, 1e3, 1e1)
    W, V, d = G["W"], G["V"], G["d"]
    g = I.rng(8)
    x, y, z = g.standard_normal(m), g.standard_normal(p), g.standard_normal(n)
    f1, f2, f3 = zeros(p), zeros(n), zeros(m)
    h.gls_residual(dev(W), dev(V), dev(d), dev(x), dev(y), dev(z), f1, f2, f3)
    e1, e2, e3 = oracle_mod.gls_residual(W, V, d, x, y, z, dd=True)
    got = np.concatenate([host(f1), host(f2), host(f3)])
    ref = np.concatenate([e1, e2, e3])
    F = gls_aug(W, V)
    u = np.concatenate([y, -z, x])
    rhs = np.concatenate([np.zeros(p), d, np.zeros(m)])
    bound = (m + n + p + 2) * U64 * (np.abs(rhs) + np.abs(F) @ np.abs(u))
    assert np.all(np.abs(got - ref) <= bound)


# --------------------------------------------------------- factorizations --

def _explicit(h, which, k):
    import torch
    cols = []
    for j in range(k):
        e = torch.zeros(k, dtype=torch.float64, device="cuda")
        e[j] = 1.0
        h.apply_factor(which, False, e)
        cols.append(host(e))
    return np.column_stack(cols)


@pytest.mark.parametrize("fact,tol", [("fp32", 3e-6), ("fp64", 1e-14)])
@pytest.mark.parametrize("m,n,p", [(150, 90, 20), (70, 100, 45), (96, 96, 33)])
def test_grq_invariants(h, fact, tol, m, n, p):
    """Lemma 4.5 on the GPU factors: B ~ [0 R] Q, A ~ Z T Q with backward
    errors O(u_f) ||.||_F; Q, Z orthogonal; R, T triangular."""
    import torch
    P = I.lse_svd(3 * m + n + p, m, n, p, 1e2, 1e1)
    A, B = P["A"], P["B"]
    h.lse_factor(dev(A), dev(B), fact)
    R = torch.zeros((p, p), dtype=torch.float64, device="cuda").t().contiguous().t()
    T = torch.zeros((n, m), dtype=torch.float64, device="cuda").t()
    h.get_RT(R, T)
    R, T = host(R), host(T)
    Q = _explicit(h, "Q", n)
    Z = _explicit(h, "Z", m)
    RB = np.zeros((p, n))
    RB[:, n - p:] = R
    assert np.allclose(R, np.triu(R)) and np.allclose(T, np.triu(T))
    assert np.linalg.norm(B - RB @ Q) <= tol * 30 * np.linalg.norm(B)
    assert np.linalg.norm(A - Z @ T @ Q) <= tol * 30 * np.linalg.norm(A)
    assert np.linalg.norm(Q.T @ Q - np.eye(n)) <= tol * 30 * n
    assert np.linalg.norm(Z.T @ Z - np.eye(m)) <= tol * 30 * m


@pytest.mark.parametrize("fact,tol", [("fp32", 3e-6), ("fp64", 1e-14)])
@pytest.mark.parametrize("n,m,p", [(150, 40, 200), (130, 70, 130), (140, 90, 60)])
def test_gqr_invariants(h, fact, tol, n, m, p):
    """Lemma 4.6 on the GPU factors: W ~ Q [R; 0], V ~ Q T Z, T upper
    trapezoidal in the RQ sense with T22 upper triangular."""
    import torch
    G = I.gls_svd(n + 3 * m + p, n, m, p, 1e2, 1e1)
    W, V = G["W"], G["V"]
    h.gls_factor(dev(W), dev(V), fact)
    R = torch.zeros((m, m), dtype=torch.float64, device="cuda").t()
    T = torch.zeros((p, n), dtype=torch.float64, device="cuda").t()
    h.get_RT(R, T)
    R, T = host(R), host(T)
    Q = _explicit(h, "Q", n)
    Z = _explicit(h, "Z", p)
    RW = np.zeros((n, m))
    RW[:m] = R
    o = p - n + m
    assert np.allclose(T[m:, :o], 0.0)
    assert np.allclose(T[m:, o:], np.triu(T[m:, o:]))
    assert np.linalg.norm(W - Q @ RW) <= tol * 30 * np.linalg.norm(W)
    assert np.linalg.norm(V - Q @ T @ Z) <= tol * 30 * np.linalg.norm(V)
    assert np.linalg.norm(Q.T @ Q - np.eye(n)) <= tol * 30 * n
    assert np.linalg.norm(Z.T @ Z - np.eye(p)) <= tol * 30 * p


def _explicit_t(h, which, k):
    """Columns of Q^T (or Z^T) through the transposed application."""
    import torch
    cols = []
    for j in range(k):
        e = torch.zeros(k, dtype=torch.float64, device="cuda")
        e[j] = 1.0
        h.apply_factor(which, True, e)
        cols.append(host(e))
    return np.column_stack(cols)


def test_grq_gqr_many_blocks(h):
    """Reflector sets of several 128-wide outer blocks (the FP32 path applies
    them through the aggregated compact-WY factor): Lemma 4.5 / 4.6 still
    hold, and the transposed application is the transpose of the forward one."""
    tol = 3e-6
    m, n, p = 700, 600, 300
    P = I.lse_svd(3 * m + n + p, m, n, p, 1e2, 1e1)
    A, B = P["A"], P["B"]
    h.lse_factor(dev(A), dev(B), "fp32")
    import torch
    R = torch.zeros((p, p), dtype=torch.float64, device="cuda").t().contiguous().t()
    T = torch.zeros((n, m), dtype=torch.float64, device="cuda").t()
    h.get_RT(R, T)
    R, T = host(R), host(T)
    Q, Z = _explicit(h, "Q", n), _explicit(h, "Z", m)
    RB = np.zeros((p, n))
    RB[:, n - p:] = R
    assert np.linalg.norm(B - RB @ Q) <= tol * 30 * np.linalg.norm(B)
    assert np.linalg.norm(A - Z @ T @ Q) <= tol * 30 * np.linalg.norm(A)
    assert np.linalg.norm(Q.T @ Q - np.eye(n)) <= tol * 30 * n
    assert np.linalg.norm(Z.T @ Z - np.eye(m)) <= tol * 30 * m
    assert np.abs(_explicit_t(h, "Q", n) - Q.T).max() <= 1e-5
    assert np.abs(_explicit_t(h, "Z", m) - Z.T).max() <= 1e-5
    n, m, p = 900, 400, 800
    G = I.gls_svd(n + 3 * m + p, n, m, p, 1e2, 1e1)
    W, V = G["W"], G["V"]
    h.gls_factor(dev(W), dev(V), "fp32")
    R = torch.zeros((m, m), dtype=torch.float64, device="cuda").t()
    T = torch.zeros((p, n), dtype=torch.float64, device="cuda").t()
    h.get_RT(R, T)
    R, T = host(R), host(T)
    Q, Z = _explicit(h, "Q", n), _explicit(h, "Z", p)
    RW = np.zeros((n, m))
    RW[:m] = R
    assert np.linalg.norm(W - Q @ RW) <= tol * 30 * np.linalg.norm(W)
    assert np.linalg.norm(V - Q @ T @ Z) <= tol * 30 * np.linalg.norm(V)
    assert np.linalg.norm(Q.T @ Q - np.eye(n)) <= tol * 30 * n
    assert np.linalg.norm(Z.T @ Z - np.eye(p)) <= tol * 30 * p
    assert np.abs(_explicit_t(h, "Q", n) - Q.T).max() <= 1e-5
    assert np.abs(_explicit_t(h, "Z", p) - Z.T).max() <= 1e-5


@pytest.mark.parametrize("m,n,p,fact", [(12288, 384, 64, "fp32"), (40960, 160, 32, "fp32"),
                                        (20480, 96, 16, "fp64")])
def test_grq_invariants_tall(h, m, n, p, fact):
    """Panels taller than one cluster's shared memory (m = 12288 rows, the
    row-chunked inner updates) and taller than a 16-CTA cluster holds in
    registers (m = 40960 FP32 / 20480 FP64 rows: the grid-exchange panel on
    one CTA per 1024 rows): Lemma 4.5 through products with random vectors,
    B x ~ [0 R] Q x and A x ~ Z T Q x with backward errors
    O(u_f) ||.||_F ||x||, and Q^T Q x = x, Z^T Z y = y."""
    import torch
    tol = 3e-6 if fact == "fp32" else 1e-14
    T = I.lse_svd_torch(31, m, n, p, 1e2, 1e1, "cuda")
    A, B = T["A"], T["B"]
    h.lse_factor(A, B, fact)
    R = torch.zeros((p, p), dtype=torch.float64, device="cuda").t().contiguous().t()
    Tm = torch.zeros((n, m), dtype=torch.float64, device="cuda").t()
    h.get_RT(R, Tm)
    assert torch.allclose(Tm, torch.triu(Tm)) and torch.allclose(R, torch.triu(R))
    nA, nB = float(torch.linalg.norm(A)), float(torch.linalg.norm(B))
    g = torch.Generator(device="cuda")
    g.manual_seed(3)
    for _ in range(4):
        x = torch.randn(n, dtype=torch.float64, device="cuda", generator=g)
        nx = float(torch.linalg.norm(x))
        qx = x.clone()
        h.apply_factor("Q", False, qx)
        assert float(torch.linalg.norm(B @ x - R @ qx[n - p:])) <= tol * 30 * nB * nx
        ztqx = Tm @ qx
        h.apply_factor("Z", False, ztqx)
        assert float(torch.linalg.norm(A @ x - ztqx)) <= tol * 30 * nA * nx
        back = qx.clone()
        h.apply_factor("Q", True, back)
        assert float(torch.linalg.norm(back - x)) <= tol * 30 * np.sqrt(n) * nx
        y = torch.randn(m, dtype=torch.float64, device="cuda", generator=g)
        zy = y.clone()
        h.apply_factor("Z", False, zy)
        h.apply_factor("Z", True, zy)
        assert float(torch.linalg.norm(zy - y)) <= tol * 30 * np.sqrt(m) * float(torch.linalg.norm(y))


# ------------------------------------------------- initial solutions --

@pytest.mark.parametrize("fact", ["fp32", "fp64"])
def test_lse_initial_and_multipliers(h, oracle_mod, fact):
    """Null-space start (Sec. 2.1) and v0 (Sec. 3.1) at u_f agree with the
    oracle's solution to O(kappa u_f)."""
    P = I.lse_small()
    A, B, b, d = P["A"], P["B"], P["b"], P["d"]
    m, n, p = 200, 100, 20
    t = oracle_mod.lse_truth(A, B, b, d)
    dA = dev(A)
    h.lse_factor(dA, dev(B), fact)
    x, r, v = zeros(n), zeros(m), zeros(p)
    db = dev(b)
    h.lse_initial(db, dev(d), x)
    h.lse_multipliers(dA, db, x, r, v)
    u = U32 if fact == "fp32" else U64
    F = oracle_mod.lse_factor(A, B, "fp64")
    kap = oracle_mod.lse_kappa(F, t["x"], t["r"])[0]
    assert rel(host(x), t["x"]) < 30 * kap * u
    assert rel(host(r), t["r"]) < 30 * kap * u * 1e3
    assert rel(host(v), t["v"]) < 30 * kap * u * 1e3


@pytest.mark.parametrize("fact", ["fp32", "fp64"])
def test_gls_initial_and_multipliers(h, oracle_mod, fact):
    """Paige's method (Sec. 2.2) and z0 = Q [0; h] (Sec. 3.2) at u_f."""
    G = I.gls_svd(31, 300, 77, 300, 1e2, 1e1)
    W, V, d = G["W"], G["V"], G["d"]
    n, m, p = 300, 77, 300
    t = oracle_mod.gls_truth(W, V, d)
    h.gls_factor(dev(W), dev(V), fact)
    x, y, z = zeros(m), zeros(p), zeros(n)
    h.gls_initial(dev(d), x, y)
    h.gls_multipliers(y, z)
    u = U32 if fact == "fp32" else U64
    tol = 3e4 * u
    assert rel(host(x), t["x"]) < tol
    assert rel(host(y), t["y"]) < tol
    assert rel(host(z), t["z"]) < tol


# -------------------------------------------------------- correction --

@pytest.mark.parametrize("fact,eta_max", [("fp32", 1e-5), ("fp64", 1e-13)])
@pytest.mark.parametrize("m,n,p", [(200, 100, 20), (130, 97, 50), (64, 80, 16), (900, 700, 200),
                                   pytest.param(2600, 2300, 200, id="segmented-2100")])
def test_lse_correction_backward_error(h, fact, eta_max, m, n, p):
    """Theorem 4.3: the GPU correction solve (Alg. 1 on the held factors)
    satisfies eq. correction-system-lse with a normwise backward error of
    O(u_f)."""
    P = I.lse_svd(m * 3 + n + 2 * p, m, n, p, 1e2, 1e1)
    A, B = P["A"], P["B"]
    h.lse_factor(dev(A), dev(B), fact)
    g = I.rng(m + n)
    f1, f2, f3 = g.standard_normal(m), g.standard_normal(p), g.standard_normal(n)
    dr, dv, dx = zeros(m), zeros(p), zeros(n)
    h.lse_correction(dev(f1), dev(f2), dev(f3), dr, dv, dx)
    sol = np.concatenate([host(dr), -host(dv)[:p], host(dx)])
    Fa = lse_aug(A, B)
    f = np.concatenate([f1, f2, f3])
    eta = np.linalg.norm(Fa @ sol - f) / (np.linalg.norm(Fa) * np.linalg.norm(sol) + np.linalg.norm(f))
    assert eta < eta_max


@pytest.mark.parametrize("fact,eta_max", [("fp32", 1e-5), ("fp64", 1e-13)])
@pytest.mark.parametrize("n,m,p", [(150, 40, 200), (130, 70, 130), (140, 90, 60), (900, 400, 800),
                                   pytest.param(2600, 1100, 2400, id="segmented-1500")])
def test_gls_correction_backward_error(h, fact, eta_max, n, m, p):
    """Theorem 4.7: the GPU correction solve (Alg. 3 read with T22 g2 = u2
    and dz = -Q h) satisfies eq. correction-system-gls to O(u_f)."""
    G = I.gls_svd(2 * n + m + 5 * p, n, m, p, 1e2, 1e1)
    W, V = G["W"], G["V"]
    h.gls_factor(dev(W), dev(V), fact)
    g = I.rng(n + p)
    f1, f2, f3 = g.standard_normal(p), g.standard_normal(n), g.standard_normal(m)
    dy, dz, dx = zeros(p), zeros(n), zeros(m)
    h.gls_correction(dev(f1), dev(f2), dev(f3), dy, dz, dx)
    sol = np.concatenate([host(dy), -host(dz), host(dx)])
    Fa = gls_aug(W, V)
    f = np.concatenate([f1, f2, f3])
    eta = np.linalg.norm(Fa @ sol - f) / (np.linalg.norm(Fa) * np.linalg.norm(sol) + np.linalg.norm(f))
    assert eta < eta_max
