"""Batched uneven GLS solves (xGGGLM convention, one persistent launch; the
same kernel, queue, buckets, graph and autotuner as the batched LSE solves)
against the oracle.

Every problem must meet the single-problem bar: the constraint residual
||Wx+Vy-d|| / (||W|| ||x|| + ||V|| ||y|| + ||d||) <= 1e-14 (err-1 of
Table 5, double-double residual) and forward error of x and y <= kappa
max(10 u, 2 tol) with kappa the oracle's estimate (reading C13) and tol
= 1e-15 the stop test's bound on the backward error.  The batch API
returns x and y, so the augmented residual's third block is not checked
here; the single-problem tests cover it."""
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


def run_batch(h, probs, **kw):
    from paper_2406_16499_gb300 import mpir
    dp = [dict(W=dev(G["W"]), V=dev(G["V"]), d=dev(G["d"])) for G in probs]
    xs = [zeros(G["W"].shape[1]) for G in probs]
    ys = [zeros(G["V"].shape[1]) for G in probs]
    st, infos = h.gls_solve_batched(dp, xs, ys, mpir.make_opts(**kw))
    return st, infos, [host(x) for x in xs], [host(y) for y in ys]


def check(oracle_mod, G, x, y):
    W, V, d = G["W"], G["V"], G["d"]
    n, m = W.shape
    p = V.shape[1]
    t = oracle_mod.gls_truth(W, V, d)
    f2 = d - W @ x - V @ y
    e_con = np.linalg.norm(f2) / (np.linalg.norm(W) * np.linalg.norm(x) + np.linalg.norm(V) * np.linalg.norm(y)
                                  + np.linalg.norm(d))
    F = oracle_mod.gls_factor(W, V, "fp64")
    kap = oracle_mod.gls_kappa(F, t["x"], t["y"])[0] if n <= p else None
    fx, fy = rel(x, t["x"]), rel(y, t["y"])
    if kap is not None:
        # the stop test bounds the backward error of eq. gls-stop by tol =
        # 1e-15, whose denominators (||d|| + ||W|| ||x|| + ...) reach 2 ||d||
        # (W = V = 1, x = d), so x may carry up to kappa 2 tol of it
        bound = kap * max(10 * 1.1e-16, 2.2e-15)
        assert fx <= bound and fy <= bound, (fx, fy, kap)
    else:
        assert fx <= 1e-10 and fy <= 1e-10, (fx, fy)
    assert e_con <= 1e-14, e_con
    return e_con, fx, kap


def test_batched_gls_uneven(h, oracle_mod):
    """40 problems of the uneven distribution (n ~ U[32, 512], m ~ U[4, n/2],
    p ~ U[n, 5n/4], cond(W) log-uniform in [1e1, 1e5])."""
    probs = I.gls_batch(seed=31, count=40)
    st, infos, xs, ys = run_batch(h, probs)
    assert st == 0
    for G, inf, x, y in zip(probs, infos, xs, ys):
        assert inf.status == 0 and inf.escalated == 0 and inf.fact_used == 2
        check(oracle_mod, G, x, y)


def test_batched_gls_edge_shapes(h, oracle_mod):
    """Square W (n = m: y = 0), p < n <= m + p, n = p, tiny problems, the
    AR(1) covariance factor, and problems whose factors go to global
    scratch."""
    shapes = [(40, 40, 10), (60, 30, 40), (64, 16, 64), (5, 2, 4), (1, 1, 1), (97, 33, 97), (480, 200, 500),
              (512, 128, 640), (300, 150, 160)]
    probs = [I.gls_svd(200 + k, n, m, p, 1e3, 1e1) for k, (n, m, p) in enumerate(shapes)]
    probs.append(I.gls_ar1(seed=9, n=256, m=64))
    st, infos, xs, ys = run_batch(h, probs)
    assert st == 0
    for G, inf, x, y in zip(probs, infos, xs, ys):
        assert inf.status == 0
        check(oracle_mod, G, x, y)
    # n = m: W x = d - V y has y = 0 as the minimum-norm choice
    assert np.abs(ys[0]).max() <= 1e-12 * max(1.0, np.abs(xs[0]).max())


def test_batched_gls_matches_single(h, oracle_mod):
    from paper_2406_16499_gb300 import mpir
    probs = I.gls_batch(seed=32, count=10)
    st, infos, xs, ys = run_batch(h, probs)
    assert st == 0
    for G, x, y in zip(probs, xs, ys):
        n, m = G["W"].shape
        p = G["V"].shape[1]
        xd, yd = zeros(m), zeros(p)
        s1, _ = h.gls_solve(dev(G["W"]), dev(G["V"]), dev(G["d"]), xd, yd, None, mpir.make_opts())
        assert s1 == 0
        t = oracle_mod.gls_truth(G["W"], G["V"], G["d"])
        assert rel(x, host(xd)) <= 2 * (rel(x, t["x"]) + rel(host(xd), t["x"])) + 1e-15


def test_batched_gls_fp64_direct(h, oracle_mod):
    probs = I.gls_batch(seed=33, count=12)
    st, infos, xs, ys = run_batch(h, probs, fact="fp64", refine="direct")
    assert st == 0
    for G, inf, x in zip(probs, infos, xs):
        assert inf.fact_used == 3 and inf.iters == 0
        t = oracle_mod.gls_truth(G["W"], G["V"], G["d"])
        F = oracle_mod.gls_factor(G["W"], G["V"], "fp64")
        kap = oracle_mod.gls_kappa(F, t["x"], t["y"])[0]
        assert rel(x, t["x"]) <= 100 * kap * 1.1e-16


def test_batched_gls_escalation(h, oracle_mod):
    """A problem with cond(W) = 1e10 in the batch is re-solved with FP64
    factors; without escalation it reports non-convergence."""
    probs = I.gls_batch(seed=34, count=6)
    probs.insert(2, I.gls_svd(77, 200, 60, 220, 1e10, 1e1))
    st, infos, xs, ys = run_batch(h, probs)
    assert st == 0
    assert infos[2].escalated == 1 and infos[2].fact_used == 3
    assert all(infos[k].escalated == 0 for k in range(len(probs)) if k != 2)
    check(oracle_mod, probs[2], xs[2], ys[2])
    st, infos, xs, ys = run_batch(h, probs, escalate=False)
    assert st == 3 and infos[2].status == 3


@pytest.mark.parametrize("group", [512, 256, 128])
def test_batched_gls_launch_shapes(h, oracle_mod, group):
    probs = I.gls_batch(seed=35, count=16, n_hi=160)
    h.batched_set_shape(group)
    try:
        st, infos, xs, ys = run_batch(h, probs)
    finally:
        h.batched_set_shape(0)
    assert st == 0
    for G, x, y in zip(probs, xs, ys):
        check(oracle_mod, G, x, y)
