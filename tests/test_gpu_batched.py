"""Batched uneven LSE solves (one persistent launch) against the oracle.

Every problem of the batch must meet the single-problem bar: eq. lse-stop
ratios <= 1e-14 (double-double residual), ||Bx-d|| / (||B|| ||x|| + ||d||)
<= 1e-14 and forward error <= 10 kappa 1.1e-16 (kappa from the oracle).
The batches mix shapes whose factors stay in shared memory with shapes whose
factors go to the per-CTA global scratch, and the degenerate shapes of the
problem statement (p = 0, p = n, m < n)."""
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


def to_dev(P):
    return dict(A=dev(P["A"]), B=dev(P["B"]), b=dev(P["b"]), d=dev(P["d"]))


def run_batch(h, probs, **kw):
    from paper_2406_16499_gb300 import mpir
    dp = [to_dev(P) for P in probs]
    xs = [zeros(P["A"].shape[1]) for P in probs]
    st, infos = h.lse_solve_batched(dp, xs, mpir.make_opts(**kw))
    return st, infos, [host(x) for x in xs]


def check(oracle_mod, P, x, fe_only=False):
    A, B, b, d = P["A"], P["B"], P["b"], P["d"]
    t = oracle_mod.lse_truth(A, B, b, d)
    r = b - A @ x
    # v from the oracle's multiplier formula at x (the batched API returns x)
    F = oracle_mod.lse_factor(A, B, "fp64")
    v = oracle_mod.lse_init_v(F, A, r) if B.shape[0] else np.zeros(0)
    met = oracle_mod.lse_metrics(A, B, b, d, x, r, v)
    kap = oracle_mod.lse_kappa(F, t["x"], t["r"])[0]
    fe = rel(x, t["x"])
    assert fe <= 10 * kap * 1.1e-16, (fe, kap)
    if not fe_only:
        assert met["e_con"] <= 1e-14, met
    return met, fe, kap


def test_batched_uneven_small(h, oracle_mod):
    """48 problems of the uneven distribution (m ~ U[32, 512], n ~ U[16, m/2],
    p ~ U[1, n/4], cond(A) log-uniform in [1e1, 1e6])."""
    probs = I.lse_batch(seed=11, count=48)
    st, infos, xs = run_batch(h, probs)
    assert st == 0
    for P, inf, x in zip(probs, infos, xs):
        assert inf.status == 0 and inf.escalated == 0 and inf.fact_used == 2
        check(oracle_mod, P, x)


def test_batched_edge_shapes(h, oracle_mod):
    """p = 0 (least squares), p = n (x fixed by B), m < n <= m + p, tiny
    problems, and large ones whose factors live in global scratch."""
    shapes = [(40, 20, 0), (64, 32, 32), (30, 40, 15), (5, 3, 1), (1, 1, 1), (33, 17, 16),
              (512, 256, 64), (480, 240, 7), (300, 150, 1), (257, 129, 31)]
    probs = [I.lse_svd(100 + k, m, n, p, 1e3, 1e1) for k, (m, n, p) in enumerate(shapes)]
    st, infos, xs = run_batch(h, probs)
    assert st == 0
    for P, inf, x in zip(probs, infos, xs):
        assert inf.status == 0
        check(oracle_mod, P, x)
    # p = 0 is ordinary least squares
    x_ls = np.linalg.lstsq(probs[0]["A"], probs[0]["b"], rcond=None)[0]
    assert rel(xs[0], x_ls) < 1e-11


def test_batched_matches_single(h, oracle_mod):
    """The batched kernel and the single-problem path reach the same
    solution (both to the FP64-level bar)."""
    from paper_2406_16499_gb300 import mpir
    probs = I.lse_batch(seed=12, count=12)
    st, infos, xs = run_batch(h, probs)
    assert st == 0
    for P, x in zip(probs, xs):
        m, n = P["A"].shape
        p = P["B"].shape[0]
        xd = zeros(n)
        s1, _ = h.lse_solve(dev(P["A"]), dev(P["B"]), dev(P["b"]), dev(P["d"]), xd, None, None, mpir.make_opts())
        assert s1 == 0
        t = oracle_mod.lse_truth(P["A"], P["B"], P["b"], P["d"])
        assert rel(x, host(xd)) <= 2 * (rel(x, t["x"]) + rel(host(xd), t["x"])) + 1e-15


def test_batched_graph_replay(h, oracle_mod):
    """A second call with the same shapes replays the captured graph on new
    data (b and d replaced) and still solves every problem."""
    probs = I.lse_batch(seed=13, count=20)
    st, infos, xs = run_batch(h, probs)
    assert st == 0
    g = np.random.default_rng(7)
    probs2 = []
    for P in probs:
        m, n = P["A"].shape
        x_true = g.standard_normal(n)
        probs2.append(dict(A=P["A"], B=P["B"], b=P["A"] @ x_true + g.standard_normal(m), d=P["B"] @ x_true))
    st, infos, xs = run_batch(h, probs2)
    assert st == 0
    for P, x in zip(probs2, xs):
        check(oracle_mod, P, x)


def test_batched_fp64_direct(h, oracle_mod):
    """fact = FP64, refine = direct: the fixed-precision comparator of the
    batched workload (FP64 GRQ + null-space method in the same kernel)."""
    probs = I.lse_batch(seed=14, count=24)
    st, infos, xs = run_batch(h, probs, fact="fp64", refine="direct")
    assert st == 0
    for P, inf, x in zip(probs, infos, xs):
        assert inf.fact_used == 3 and inf.iters == 0
        t = oracle_mod.lse_truth(P["A"], P["B"], P["b"], P["d"])
        F = oracle_mod.lse_factor(P["A"], P["B"], "fp64")
        kap = oracle_mod.lse_kappa(F, t["x"], t["r"])[0]
        assert rel(x, t["x"]) <= 100 * kap * 1.1e-16


def test_batched_escalation(h, oracle_mod):
    """A problem beyond FP32 classical IR (kappa ~ 1e9) inside a batch is
    re-solved with an FP64 factorization; the others are unaffected."""
    probs = I.lse_batch(seed=15, count=8)
    probs.insert(3, I.lse_paper(404, 256, 64, 2, 1e9))
    st, infos, xs = run_batch(h, probs)
    assert st == 0
    assert infos[3].escalated == 1 and infos[3].fact_used == 3
    assert all(infos[k].escalated == 0 for k in range(len(probs)) if k != 3)
    met = oracle_mod.lse_metrics(probs[3]["A"], probs[3]["B"], probs[3]["b"], probs[3]["d"], xs[3],
                                 probs[3]["b"] - probs[3]["A"] @ xs[3], np.zeros(2))
    assert met["e_con"] <= 1e-14
    st, infos, xs = run_batch(h, probs, escalate=False)
    assert st == 3 and infos[3].status == 3


def test_batched_rejects_bad_problem(h):
    from paper_2406_16499_gb300 import mpir
    probs = I.lse_batch(seed=16, count=3)
    bad = dict(probs[1])
    bad["B"] = np.zeros((bad["A"].shape[1] + 1, bad["A"].shape[1]))   # p > n
    bad["d"] = np.zeros(bad["B"].shape[0])
    probs[1] = bad
    with pytest.raises(mpir.MpirError, match="problem 1"):
        run_batch(h, probs)


@pytest.mark.parametrize("group,m_hi", [(512, 200), (256, 200), (128, 200), (64, 40)])
def test_batched_every_launch_shape(h, oracle_mod, group, m_hi):
    """Every compiled launch shape (threads per problem) solves the batch
    (64-thread groups hold only small problems in their shared memory)."""
    probs = I.lse_batch(seed=18, count=24, m_lo=32, m_hi=m_hi)
    h.batched_set_shape(group)
    try:
        st, infos, xs = run_batch(h, probs)
        used = [h.batched_get_shape(b) for b in (0, 1)]
    finally:
        h.batched_set_shape(0)
    assert st == 0
    assert any(u["group"] == group for u in used if u["problems"])
    for P, x in zip(probs, xs):
        check(oracle_mod, P, x)


def test_batched_autotuner_near_best(h):
    """The autotuned shape is within 30% of the fastest forced shape on the
    same batch (device time of the graph launch)."""
    import torch
    from paper_2406_16499_gb300 import mpir
    probs = I.lse_batch(seed=19, count=600)
    dp = [to_dev(P) for P in probs]
    xs = [zeros(P["A"].shape[1]) for P in probs]
    batch = mpir.LseBatch(dp, xs)
    times = {}
    for g in (512, 256, 128, 64, 0):
        h.batched_set_shape(g)
        h.lse_solve_batched(batch)
        best = float("inf")
        for _ in range(3):
            mpir.profile(True)
            st, _ = h.lse_solve_batched(batch)
            torch.cuda.synchronize()
            best = min(best, mpir.profile_read()["batched"][0])
            mpir.profile(False)
        assert st == 0
        times[g] = best
    h.batched_set_shape(0)
    assert times[0] <= 1.3 * min(times[g] for g in (512, 256, 128, 64)), times
