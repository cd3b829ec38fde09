"""The learned selector on the GPU against the oracle (oracle/selector.py).

* Forward, gradients and the Adam step of the MLP kernels against the FP64
  oracle on the same bfloat16-rounded weights.
* The 16 features (norms, dimensions, Golub-Kahan-Lanczos condition sketch)
  against the oracle with the same start vector.
* Training with the library's kernels lowers the loss.
* Gain: a selector trained on solves the library itself timed picks, on
  held-out problems, configurations whose total time (features, inference
  and escalation included) is below that of the method without it (always
  FP32 factors + classical IR, escalating to FP64 on failure), with every
  answer meeting the FP64-level bar (oracle metrics).
"""
import time

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


def _split(flat):
    from oracle import selector as S
    o, P = 0, {}
    for name, shape in (("W1", (64, 16)), ("b1", (64,)), ("W2", (64, 64)), ("b2", (64,)), ("W3", (6, 64)),
                        ("b3", (6,))):
        k = int(np.prod(shape))
        v = np.asarray(flat[o:o + k], np.float64).reshape(shape)
        P[name] = S.bf16_round(v) if name.startswith("W") else v
        o += k
    return P


def _flat(G):
    return np.concatenate([G[k].reshape(-1) for k in ("W1", "b1", "W2", "b2", "W3", "b3")])


def test_mlp_forward_and_gradients_match_oracle(h):
    import torch
    from oracle import selector as S
    from paper_2406_16499_gb300 import selector as SEL
    g = np.random.default_rng(0)
    params = SEL.init_params(3) + np.float32(0.01) * g.standard_normal(SEL.PARAMS).astype(np.float32)
    X = g.standard_normal((37, 16)).astype(np.float32)
    y = g.integers(0, 6, 37).astype(np.int32)
    P = torch.from_numpy(params).cuda()
    prob = torch.zeros((37, 6), dtype=torch.float32, device="cuda")
    h.mlp_forward(P, torch.from_numpy(X).cuda(), prob)
    Po = _split(params)
    want, _ = S.forward(Po, X.astype(np.float64))
    assert np.abs(prob.cpu().numpy() - want).max() < 2e-6
    grad = torch.zeros(SEL.PARAMS, dtype=torch.float32, device="cuda")
    loss = torch.zeros(1, dtype=torch.float32, device="cuda")
    h.mlp_train_step(P, None, None, 1, 0.0, torch.from_numpy(X).cuda(), torch.from_numpy(y).cuda(), grad, loss)
    gw = _flat(S.backward(Po, X.astype(np.float64), y))
    gg = grad.cpu().numpy()
    assert np.abs(gg - gw).max() <= 1e-5 * np.abs(gw).max() + 1e-7
    assert abs(loss.item() - S.loss(Po, X.astype(np.float64), y)) < 1e-5


def test_adam_step_matches_oracle(h):
    import torch
    from oracle import selector as S
    from paper_2406_16499_gb300 import selector as SEL
    g = np.random.default_rng(1)
    params = SEL.init_params(4)
    X = g.standard_normal((20, 16)).astype(np.float32)
    y = g.integers(0, 6, 20).astype(np.int32)
    P = torch.from_numpy(params.copy()).cuda()
    M, V = torch.zeros_like(P), torch.zeros_like(P)
    grad = torch.zeros_like(P)
    for t in (1, 2):
        h.mlp_train_step(P, M, V, t, 1e-2, torch.from_numpy(X).cuda(), torch.from_numpy(y).cuda(), grad)
    # oracle: the same two steps from the same start, gradients on bf16 weights
    flat = params.astype(np.float64)
    state = {}
    for t in (1, 2):
        G = _flat(S.backward(_split(flat), X.astype(np.float64), y))
        Pd = {"w": flat.copy()}
        S.adam_step(Pd, {"w": G}, state, lr=1e-2)
        flat = Pd["w"]
    assert np.abs(P.cpu().numpy() - flat).max() < 2e-5


U32 = 2.0 ** -24


def _kappa_ref(M, s):
    """The oracle's kappa^ of one block (FP64, fully reorthogonalized GKL)
    and the tolerance on 1/kappa^ that float32 rounding allows.

    The GPU runs the same k steps with float32 vectors and products: its
    bidiagonal is that of a perturbed block M + E with ||E||_2 of order
    u_single ||M||_F, so its smallest Ritz value moves by at most about that
    much and |1/kappa^_gpu - 1/kappa^| <= c u_single ||M||_F / sigma_max.
    c = 2 (the float32 sums on the GPU run in another order than the
    dot products of a float32 emulation, which stayed below c = 0.25 on
    these blocks).  Above kappa^ ~ 1e6 this still separates 1e6 from 1e9.
    The bidiagonal's extreme singular values come from FP32 bisection, whose
    relative error is O(k u_single) (relative perturbation theory of
    bidiagonals), and the feature holds log kappa^ in FP32: together at most
    (4 k + |log kappa^|) u_single / kappa^ on 1/kappa^."""
    from oracle import selector as S
    M = np.asarray(M, np.float64)
    rows, cols = M.shape
    k = min(16, rows, cols)
    s0 = M.T @ (M @ s) if rows < cols else np.asarray(s, np.float64)
    Bk = S.gkl_bidiag(lambda x: M @ x, lambda y: M.T @ y, s0, k)
    sv = np.linalg.svd(Bk, compute_uv=False)
    kap = sv[0] / sv[-1]
    # + the FP32 bisection on the bidiagonal (relative O(k u_single) on each
    # of sigma_max, sigma_min: Demmel-Kahan) and the FP32 feature log kappa^
    return kap, 2 * U32 * np.linalg.norm(M) / sv[0] + (4 * k + abs(np.log(kap))) * U32 / kap


def _check_kappa(got_logs, blocks):
    for g_, (M, s) in zip(got_logs, blocks):
        want, tol = _kappa_ref(M, s)
        got = float(np.exp(g_))
        assert abs(1.0 / got - 1.0 / want) <= tol, (got, want, tol)


@pytest.mark.parametrize("shape,cond", [((200, 100, 20), 1e2), ((300, 120, 0), 1e5), ((90, 60, 15), 1e9),
                                        ((300, 12, 4), 1e6), ((300, 12, 4), 1e8)])
def test_lse_features_match_oracle(h, shape, cond):
    """Features of an LSE problem.  A 300 x 12 block is sketched in full
    (k = 12 = rank), so kappa^(A) is cond(A) itself there."""
    from oracle import selector as S
    from paper_2406_16499_gb300 import selector as SEL
    m, n, p = shape
    P = I.lse_svd(m + n + p, m, n, p, cond, 1e1)
    f = SEL.lse_features(h, P)
    sv = I.splitmix_vector(n)
    want = S.lse_features(P["A"], P["B"], P["b"], P["d"], sv)
    assert np.abs(f[:12] - want[:12]).max() < 1e-4 * (1 + np.abs(want[:12]).max())
    assert np.abs(f[15] - want[15]) < 1e-4 * abs(want[15])
    if n <= 16:
        assert abs(want[12] - np.log(cond)) < 1e-6          # the sketch is the full bidiagonalization
    blocks = [(P["A"], sv), (P["B"], sv), (np.vstack([P["A"], P["B"]]), sv)]
    if p == 0:
        blocks[1] = None
    for j, blk in enumerate(blocks):
        if blk is not None:
            _check_kappa([f[12 + j]], [blk])


@pytest.mark.parametrize("shape,cond", [((120, 40, 150), 1e3), ((64, 1, 80), 1e2), ((200, 150, 200), 1e6)])
def test_gls_features_match_oracle(h, shape, cond):
    from oracle import selector as S
    from paper_2406_16499_gb300 import selector as SEL
    n, m, p = shape
    G = I.gls_svd(n + m + p, n, m, p, cond, 1e1)
    f = SEL.gls_features(h, G)
    sv = I.splitmix_vector(m + p)
    want = S.gls_features(G["W"], G["V"], G["d"], sv)
    assert np.abs(f[:12] - want[:12]).max() < 1e-4 * (1 + np.abs(want[:12]).max())
    _check_kappa(f[12:15], [(G["W"], sv[:m]), (G["V"], sv[m:]), (np.hstack([G["W"], G["V"]]), sv)])


def test_training_lowers_loss(h):
    from paper_2406_16499_gb300 import selector as SEL
    g = np.random.default_rng(5)
    X = g.standard_normal((300, 16)).astype(np.float32)
    y = (np.argmax(X[:, :6] + 0.5 * X[:, 6:12], axis=1)).astype(np.int32)
    sel, losses = SEL.train(h, X, y, steps=400, lr=1e-2, log_every=100)
    assert losses[0][1] > 1.0 and losses[-1][1] < 0.25, losses
    pred = np.argmax(sel.predict(h, X), axis=1)
    assert (pred == y).mean() > 0.9


def _solve_wall(h, kind, P, **kw):
    import torch
    from paper_2406_16499_gb300 import mpir
    if kind == "lse":
        A, B, b, d = dev(P["A"]), dev(P["B"]), dev(P["b"]), dev(P["d"])
        m, n = P["A"].shape
        p = P["B"].shape[0]
        x, r, v = zeros(n), zeros(m), zeros(max(p, 1))
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        st, info = h.lse_solve(A, B, b, d, x, r, v if p else None, mpir.make_opts(**kw))
        torch.cuda.synchronize()
        return st, info, (time.perf_counter() - t0) * 1e3, (host(x), host(r), host(v)[:p])
    W, V, d = dev(P["W"]), dev(P["V"]), dev(P["d"])
    n, m = P["W"].shape
    p = P["V"].shape[1]
    x, y, z = zeros(m), zeros(p), zeros(n)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    st, info = h.gls_solve(W, V, d, x, y, z, mpir.make_opts(**kw))
    torch.cuda.synchronize()
    return st, info, (time.perf_counter() - t0) * 1e3, (host(x), host(y), host(z))


def test_selector_gain_over_fixed_fp32(h, oracle_mod):
    """Train on 100 LSE + 80 GLS problems (kappa log-uniform in [1, 1e12]),
    labelled by the library's own timed solves of the six classes; evaluate
    on 40 LSE + 30 GLS held-out problems: the selector's total solve time
    (features + inference + its choice + escalation) is below the method
    without it (always FP32 factors + classical IR, escalating on failure),
    and every answer meets the FP64-level bar (oracle metrics)."""
    from paper_2406_16499_gb300 import selector as SEL
    caps = dict(maxit=20, inner_maxit=200)
    train_p = [("lse", P) for P in I.selector_lse_problems(101, 100)]
    train_p += [("gls", G) for G in I.selector_gls_problems(102, 80)]
    test_p = [("lse", P) for P in I.selector_lse_problems(202, 40)]
    test_p += [("gls", G) for G in I.selector_gls_problems(203, 30)]
    X, y = [], []
    for kind, P in train_p:
        if kind == "lse":
            times, ok = SEL.time_lse_classes(h, P, **caps)
            f = SEL.lse_features(h, P)
        else:
            times, ok = SEL.time_gls_classes(h, P, **caps)
            f = SEL.gls_features(h, P)
        lab = SEL.label(times, ok)
        if lab < 0:
            continue
        X.append(f)
        y.append(lab)
    assert len(set(y)) >= 2
    sel, losses = SEL.train(h, np.array(X), np.array(y), steps=800, lr=3e-3)
    sel.install(h)
    # warm-up of both paths
    for kind, P in (test_p[0], test_p[-1]):
        _solve_wall(h, kind, P, fact="fp32")
        _solve_wall(h, kind, P, fact="auto")
    t_base = t_sel = 0.0
    for kind, P in test_p:
        st0, _, tb, _ = _solve_wall(h, kind, P, fact="fp32", refine="classical")
        st1, info, ts, sol = _solve_wall(h, kind, P, fact="auto")
        assert st0 == 0 and st1 == 0
        t_base += tb
        t_sel += ts
        if kind == "lse":
            met = oracle_mod.lse_metrics(P["A"], P["B"], P["b"], P["d"], *sol)
        else:
            met = oracle_mod.gls_metrics(P["W"], P["V"], P["d"], *sol)
        assert met["e_con"] <= 1e-14 and met["eta"] <= 1e-14, (kind, met)
    h.selector_set(None, None, None)
    print("selector total %.1f ms vs fixed FP32 + escalation %.1f ms" % (t_sel, t_base))
    assert t_sel < t_base
