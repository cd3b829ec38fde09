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


def _check_kappa(got, want):
    """The sketch runs in float32: below 1e5 the estimates agree to float32
    rounding of the Ritz values; above, both are in the saturated range."""
    for g_, w_ in zip(got, want):
        if w_ < np.log(1e5):
            assert abs(g_ - w_) < 2e-2, (got, want)
        else:
            assert g_ > np.log(1e4), (got, want)


@pytest.mark.parametrize("shape,cond", [((200, 100, 20), 1e2), ((300, 120, 0), 1e5), ((90, 60, 15), 1e9)])
def test_lse_features_match_oracle(h, shape, cond):
    from oracle import selector as S
    from paper_2406_16499_gb300 import selector as SEL
    m, n, p = shape
    P = I.lse_svd(m + n + p, m, n, p, cond, 1e1)
    f = SEL.lse_features(h, P)
    want = S.lse_features(P["A"], P["B"], P["b"], P["d"], I.splitmix_vector(n))
    assert np.abs(f[:12] - want[:12]).max() < 1e-4 * (1 + np.abs(want[:12]).max())
    assert np.abs(f[15] - want[15]) < 1e-4 * abs(want[15])
    _check_kappa(f[12:15], want[12:15])


@pytest.mark.parametrize("shape,cond", [((120, 40, 150), 1e3), ((64, 1, 80), 1e2), ((200, 150, 200), 1e6)])
def test_gls_features_match_oracle(h, shape, cond):
    from oracle import selector as S
    from paper_2406_16499_gb300 import selector as SEL
    n, m, p = shape
    G = I.gls_svd(n + m + p, n, m, p, cond, 1e1)
    f = SEL.gls_features(h, G)
    want = S.gls_features(G["W"], G["V"], G["d"], I.splitmix_vector(m + p))
    assert np.abs(f[:12] - want[:12]).max() < 1e-4 * (1 + np.abs(want[:12]).max())
    _check_kappa(f[12:15], want[12:15])


def test_training_lowers_loss(h):
    from paper_2406_16499_gb300 import selector as SEL
    g = np.random.default_rng(5)
    X = g.standard_normal((300, 16)).astype(np.float32)
    y = (np.argmax(X[:, :6] + 0.5 * X[:, 6:12], axis=1)).astype(np.int32)
    sel, losses = SEL.train(h, X, y, steps=400, lr=1e-2, log_every=100)
    assert losses[0][1] > 1.0 and losses[-1][1] < 0.25, losses
    pred = np.argmax(sel.predict(h, X), axis=1)
    assert (pred == y).mean() > 0.9


def _solve_wall(h, P, **kw):
    import torch
    from paper_2406_16499_gb300 import mpir
    A, B, b, d = dev(P["A"]), dev(P["B"]), dev(P["b"]), dev(P["d"])
    m, n = P["A"].shape
    p = P["B"].shape[0]
    x, r, v = zeros(n), zeros(m), zeros(max(p, 1))
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    st, info = h.lse_solve(A, B, b, d, x, r, v if p else None, mpir.make_opts(**kw))
    torch.cuda.synchronize()
    return st, info, (time.perf_counter() - t0) * 1e3, host(x), host(r), host(v)[:p]


def test_selector_gain_over_fixed_fp32(h, oracle_mod):
    """Train on 160 problems (kappa log-uniform in [1, 1e12]), evaluate on 60
    held-out ones: the selector's total solve time (features + inference +
    its choice + escalation) is below the method without it, and every
    answer meets the FP64-level bar."""
    from paper_2406_16499_gb300 import selector as SEL
    train_p = I.selector_lse_problems(101, 160)
    test_p = I.selector_lse_problems(202, 60)
    X, y = [], []
    for P in train_p:
        times, ok = SEL.time_lse_classes(h, P)
        lab = SEL.label(times, ok)
        if lab < 0:
            continue
        X.append(SEL.lse_features(h, P))
        y.append(lab)
    assert len(set(y)) >= 2
    sel, losses = SEL.train(h, np.array(X), np.array(y), steps=800, lr=3e-3)
    sel.install(h)
    # warm-up of both paths
    _solve_wall(h, test_p[0], fact="fp32")
    _solve_wall(h, test_p[0], fact="auto")
    t_base = t_sel = 0.0
    for P in test_p:
        st0, _, tb, *_ = _solve_wall(h, P, fact="fp32", refine="classical")
        st1, info, ts, x, r, v = _solve_wall(h, P, fact="auto")
        assert st0 == 0 and st1 == 0
        t_base += tb
        t_sel += ts
        met = oracle_mod.lse_metrics(P["A"], P["B"], P["b"], P["d"], x, r, v)
        assert met["e_con"] <= 1e-14 and met["eta"] <= 1e-14, met
    h.selector_set(None, None, None)
    print("selector total %.1f ms vs fixed FP32 + escalation %.1f ms" % (t_sel, t_base))
    assert t_sel < t_base
