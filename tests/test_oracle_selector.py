"""Pins of the selector oracle (oracle/selector.py) against mathematics that
does not depend on it: central finite differences of the loss, closed forms
of the untrained network, Ritz-value interlacing and exactness of the
Golub-Kahan-Lanczos sketch, the bfloat16 rounding rule and the labelling
rule."""
import numpy as np
import pytest

from oracle import selector as S


def _params(seed=3):
    return S.init_params(seed)


def test_zero_network_is_uniform():
    P = {k: np.zeros_like(v) for k, v in _params().items()}
    X = np.random.default_rng(0).standard_normal((9, 16))
    prob, _ = S.forward(P, X)
    assert np.allclose(prob, 1.0 / 6.0)
    assert abs(S.loss(P, X, np.arange(9) % 6) - np.log(6.0)) < 1e-15


def test_softmax_rows_sum_to_one():
    P = _params()
    X = np.random.default_rng(1).standard_normal((20, 16)) * 3
    prob, _ = S.forward(P, X)
    assert np.allclose(prob.sum(axis=1), 1.0, atol=1e-14) and (prob > 0).all()


def test_gradients_match_central_differences():
    P = _params(5)
    g = np.random.default_rng(2)
    X = g.standard_normal((7, 16))
    y = g.integers(0, 6, 7)
    G = S.backward(P, X, y)
    h = 1e-6
    for name in ("W1", "b1", "W2", "b2", "W3", "b3"):
        flat = P[name].reshape(-1)
        for idx in g.choice(flat.size, size=min(12, flat.size), replace=False):
            old = flat[idx]
            flat[idx] = old + h
            lp = S.loss(P, X, y)
            flat[idx] = old - h
            lm = S.loss(P, X, y)
            flat[idx] = old
            fd = (lp - lm) / (2 * h)
            an = G[name].reshape(-1)[idx]
            assert abs(fd - an) <= 1e-7 + 1e-5 * abs(an), (name, idx, fd, an)


def test_adam_first_step_is_signed_lr():
    """With bias correction, the first Adam step moves every parameter with a
    nonzero gradient by lr * g / (|g| + eps) ~ lr * sign(g)."""
    P = _params(7)
    g = np.random.default_rng(4)
    G = {k: g.standard_normal(v.shape) for k, v in P.items()}
    old = {k: v.copy() for k, v in P.items()}
    S.adam_step(P, G, {}, lr=1e-2)
    for k in P:
        assert np.allclose(old[k] - P[k], 1e-2 * G[k] / (np.abs(G[k]) + 1e-8), rtol=1e-12)


@pytest.mark.parametrize("shape,cond", [((120, 40), 1e3), ((60, 30), 1e6), ((300, 200), 1e2), ((15, 60), 1e1),
                                        ((40, 300), 1e4)])
def test_kappa_hat_below_kappa(shape, cond):
    """Interlacing: sigma_max / sigma_rank bounds the sketch (wide matrices
    included, whose start vector is mapped into range(M^T))."""
    from paper_2406_16499_gb300 import inputs as I
    g = I.rng(11)
    r = min(shape)
    M = I.svd_matrix(g, shape[0], shape[1], I.logspace_sigma(r, cond))
    s = g.standard_normal(shape[1])
    kh = S.kappa_hat(lambda x: M @ x, lambda y: M.T @ y, s, min(16, r), shape[0] < shape[1])
    assert 1.0 <= kh <= cond * (1 + 1e-8)
    if r <= 16:
        assert abs(kh / cond - 1) < 1e-6


def test_kappa_hat_exact_for_few_columns():
    """k >= number of columns: the sketch is the full bidiagonalization."""
    from paper_2406_16499_gb300 import inputs as I
    g = I.rng(12)
    M = I.svd_matrix(g, 50, 10, I.logspace_sigma(10, 1e3))
    s = g.standard_normal(10)
    kh = S.kappa_hat(lambda x: M @ x, lambda y: M.T @ y, s, 16)
    assert abs(kh / 1e3 - 1) < 1e-8


def test_kappa_hat_exact_at_rank_ill_conditioned():
    """k = rank on a tall block with cond 1e10: the fully reorthogonalized
    FP64 sketch is the complete bidiagonalization, so kappa^ is the
    condition number itself (a single-precision sketch, or one stopped at
    single-precision rounding level, saturates orders of magnitude lower)."""
    from paper_2406_16499_gb300 import inputs as I
    for seed, cond in ((13, 1e6), (14, 1e10)):
        g = I.rng(seed)
        M = I.svd_matrix(g, 300, 12, I.logspace_sigma(12, cond))
        s = I.splitmix_vector(12)
        kh = S.kappa_of(M, s, 12)
        assert abs(kh / cond - 1) < 1e-5, (kh, cond)


def test_features_layout():
    from paper_2406_16499_gb300 import inputs as I
    P = I.lse_small()
    s = np.random.default_rng(0).standard_normal(100)
    f = S.lse_features(P["A"], P["B"], P["b"], P["d"], s)
    assert f.shape == (16,)
    assert f[0] == pytest.approx(np.log(200)) and f[1] == pytest.approx(np.log(100))
    assert f[3] == pytest.approx(0.5) and f[4] == pytest.approx(0.2) and f[5] == 0.0
    assert f[7] == pytest.approx(np.log(np.linalg.norm(P["A"])))
    assert f[12] <= np.log(1e2) + 1e-5          # kappa(A) = 1e2 by construction
    G = I.gls_svd(5, 60, 20, 80, 1e3, 1e1)
    s = np.random.default_rng(1).standard_normal(100)
    f = S.gls_features(G["W"], G["V"], G["d"], s)
    assert f[5] == 1.0 and f[0] == pytest.approx(np.log(60)) and f[4] == pytest.approx(60 / 80)
    assert f[12] <= np.log(1e3) + 1e-5


def test_bf16_rounding():
    x = np.array([1.0, 1 + 2 ** -8, 1 + 3 * 2 ** -9, 1 + 2 ** -7, -2.5, 3.0e38, 1e-40])
    r = S.bf16_round(x)
    assert r[0] == 1.0
    assert r[1] == 1.0                     # halfway, ties to even
    assert r[2] == 1 + 2 ** -7
    assert r[3] == 1 + 2 ** -7
    assert r[4] == -2.5
    assert abs(r[5] / 3.0e38 - 1) < 2 ** -8


def test_label_rule():
    t = [1.0, 1.0, 1.02, 5.0, 3.0, 9.0]
    assert S.label(t, [True] * 6) == 2           # fp32 classical within 3% beats bf16
    assert S.label(t, [False, False, False, True, True, True]) == 4
    assert S.label(t, [False] * 6) == -1
    assert S.label([2.0, 2.0, 2.0, 2.0, 2.0, 2.0], [True] * 6) == 4   # fp64 classical on a tie
