"""Pins for the mixer (Sec. 3.5), the adaptive bias head (Sec. 3.6) and the
mixed-NLL gradient: the paper's worked example, identity at zero bias, the
zero-sum invariant, the Bayesian closed form of exponential weights and
central finite differences."""
import json
import os

import numpy as np

from oracle.head import BiasHead, p_llm, softmax
from oracle.mixer import Mixer, mixed_nll, mixed_nll_grad

GOLD = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "paper_values.json")))


def test_mixer_worked_example_lower_bound():
    ex = GOLD["mixer_example"]
    m = Mixer(2, w_llm=ex["w_llm"])
    w = m.weights()
    assert abs(w[0] - GOLD["mixer_init_w_llm"]["value"]) < 1e-15 and abs(w[1] - 0.15) < 1e-15
    rng = np.random.default_rng(0)
    V = 50
    pl = rng.dirichlet(np.ones(V)) * 0.1
    pl[3] = 0.0
    pl = pl / pl.sum() * 0.1
    pl[3] = ex["p_llm"]
    pn = rng.dirichlet(np.ones(V))
    pm = m.mix([pl, pn], i=GOLD["mixer_warmup_tokens"]["value"] + 1)
    assert pm[3] >= ex["lower_bound"] - 1e-15
    assert abs(ex["w_llm"] * ex["p_llm"] - ex["lower_bound"]) < 1e-12
    assert np.all(pm >= w[0] * pl - 1e-17)
    assert abs(pm.sum() - 1.0) < 1e-12


def test_warmup_uses_llm_only_and_freezes():
    m = Mixer(2)
    pl, pn = np.array([0.7, 0.3]), np.array([0.1, 0.9])
    for i in range(1, 101):
        assert np.array_equal(m.mix([pl, pn], i), pl)
        m.update([0.7, 0.1], i)
    assert np.allclose(m.weights(), [0.85, 0.15], rtol=0, atol=1e-15)
    assert not np.array_equal(m.mix([pl, pn], 101), pl)


def test_exponential_weights_is_bayes_posterior():
    """eta = 1: w_j(after n) is proportional to w_j(0) * prod_i p^(j)(t_i)."""
    rng = np.random.default_rng(1)
    m = Mixer(2, warmup=0)
    logs = np.zeros(2)
    for i in range(1, 60):
        pj = rng.random(2) * 0.5 + 1e-3
        m.update(pj, i)
        logs += np.log(pj)
    post = np.array([0.85, 0.15]) * np.exp(logs - logs.max())
    post /= post.sum()
    np.testing.assert_allclose(m.weights(), post, rtol=1e-10)


def test_head_identity_at_zero_bias():
    rng = np.random.default_rng(2)
    z = rng.normal(0, 1, 300)
    p = p_llm(z)
    h = BiasHead(300)
    np.testing.assert_allclose(h.adjust(p), p, rtol=1e-13)


def test_head_sum_zero_and_fd_gradient():
    rng = np.random.default_rng(3)
    V = 64
    h = BiasHead(V)
    for _ in range(50):
        z = rng.normal(0, 1, V)
        pt = h.adjust(p_llm(z))
        t = int(rng.integers(V))
        # central finite difference of L(b) = -log softmax(log p_llm + b)[t]
        lp = np.log(p_llm(z))
        eps = 1e-3
        g_fd = np.empty(V)
        for k in range(V):
            e = np.zeros(V)
            e[k] = eps
            g_fd[k] = (-np.log(softmax(lp + h.b + e)[t]) + np.log(softmax(lp + h.b - e)[t])) / (2 * eps)
        np.testing.assert_allclose(h.grad(pt, t), g_fd, rtol=1e-5, atol=1e-8)
        h.update(pt, t)
        assert abs(h.b.sum()) < 1e-14


def test_mixed_nll_gradient_fd_and_reduction():
    rng = np.random.default_rng(4)
    V = 40
    for trial in range(8):
        lp = np.log(p_llm(rng.normal(0, 1, V)))
        b = rng.normal(0, 0.1, V)
        theta = np.log(np.array([0.7, 0.3])) + rng.normal(0, 0.3, 2)
        png = rng.dirichlet(np.ones(V))
        t = int(rng.integers(V))
        pt = softmax(lp + b)
        for warm in (False, True):
            gb, gth = mixed_nll_grad(pt, png, theta, t, warm)
            eps = 1e-3
            fb = np.array([(mixed_nll(b + eps * e, theta, lp, png, t, warm)
                            - mixed_nll(b - eps * e, theta, lp, png, t, warm)) / (2 * eps)
                           for e in np.eye(V)])
            ft = np.array([(mixed_nll(b, theta + eps * e, lp, png, t, warm)
                            - mixed_nll(b, theta - eps * e, lp, png, t, warm)) / (2 * eps)
                           for e in np.eye(2)])
            np.testing.assert_allclose(gb, fb, rtol=1e-5, atol=1e-8)
            np.testing.assert_allclose(gth, ft, rtol=1e-5, atol=1e-8)
    # w_ng -> 0 gives rho -> 1: the paper's head gradient
    theta = np.array([0.0, -800.0])
    gb, gth = mixed_nll_grad(pt, png, theta, t, False)
    g_paper = pt.copy()
    g_paper[t] -= 1
    np.testing.assert_allclose(gb, g_paper, rtol=1e-12, atol=1e-15)
    assert np.allclose(gth, 0, atol=1e-300)


def test_temperature_softmax_power_identity_and_limits():
    """p_llm at temperature tau (Sec. 3.2) against facts that do not restate
    its formula: softmax(z / tau) is the tau-th root power of softmax(z),
    renormalised; tau = 1 is the plain softmax; tau -> 0 tends to the one-hot
    argmax and large tau to the uniform distribution; the order of the
    probabilities never changes."""
    rng = np.random.default_rng(3)
    z = rng.normal(0, 2, 500)
    e = np.exp(z - z.max())
    p1 = e / e.sum()
    assert np.allclose(p_llm(z, 1.0), p1, rtol=1e-13, atol=0)
    for tau in (0.7, 0.8, 1.3, 2.5):
        q = p1 ** (1.0 / tau)
        assert np.allclose(p_llm(z, tau), q / q.sum(), rtol=1e-10, atol=1e-300)
        assert np.array_equal(np.argsort(p_llm(z, tau), kind="stable"), np.argsort(p1, kind="stable"))
    cold = p_llm(z, 1e-3)
    assert abs(cold[np.argmax(z)] - 1.0) < 1e-12
    hot = p_llm(z, 1e6)
    assert np.max(np.abs(hot * len(z) - 1.0)) < 1e-4
