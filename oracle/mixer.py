"""Adaptive context mixer (Sec. 3.5), FP64, and the mixed-NLL gradient.

    p_mix = sum_j w_j p^(j),  sum_j w_j = 1   (linear mixing)
    exponential weights: log w_j += eta * log p^(j)(t*), then renormalise.
    w_llm = 0.85 initially, the remaining 0.15 split over the other models;
    during the first 100 tokens only the LLM distribution is used.

Readings where the paper is silent: eta = 1 (the Bayesian-posterior case the
paper equates the rule with); the LLM component is the bias-adjusted
p_tilde; the weights stay frozen during warm-up.

Mixed-distribution NLL (differentiable update rule).  With w = softmax(theta)
and L = -log p_mix(t*), p_mix = w_0 p_tilde + w_1 p_ng, p_tilde =
softmax(log p_llm + b):
    dL/db_t     = rho * (p_tilde(t) - 1[t = t*]),  rho = w_0 p_tilde(t*) / p_mix(t*)
    dL/dtheta_j = w_j - w_j p^(j)(t*) / p_mix(t*)
and during warm-up (p = p_tilde): dL/db = p_tilde - e_{t*}, dL/dtheta = 0.
"""
from __future__ import annotations

import numpy as np


class Mixer:
    def __init__(self, n_models: int = 2, w_llm: float = 0.85, eta: float = 1.0,
                 warmup: int = 100):
        w = np.full(n_models, (1.0 - w_llm) / (n_models - 1))
        w[0] = w_llm
        self.logw = np.log(w)
        self.eta = eta
        self.warmup = warmup

    def weights(self):
        m = self.logw.max()
        e = np.exp(self.logw - m)
        return e / e.sum()

    def in_warmup(self, i: int) -> bool:
        """i is the 1-based index of the token being coded."""
        return i <= self.warmup

    def mix(self, ps, i: int):
        if self.in_warmup(i):
            return ps[0]
        w = self.weights()
        return sum(wj * pj for wj, pj in zip(w, ps))

    def update(self, p_at_tstar, i: int):
        """Exponential-weights step with the probabilities each model gave
        the observed token; skipped during warm-up."""
        if self.in_warmup(i):
            return
        self.logw = self.logw + self.eta * np.log(np.asarray(p_at_tstar, dtype=np.float64))
        m = self.logw.max()
        self.logw = self.logw - (m + np.log(np.exp(self.logw - m).sum()))


def mixed_nll(b, theta, log_p_llm, p_ng, t_star, warm: bool):
    """L = -log p_mix(t*) as a function of (b, theta); used for the
    finite-difference check of the closed-form gradient."""
    p_t = np.exp(log_p_llm + b - np.max(log_p_llm + b))
    p_t /= p_t.sum()
    if warm:
        return -np.log(p_t[t_star])
    w = np.exp(theta - theta.max())
    w /= w.sum()
    return -np.log(w[0] * p_t[t_star] + w[1] * p_ng[t_star])


def mixed_nll_grad(p_tilde, p_ng, theta, t_star, warm: bool):
    """Closed-form (dL/db, dL/dtheta) of ``mixed_nll``."""
    gb = p_tilde.copy()
    gb[t_star] -= 1.0
    if warm:
        return gb, np.zeros_like(theta)
    w = np.exp(theta - theta.max())
    w /= w.sum()
    pj = np.array([p_tilde[t_star], p_ng[t_star]])
    pm = float(w @ pj)
    rho = w[0] * pj[0] / pm
    return rho * gb, w - w * pj / pm
