"""Adaptive log-space bias head (Sec. 3.6), FP64.

    p_tilde = softmax(log p_llm + b),   b in R^V, b_0 = 0
    after the observed token t*:  b_t -= alpha * (p_tilde(t) - 1[t = t*]),
    alpha = 1e-3 (the gradient of -log p_tilde(t*) w.r.t. b).

p_llm is the temperature softmax of the logits, softmax(z / tau) (Sec. 3.2,
tau = 1 by default).
"""
from __future__ import annotations

import numpy as np


def softmax(x):
    e = np.exp(x - np.max(x))
    return e / e.sum()


def p_llm(z, tau: float = 1.0):
    return softmax(np.asarray(z, dtype=np.float64) / tau)


class BiasHead:
    def __init__(self, vocab: int, alpha: float = 1e-3):
        self.b = np.zeros(vocab)
        self.alpha = alpha

    def adjust(self, p):
        """p_tilde = softmax(log p + b)."""
        with np.errstate(divide="ignore"):
            return softmax(np.log(p) + self.b)

    def grad(self, p_tilde, t_star):
        g = p_tilde.copy()
        g[t_star] -= 1.0
        return g

    def update(self, p_tilde, t_star, scale: float = 1.0):
        """b -= alpha * scale * (p_tilde - e_{t*}).  scale = 1 is the paper's
        rule; the mixed-NLL rule passes the LLM responsibility rho."""
        self.b -= self.alpha * scale * self.grad(p_tilde, t_star)
