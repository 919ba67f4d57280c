"""Interpolated token N-gram model (Sec. 3.4), FP64.

Unigram base, Laplace smoothed:   P_uni(t) = (c(t) + 1) / (N + V).
For k = 1..order, with context c_k = (t_{i-k}, ..., t_{i-1}) seen n_k times:
    P_k = lambda_k * Phat_k(. | c_k) + (1 - lambda_k) * P_{k-1},
    lambda_k = n_k / (n_k + eps),  eps = 5,  Phat_k(t | c_k) = cnt(c_k, t) / n_k.

Storage (Sec. 3.4, second half): each context keeps at most 64 continuation
slots; when a 65th distinct continuation arrives, the slot with the lowest
count is evicted (ties: lowest slot index) and the new token takes it with
count 1.

Readings where the paper is silent:
* n_k is the sum of the retained continuation counts of c_k, so Phat_k is a
  distribution even after evictions;
* an unseen context (or fewer than k tokens of history) gives lambda_k = 0;
* context keys are exact tuples (the paper's 64-bit rolling hash only speeds
  up lookups; with V < 2^16 three ids pack injectively into 64 bits, so
  there are no collisions to model);
* predict happens before the update; the update adds one count to each
  available context order, to c(t) and to N.
"""
from __future__ import annotations

import numpy as np

EPS = 5.0
MAX_SLOTS = 64


class NGram:
    def __init__(self, vocab: int, order: int = 3, max_slots: int = MAX_SLOTS, eps: float = EPS):
        self.V = vocab
        self.order = order
        self.max_slots = max_slots
        self.eps = eps
        self.uni = np.zeros(vocab, dtype=np.int64)
        self.N = 0
        # per order k: dict context-tuple -> list of [token, count]
        self.tables = [dict() for _ in range(order + 1)]
        self.hist: list[int] = []

    def context_entry(self, k: int):
        if len(self.hist) < k:
            return None
        return self.tables[k].get(tuple(self.hist[-k:]))

    def lambdas(self):
        """lambda_k for k = 1..order at the current history (index 0 unused)."""
        lam = [0.0] * (self.order + 1)
        for k in range(1, self.order + 1):
            e = self.context_entry(k)
            if e:
                n = sum(c for _, c in e)
                lam[k] = n / (n + self.eps)
        return lam

    def predict(self) -> np.ndarray:
        """P_order over the vocabulary (float64[V]), by the recursion above."""
        P = (self.uni + 1.0) / (self.N + self.V)
        for k in range(1, self.order + 1):
            e = self.context_entry(k)
            if not e:
                continue
            n = sum(c for _, c in e)
            lam = n / (n + self.eps)
            phat = np.zeros(self.V)
            for t, c in e:
                phat[t] = c / n
            P = lam * phat + (1.0 - lam) * P
        return P

    def update(self, t: int):
        for k in range(1, min(self.order, len(self.hist)) + 1):
            key = tuple(self.hist[-k:])
            slots = self.tables[k].setdefault(key, [])
            for s in slots:
                if s[0] == t:
                    s[1] += 1
                    break
            else:
                if len(slots) < self.max_slots:
                    slots.append([t, 1])
                else:
                    j = min(range(len(slots)), key=lambda i: (slots[i][1], i))
                    slots[j] = [t, 1]
        self.uni[t] += 1
        self.N += 1
        self.hist.append(int(t))
