"""Pins for the oracle's token N-gram (Sec. 3.4): uniform start, normalisation,
brute-force recount through the closed form of the interpolation recursion,
and a hand-worked eviction case."""
import numpy as np
import pytest

from oracle.ngram import NGram


def brute_predict(hist, V, order=3, eps=5.0):
    """Independent formulation: counts by scanning the history, and the
    closed form of the recursion,
        P = prod_k (1 - l_k) P_uni + sum_k l_k prod_{j>k} (1 - l_j) Phat_k."""
    N = len(hist)
    uni = np.bincount(np.asarray(hist, dtype=np.int64), minlength=V).astype(np.float64) if N else np.zeros(V)
    P_uni = (uni + 1.0) / (N + V)
    lam = np.zeros(order + 1)
    phat = [None] * (order + 1)
    for k in range(1, order + 1):
        if N < k:
            continue
        ctx = tuple(hist[N - k:])
        cnt = np.zeros(V)
        for i in range(k, N):                        # t_i follows hist[i-k:i]
            if tuple(hist[i - k:i]) == ctx:
                cnt[hist[i]] += 1
        n = cnt.sum()
        if n > 0:
            lam[k] = n / (n + eps)
            phat[k] = cnt / n
    out = np.prod(1 - lam[1:]) * P_uni
    for k in range(1, order + 1):
        if lam[k] > 0:
            out = out + lam[k] * np.prod(1 - lam[k + 1:]) * phat[k]
    return out


def test_first_step_uniform():
    g = NGram(1000)
    p = g.predict()
    assert np.allclose(p, 1.0 / 1000, rtol=0, atol=1e-18)


@pytest.mark.parametrize("seed", [0, 1, 2])
def test_bruteforce_recount(seed):
    V = 40
    rng = np.random.default_rng(seed)
    # low-entropy stream so contexts repeat, short enough that no context
    # reaches 64 continuations (no eviction)
    toks = []
    for i in range(400):
        if i >= 2 and rng.random() < 0.6:
            toks.append((toks[-1] * 7 + toks[-2]) % 11)
        else:
            toks.append(int(rng.integers(V)))
    g = NGram(V)
    for i, t in enumerate(toks):
        p = g.predict()
        assert abs(p.sum() - 1.0) < 1e-12
        if i % 17 == 0 or i < 10:
            np.testing.assert_allclose(p, brute_predict(toks[:i], V), rtol=1e-12, atol=1e-15)
        g.update(t)


def test_eviction_hand_worked():
    """Context (9,) with 3 slots: continuations 1,2,2,3,3,3 fill the slots
    as [1:1, 2:2, 3:3]; a 4th distinct continuation 4 evicts the lowest
    count (token 1, slot 0) -> [4:1, 2:2, 3:3]; then 5 evicts the lowest
    count with the lowest slot index (token 4, slot 0, count 1) -> [5:1, 2:2, 3:3];
    then 2 increments -> [5:1, 2:3, 3:3]; then 6 evicts slot 0 again."""
    g = NGram(16, order=1, max_slots=3)
    seq = [9, 1, 9, 2, 9, 2, 9, 3, 9, 3, 9, 3]
    for t in seq:
        g.update(t)
    assert g.tables[1][(9,)] == [[1, 1], [2, 2], [3, 3]]
    for t in [9, 4]:
        g.update(t)
    assert g.tables[1][(9,)] == [[4, 1], [2, 2], [3, 3]]
    for t in [9, 5]:
        g.update(t)
    assert g.tables[1][(9,)] == [[5, 1], [2, 2], [3, 3]]
    for t in [9, 2, 9, 6]:
        g.update(t)
    assert g.tables[1][(9,)] == [[6, 1], [2, 3], [3, 3]]
    # n_1 is the retained count: lambda_1 = 7 / 12 at context (9,)
    g.update(9)
    lam = g.lambdas()
    assert abs(lam[1] - 7.0 / 12.0) < 1e-15
    p = g.predict()
    assert abs(p.sum() - 1.0) < 1e-12


def test_eviction_tie_on_count_picks_lowest_slot():
    g = NGram(16, order=1, max_slots=2)
    for t in [5, 1, 5, 2, 5, 3]:           # (5): [1:1, 2:1] then 3 evicts slot 0
        g.update(t)
    assert g.tables[1][(5,)] == [[3, 1], [2, 1]]
