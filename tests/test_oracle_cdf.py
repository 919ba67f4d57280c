"""Pins for the oracle's CDF quantiser (Sec. 3.3) against closed forms, the
paper's printed figures and exact rational arithmetic."""
import json
import math
import os

import numpy as np
import pytest

from oracle import cdf as Q

GOLD = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "paper_values.json")))
V = GOLD["vocab"]["value"]
T24 = GOLD["T24"]["value"]


def test_k_bins_and_paper_slip():
    K = Q.k_bins(T24, V, 1)
    assert K == 16_728_064
    # the paper's printed figure is exactly 1,000 short of T - V
    assert K - GOLD["K_T24_as_printed"]["value"] == 1000


def test_floor_share_closed_forms():
    assert V / (1 << 16) == 0.75                                   # exact
    assert abs(V / (1 << 16) - GOLD["floor_share_T16"]["value"]) < 1e-12
    assert (1 << 16) - V == GOLD["free_counts_T16"]["value"]
    assert abs(100 * V / T24 - GOLD["floor_share_T24_percent"]["value"]) < 0.005
    dH16 = math.log2((1 << 16) / ((1 << 16) - V))
    assert dH16 == GOLD["delta_H_T16_bits"]["value"]              # log2(4) exactly
    dH24 = math.log2(T24 / (T24 - V))
    assert abs(dH24 - 0.004233) < 1e-6
    assert abs(dH24 - GOLD["floor_overhead_T24_bits"]["value"]) < 5e-4


def test_uniform_T24_worked_example():
    p = np.full(V, np.float32(1.0) / np.float32(V), dtype=np.float32)
    c = Q.probs_to_counts(p, T24)
    # floor(fp32(1/V) * K) = 340 for every symbol, sum 16,711,680,
    # residual 65,536 to the first maximum (index 0)
    assert np.all(c[1:] == 340)
    assert 340 * V == 16_711_680
    assert c[0] == 340 + 65_536 == 65_876
    assert c.sum() == T24


def test_one_hot_T24_worked_example():
    p = np.zeros(V, dtype=np.float32)
    j = 12345
    p[j] = 1.0
    c = Q.probs_to_counts(p, T24)
    assert c[j] == Q.k_bins(T24, V) + 1 == 16_728_065
    assert np.all(np.delete(c, j) == 1)
    cdf = Q.probs_to_cdf(p, T24)
    bits = Q.code_length_bits(cdf, j, T24)
    assert abs(bits - 0.004233) < 1e-6          # the paper's ~0.004 bits/token


def test_T16_worked_examples():
    T = 1 << 16
    p = np.full(V, np.float32(1.0) / np.float32(V), dtype=np.float32)
    c = Q.probs_to_counts(p, T)
    assert np.all(c[1:] == 1) and c[0] == 1 + 16_384
    p = np.zeros(V, dtype=np.float32)
    p[7] = 1.0
    cdf = Q.probs_to_cdf(p, T)
    assert cdf[8] - cdf[7] == 16_385
    bits = Q.code_length_bits(cdf, 7, T)
    assert abs(bits - 2.0) < 1e-3                # the paper's ~2 bits/token


@pytest.mark.parametrize("seed", range(5))
def test_invariants_random(seed):
    rng = np.random.default_rng(seed)
    for shape_kind in ("dirichlet", "peaked", "sparse"):
        if shape_kind == "dirichlet":
            p = rng.dirichlet(np.full(V, 0.1))
        elif shape_kind == "peaked":
            z = rng.normal(0, 4, V)
            p = np.exp(z - z.max())
            p /= p.sum()
        else:
            p = np.zeros(V)
            idx = rng.choice(V, 50, replace=False)
            p[idx] = rng.random(50)
            p /= p.sum()
        p32 = p.astype(np.float32)
        cdf = Q.probs_to_cdf(p32, T24)
        c = np.diff(cdf)
        assert cdf[0] == 0 and cdf[-1] == T24
        assert np.all(c >= 1)                     # strictly monotone, floor 1
        # every non-argmax count is exactly max(1, floor(p*K)) by exact rationals
        K = Q.k_bins(T24, V)
        j = int(np.argmax(p32))
        for i in rng.choice(V, 200, replace=False):
            if i != j:
                assert c[i] == max(1, Q.floor_product_exact(p32[i], K))


def test_argmax_tie_lowest_index():
    p = np.zeros(V, dtype=np.float32)
    p[[10, 20, 30]] = np.float32(1.0 / 3.0)
    c = Q.probs_to_counts(p, T24)
    assert c[10] > c[20] == c[30]


def test_floor_product_exact_vs_float64_sampled():
    """binary64 product of a binary32 and K < 2^24 is exact: compare against
    rational arithmetic on random bit patterns and edge values in [0, 1]."""
    rng = np.random.default_rng(0)
    bits = rng.integers(0, 0x3F800001, size=20000, dtype=np.int64).astype(np.uint32)
    edge = np.array([0, 1, 2, 0x007FFFFF, 0x00800000, 0x3F7FFFFF, 0x3F800000,
                     0x33800000, 0x34000000, 0x3E800000], dtype=np.uint32)
    ps = np.concatenate([bits, edge]).view(np.float32)
    for K in (Q.k_bins(T24, V), (1 << 16) - V, 12_345_679):
        got = np.floor(ps.astype(np.float64) * K).astype(np.int64)
        for p, g in zip(ps[::7], got[::7]):
            assert g == Q.floor_product_exact(p, K)


def test_errors():
    p = np.full(V, np.float32(1.0) / np.float32(V), dtype=np.float32)
    p[3] = np.nan
    with pytest.raises(Q.QuantiseError):
        Q.probs_to_counts(p)
    # sum of binary32 probabilities far above 1 pushes argmax below the floor
    p = np.full(V, np.float32(2.0) / np.float32(V), dtype=np.float32)
    with pytest.raises(Q.QuantiseError):
        Q.probs_to_counts(p)


def test_zero_and_subnormal_get_floor():
    p = np.zeros(V, dtype=np.float32)
    p[0] = 1.0
    p[1] = np.float32(1e-45)          # smallest subnormal
    p[2] = np.float32(5e-8)           # p*K < 1
    c = Q.probs_to_counts(p, T24)
    assert c[1] == 1 and c[2] == 1 and c[3] == 1
