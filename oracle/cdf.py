"""CDF quantisation with per-symbol floors (Sec. 3.3), exact integers.

    K   = T - V * floor           (T = 2^24 and floor 1 give K = 16,728,064;
                                   the paper prints 16,727,064, a slip)
    c_i = max(floor, floor_int(p_i * K))
    r   = T - sum_i c_i  is added to c_j, j = argmax_i p_i (lowest index on ties)
    cdf[0] = 0, cdf[i + 1] = cdf[i] + c_i, so cdf[V] = T.

The probabilities handed to the quantiser are binary32 values (the contract
with the GPU path).  A binary32 has a 24-bit significand and K < 2^24, so
p_i * K has at most 48 significant bits and is exact in binary64; the floor of
an exact product is exact.  ``probs_to_counts_fraction`` redoes the product
with Python rationals for the exhaustive checks.

Errors: a NaN/inf probability, or a residual that would push c_j below the
floor (only possible when the binary32 probabilities sum to more than 1),
raise ``QuantiseError``.
"""
from __future__ import annotations

from fractions import Fraction

import numpy as np


class QuantiseError(ValueError):
    pass


def k_bins(T: int, V: int, floor: int = 1) -> int:
    return T - V * floor


def floor_counts(p32, K: int, floor: int = 1) -> np.ndarray:
    """max(floor, floor(p * K)) elementwise for binary32 p in [0, 2)."""
    p = np.asarray(p32, dtype=np.float32)
    return np.maximum(np.floor(p.astype(np.float64) * float(K)), floor).astype(np.int64)


def probs_to_counts(p32, T: int = 1 << 24, floor: int = 1) -> np.ndarray:
    p = np.asarray(p32, dtype=np.float32)
    if not np.all(np.isfinite(p)):
        raise QuantiseError("non-finite probability")
    V = p.shape[0]
    K = k_bins(T, V, floor)
    if K <= 0:
        raise QuantiseError("total too small for the floors")
    c = floor_counts(p, K, floor)               # exact: <= 48 significant bits
    j = int(np.argmax(p))                       # numpy argmax: first maximum
    r = T - int(c.sum())
    if c[j] + r < floor:
        raise QuantiseError("residual underflows the floor at argmax")
    c[j] += r
    return c


def probs_to_cdf(p32, T: int = 1 << 24, floor: int = 1) -> np.ndarray:
    c = probs_to_counts(p32, T, floor)
    cdf = np.zeros(c.shape[0] + 1, dtype=np.int64)
    np.cumsum(c, out=cdf[1:])
    return cdf


def floor_product_exact(p32_scalar, K: int) -> int:
    """floor(p * K) with the binary32 value taken as an exact rational."""
    return int(Fraction(float(np.float32(p32_scalar))) * K // 1)


def code_length_bits(cdf, s: int, T: int) -> float:
    return -np.log2((int(cdf[s + 1]) - int(cdf[s])) / T)
