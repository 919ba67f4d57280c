"""Reduced-precision weight formats, written from the format definitions.

* bfloat16: the top 16 bits of an IEEE binary32, rounded to nearest, ties to
  even (RNE) on the dropped 16 bits.
* FP8 E4M3 (OCP 8-bit floating point, "E4M3FN"): 1 sign, 4 exponent (bias 7),
  3 mantissa bits, no infinities, largest finite 448, subnormal step 2^-9.
  Conversion rounds to nearest even and saturates to +-448.
* Per-output-channel scaling: scale_r = fp32(amax_r / 448) (IEEE division in
  binary32), q = e4m3(fp32(w / scale_r)), dequantised weight = q * scale_r.
  An all-zero row uses scale 1.

These are the weight variants the GPU path stores; the oracle evaluates the
model in FP64 on the dequantised values so that weight rounding and compute
error can be told apart.
"""
from __future__ import annotations

import numpy as np


def bf16_round(x) -> np.ndarray:
    """Round float32 values to bfloat16 (RNE) and return them as float32."""
    x = np.ascontiguousarray(x, dtype=np.float32)
    u = x.view(np.uint32).astype(np.uint64)
    lsb = (u >> 16) & 1
    r = (u + 0x7FFF + lsb) >> 16
    out = (r << 16).astype(np.uint32).view(np.float32)
    nan = np.isnan(x)
    if nan.any():
        out = out.copy()
        out[nan] = np.nan
    return out


def _e4m3_grid() -> np.ndarray:
    """All non-negative finite E4M3 values in increasing order (codes 0..126)."""
    vals = []
    for code in range(0x7F):  # 0x7F is NaN in E4M3FN
        e = code >> 3
        m = code & 7
        if e == 0:
            v = m * 2.0 ** -9
        else:
            v = (1 + m / 8.0) * 2.0 ** (e - 7)
        vals.append(v)
    return np.array(vals, dtype=np.float64)


_GRID = _e4m3_grid()


def e4m3_round(x) -> np.ndarray:
    """Round to the nearest E4M3 value (ties to the even code), saturating at
    +-448.  Input float32/float64, output float64 holding exact E4M3 values."""
    x = np.asarray(x, dtype=np.float64)
    a = np.minimum(np.abs(x), 448.0)
    hi = np.searchsorted(_GRID, a, side="left")
    hi = np.minimum(hi, len(_GRID) - 1)
    lo = np.maximum(hi - 1, 0)
    vlo, vhi = _GRID[lo], _GRID[hi]
    dlo, dhi = a - vlo, vhi - a
    pick_hi = (dhi < dlo) | ((dhi == dlo) & (hi % 2 == 0))
    exact = vhi == a
    code = np.where(exact | pick_hi, hi, lo)
    return np.sign(x) * _GRID[code]


def fp8_rowwise(w):
    """Per-output-channel E4M3 quantisation of a [out, in] FP32 matrix.
    Returns (q as float64 E4M3 values, scale float32 [out])."""
    w = np.asarray(w, dtype=np.float32)
    amax = np.max(np.abs(w), axis=1).astype(np.float32)
    scale = (amax / np.float32(448.0)).astype(np.float32)
    scale = np.where(amax > 0, scale, np.float32(1.0)).astype(np.float32)
    ratio = (w / scale[:, None]).astype(np.float32)
    return e4m3_round(ratio), scale


def fp8_dequant(w) -> np.ndarray:
    q, scale = fp8_rowwise(w)
    return q * scale.astype(np.float64)[:, None]
