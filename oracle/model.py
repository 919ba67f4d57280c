"""FP64 decoder-only transformer decode step with a sliding KV window.

Follows Sec. 3.2 (Eq. lm: next-token distribution = softmax of the tied
output projection of the last hidden state) and Sec. 3.9 (sliding KV window).
The paper fixes only the family (a 30-layer causal transformer with a 49,152
token vocabulary); the block is the standard pre-norm Llama/SmolLM2 block:

    x  = E[t]
    per layer:
        a  = RMSNorm(x) * g_attn
        q, k, v = Wq a, Wk a, Wv a          (per head, d_head = 64)
        q, k rotated by RoPE (rotate-half pairing (j, j + d_head/2),
             inverse frequency theta^(-2j/d_head)) at their positions
        o  = softmax(q k^T / sqrt(d_head)) v, each KV head shared by
             n_heads / n_kv_heads query heads (grouped-query attention)
        x += Wo o
        f  = RMSNorm(x) * g_ffn
        x += Wdown (silu(Wgate f) * (Wup f))
    z = E (RMSNorm(x) * g_final)            (tied head, no output bias)

Sliding window (Sec. 3.9): the cache holds at most L entries.  Before a new
entry is appended to a full cache the oldest C entries are removed and the
remaining ones are relabelled to positions 0..L-C-1; the new token then sits
at position L-C.  Cached values keep the content they were computed with;
cached keys are stored unrotated and rotated at their current position, which
is the same as re-rotating the shifted keys.  The first model input is a BOS
id 0 at position 0.
"""
from __future__ import annotations

import numpy as np

from synthetic import ModelShape, tensor_specs
from . import numerics


def dequantised_weights(shape: ModelShape, w32: dict, fmt: str) -> dict:
    """FP64 copies of the weights as a given storage format represents them:
    'fp32' (canonical), 'bf16' (RNE) or 'fp8' (E4M3, per-output-channel scale).
    Norm gains always stay FP32."""
    out = {}
    for name, _, is_gain in tensor_specs(shape):
        w = w32[name]
        if is_gain or fmt == "fp32":
            out[name] = np.asarray(w, dtype=np.float64)
        elif fmt == "bf16":
            out[name] = numerics.bf16_round(w).astype(np.float64)
        elif fmt == "fp8":
            out[name] = numerics.fp8_dequant(w)
        else:
            raise ValueError(fmt)
    return out


def rms_norm(x, g, eps):
    return x / np.sqrt(np.mean(x * x) + eps) * g


def silu(a):
    return a / (1.0 + np.exp(-a))


def rope_inv_freq(d_head: int, theta: float) -> np.ndarray:
    j = np.arange(d_head // 2, dtype=np.float64)
    return theta ** (-2.0 * j / d_head)


def rope_tables(n_pos: int, inv_freq):
    """cos / sin of position * inverse frequency for positions 0..n_pos-1."""
    ang = np.multiply.outer(np.arange(n_pos, dtype=np.float64), inv_freq)
    return np.cos(ang), np.sin(ang)


def rope(x, c, s):
    """Rotate-half RoPE of x[..., d_head] given cos/sin broadcastable to
    x[..., :d_head/2]: (x1, x2) -> (x1 cos - x2 sin, x2 cos + x1 sin)."""
    half = x.shape[-1] // 2
    x1, x2 = x[..., :half], x[..., half:]
    return np.concatenate([x1 * c - x2 * s, x2 * c + x1 * s], axis=-1)


class KVWindow:
    """Per-stream cache: unrotated keys and values, [layers, L, kv_heads, d_head]."""

    def __init__(self, shape: ModelShape):
        s = shape
        self.shape = s
        self.k = np.zeros((s.n_layers, s.ctx_len, s.n_kv_heads, s.d_head))
        self.v = np.zeros_like(self.k)
        self.n = 0          # entries held; the next token's position is n
        self.slides = 0

    def make_room(self):
        """Drop the oldest C entries of a full cache and relabel the rest."""
        s = self.shape
        if self.n == s.ctx_len:
            keep = s.ctx_len - s.slide
            self.k[:, :keep] = self.k[:, s.slide:].copy()
            self.v[:, :keep] = self.v[:, s.slide:].copy()
            self.n = keep
            self.slides += 1


class Model:
    """FP64 evaluation of the decode step on a given weight set."""

    BOS = 0

    def __init__(self, shape: ModelShape, w32: dict, fmt: str = "fp32"):
        self.s = shape
        self.w = dequantised_weights(shape, w32, fmt)
        self.inv_freq = rope_inv_freq(shape.d_head, shape.rope_theta)
        self.cos, self.sin = rope_tables(shape.ctx_len, self.inv_freq)

    def new_cache(self) -> KVWindow:
        return KVWindow(self.s)

    def attend(self, q, k_raw, v):
        """Grouped-query attention of the newest token (position n-1) over the
        n cached entries at positions 0..n-1; q [hq, dh], k_raw/v [n, hkv, dh]."""
        s = self.s
        n = k_raw.shape[0]
        group = s.n_heads // s.n_kv_heads
        qr = rope(q, self.cos[n - 1], self.sin[n - 1])                  # [hq, dh]
        kr = rope(k_raw, self.cos[:n, None], self.sin[:n, None])        # [n, hkv, dh]
        o = np.empty((s.n_heads, s.d_head))
        for h in range(s.n_heads):
            g = h // group
            sc = kr[:, g, :] @ qr[h] / np.sqrt(s.d_head)
            e = np.exp(sc - sc.max())
            o[h] = (e / e.sum()) @ v[:, g, :]
        return o

    def step(self, cache: KVWindow, token: int) -> np.ndarray:
        """Feed one token, append its K/V, return logits z (float64[V])."""
        s, w = self.s, self.w
        dh, hq, hkv = s.d_head, s.n_heads, s.n_kv_heads
        cache.make_room()
        pos = cache.n
        x = w["embed"][token].copy()
        for l in range(s.n_layers):
            p = f"l{l}."
            a = rms_norm(x, w[p + "attn_norm"], s.rms_eps)
            q = (w[p + "wq"] @ a).reshape(hq, dh)
            k = (w[p + "wk"] @ a).reshape(hkv, dh)
            v = (w[p + "wv"] @ a).reshape(hkv, dh)
            cache.k[l, pos] = k
            cache.v[l, pos] = v
            n = pos + 1
            o = self.attend(q, cache.k[l, :n], cache.v[l, :n])
            x = x + w[p + "wo"] @ o.reshape(-1)
            f = rms_norm(x, w[p + "ffn_norm"], s.rms_eps)
            x = x + w[p + "w_down"] @ (silu(w[p + "w_gate"] @ f) * (w[p + "w_up"] @ f))
        cache.n = pos + 1
        hN = rms_norm(x, w["final_norm"], s.rms_eps)
        return w["embed"] @ hN
