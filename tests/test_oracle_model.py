"""Pins for the oracle's transformer decode step (Sec. 3.2, Sec. 3.9):
RoPE against the complex-exponential form, attention special cases, the
zero-weight residual identity, and the step-by-step cached decode against an
independent full causal forward written with torch.float64 library ops."""
import numpy as np
import pytest
import torch

import synthetic as S
from oracle import numerics
from oracle.model import Model, rope, rope_inv_freq, rope_tables

TINY = S.ModelShape(n_layers=2, d_model=32, n_heads=4, n_kv_heads=2, d_ffn=48,
                    vocab=97, ctx_len=16, slide=4)


def test_rope_complex_form_and_position_zero():
    rng = np.random.default_rng(0)
    dh = 64
    inv = rope_inv_freq(dh, 1e5)
    c, s = rope_tables(50, inv)
    x = rng.normal(size=dh)
    for pos in (0, 1, 7, 49):
        got = rope(x, c[pos], s[pos])
        zc = (x[:32] + 1j * x[32:]) * np.exp(1j * pos * inv)
        np.testing.assert_allclose(got, np.concatenate([zc.real, zc.imag]), rtol=1e-13, atol=1e-13)
    np.testing.assert_array_equal(rope(x, c[0], s[0]), x)
    # relative-position property: <R(m)q, R(n)k> depends only on m - n
    q, k = rng.normal(size=dh), rng.normal(size=dh)
    a = rope(q, c[10], s[10]) @ rope(k, c[3], s[3])
    b = rope(q, c[27], s[27]) @ rope(k, c[20], s[20])
    assert abs(a - b) < 1e-12
    assert inv[0] == 1.0 and abs(inv[-1] - 1e5 ** (-62 / 64)) < 1e-18


def test_attention_single_entry_returns_v():
    w = S.weights(TINY, 3)
    m = Model(TINY, w)
    rng = np.random.default_rng(1)
    q = rng.normal(size=(4, 8))
    k = rng.normal(size=(1, 2, 8))
    v = rng.normal(size=(1, 2, 8))
    o = m.attend(q, k, v)
    np.testing.assert_allclose(o, v[0][[0, 0, 1, 1]], rtol=1e-15)


def test_zero_weights_identity_residual():
    w = dict(S.weights(TINY, 3))
    for name, _, is_gain in S.tensor_specs(TINY):
        if name != "embed" and not is_gain:
            w[name] = np.zeros_like(w[name])
    m = Model(TINY, w)
    cache = m.new_cache()
    E = w["embed"].astype(np.float64)
    for t in (5, 9, 11):
        z = m.step(cache, t)
        x = E[t]
        np.testing.assert_allclose(z, E @ (x / np.sqrt(np.mean(x * x) + TINY.rms_eps)), rtol=1e-13)


def torch_full_forward(shape, w, tokens):
    """Independent FP64 restatement: the whole causal sequence at once with
    torch ops (scaled_dot_product_attention, repeat_interleave for GQA,
    complex-multiplication RoPE); returns logits at every position."""
    s = shape
    T = len(tokens)
    dh = s.d_head
    W = {k: torch.tensor(np.asarray(v, dtype=np.float64)) for k, v in w.items()}
    x = W["embed"][torch.tensor(tokens)]
    inv = s.rope_theta ** (-torch.arange(0, dh, 2, dtype=torch.float64) / dh)
    rot = torch.polar(torch.ones(T, dh // 2, dtype=torch.float64),
                      torch.arange(T, dtype=torch.float64)[:, None] * inv[None])

    def rms(v, g):
        return v * torch.rsqrt((v * v).mean(-1, keepdim=True) + s.rms_eps) * g

    def rope_c(v):  # [T, H, dh]
        vc = torch.complex(v[..., : dh // 2], v[..., dh // 2:]) * rot[:, None, :]
        return torch.cat([vc.real, vc.imag], -1)

    for l in range(s.n_layers):
        p = f"l{l}."
        a = rms(x, W[p + "attn_norm"])
        q = rope_c((a @ W[p + "wq"].T).view(T, s.n_heads, dh))
        k = rope_c((a @ W[p + "wk"].T).view(T, s.n_kv_heads, dh))
        v = (a @ W[p + "wv"].T).view(T, s.n_kv_heads, dh)
        rep = s.n_heads // s.n_kv_heads
        k = k.repeat_interleave(rep, dim=1)
        v = v.repeat_interleave(rep, dim=1)
        o = torch.nn.functional.scaled_dot_product_attention(
            q.transpose(0, 1), k.transpose(0, 1), v.transpose(0, 1), is_causal=True)
        x = x + o.transpose(0, 1).reshape(T, -1) @ W[p + "wo"].T
        f = rms(x, W[p + "ffn_norm"])
        x = x + (torch.nn.functional.silu(f @ W[p + "w_gate"].T) * (f @ W[p + "w_up"].T)) @ W[p + "w_down"].T
    return (rms(x, W["final_norm"]) @ W["embed"].T).numpy()


@pytest.mark.parametrize("fmt", ["fp32", "bf16"])
def test_cached_decode_matches_full_causal_forward(fmt):
    w = S.weights(TINY, 5)
    m = Model(TINY, w, fmt)
    seq = [0] + list(S.token_stream(5, 0, TINY.ctx_len - 1, TINY.vocab))  # BOS + tokens, fills L
    ref = torch_full_forward(TINY, m.w, seq)
    cache = m.new_cache()
    for i, t in enumerate(seq):
        z = m.step(cache, t)
        np.testing.assert_allclose(z, ref[i], rtol=1e-10, atol=1e-12)


def test_slide_keeps_window_and_relabels():
    w = S.weights(TINY, 6)
    m = Model(TINY, w)
    cache = m.new_cache()
    toks = list(S.token_stream(6, 1, 40, TINY.vocab))
    ns = []
    for t in toks:
        m.step(cache, t)
        ns.append(cache.n)
    L, C = TINY.ctx_len, TINY.slide
    # fills to L, then drops C before the next append: L-C+1, ..., L, L-C+1, ...
    assert ns[:L] == list(range(1, L + 1))
    assert ns[L] == L - C + 1
    assert max(ns) == L and cache.slides == (40 - L) // C + (1 if (40 - L) % C else 0)


def test_slide_relabelling_equals_absolute_rotation():
    """Across slides the oracle rotates the query and the cached keys at their
    relabelled positions.  Attention computed instead at the tokens' absolute
    positions, with an independent complex-exponential rotation and no
    relabelling, gives the same output (RoPE scores depend only on position
    differences): the window slide is a start bump for an absolute-position
    cache, which is what the GPU's ring buffer does (Sec. 3.9)."""
    w = S.weights(TINY, 11)
    m = Model(TINY, w)
    dh, hq, hkv = TINY.d_head, TINY.n_heads, TINY.n_kv_heads
    inv = TINY.rope_theta ** (-2.0 * np.arange(dh // 2) / dh)

    def rot(x, pos):                                  # x [..., dh] at absolute positions pos
        z = (x[..., : dh // 2] + 1j * x[..., dh // 2:]) * np.exp(1j * np.multiply.outer(pos, inv))
        return np.concatenate([z.real, z.imag], axis=-1)

    state = {"abs": 0, "checked": 0}
    orig = m.attend

    def attend(q, k_raw, v):
        out = orig(q, k_raw, v)
        n, a = k_raw.shape[0], state["abs"]
        pos = np.arange(a - n + 1, a + 1, dtype=np.float64)     # absolute positions of the window
        qa = rot(q, np.full(hq, float(a)))
        ka = rot(k_raw, pos[:, None] * np.ones((1, hkv)))
        o = np.empty_like(out)
        for h in range(hq):
            g = h // (hq // hkv)
            sc = ka[:, g, :] @ qa[h] / np.sqrt(dh)
            e = np.exp(sc - sc.max())
            o[h] = (e / e.sum()) @ v[:, g, :]
        np.testing.assert_allclose(out, o, rtol=1e-9, atol=1e-12)
        state["checked"] += 1
        return out

    m.attend = attend
    cache = m.new_cache()
    toks = [0] + list(S.token_stream(11, 2, 60, TINY.vocab))
    for i, t in enumerate(toks):
        state["abs"] = i
        m.step(cache, t)
    assert cache.slides >= 10 and state["checked"] == len(toks) * TINY.n_layers


def test_dequantised_formats():
    w = S.weights(TINY, 7)
    b = Model(TINY, w, "bf16").w["l0.wq"]
    assert np.all(numerics.bf16_round(b.astype(np.float32)) == b.astype(np.float32))
    f = Model(TINY, w, "fp8").w["l0.wq"]
    rel = np.abs(f - w["l0.wq"]) / np.max(np.abs(w["l0.wq"]), axis=1, keepdims=True)
    assert rel.max() <= 2.0 ** -4 * 1.0001 * 448 / 256     # half an E4M3 step at the top binade
