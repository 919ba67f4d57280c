"""Seeded synthetic inputs shared by the FP64 oracle and the CUDA path.

This module holds no arithmetic of the compression method. It only draws
random numbers and lays them out:

* model shapes of the two transformer configurations (the paper's SmolLM2-135M
  shape from Sec. 3.2, and a 4-layer small model for fast parity runs);
* random-init weights, N(0, 0.02) drawn in FP64 from PCG64 seeded by
  ``SeedSequence([seed, tensor_index])`` and rounded to FP32 (the canonical
  model), RMSNorm gains set to one;
* the flat FP32 weight buffer in the tensor order that ``nc_ctx_create``
  expects (see ``WEIGHT_ORDER``);
* token streams: Zipf(1.1) ids over the whole vocabulary with seeded
  order-2 Markov structure, standing in for tokenised text (the paper's
  alice29 / enwik8 / OOD texts are not available here);
* stream lengths, log-uniform between two bounds;
* a bytes-per-token convention for reporting bits per byte on synthetic ids.
"""
from __future__ import annotations

import functools
from dataclasses import dataclass, asdict

import numpy as np

MASK64 = (1 << 64) - 1


@dataclass(frozen=True)
class ModelShape:
    """Decoder-only transformer shape (Sec. 3.2; dimensions as stated for the
    two model sizes).  ``ctx_len``/``slide`` are the sliding KV window L and
    drop count C of Sec. 3.9."""
    n_layers: int
    d_model: int
    n_heads: int
    n_kv_heads: int
    d_ffn: int
    vocab: int
    ctx_len: int
    slide: int
    rope_theta: float = 1e5
    rms_eps: float = 1e-5

    @property
    def d_head(self) -> int:
        return self.d_model // self.n_heads

    def as_dict(self):
        return asdict(self)


# SmolLM2-135M shape: 30 layers, hidden 576, 9 query / 3 KV heads, FFN 1536,
# tied 49,152-token embedding, 2,048-token window sliding by 512.
FULL = ModelShape(n_layers=30, d_model=576, n_heads=9, n_kv_heads=3, d_ffn=1536,
                  vocab=49152, ctx_len=2048, slide=512)
# Small model: 4 layers, hidden 256, 4 query / 2 KV heads, FFN 688; window 512
# sliding by 128 (same ratio as the full model).
SMALL = ModelShape(n_layers=4, d_model=256, n_heads=4, n_kv_heads=2, d_ffn=688,
                   vocab=49152, ctx_len=512, slide=128)


def tensor_specs(s: ModelShape):
    """Canonical tensor order: (name, shape, is_norm_gain).  Index in this list
    is the ``tensor_index`` of the seed sequence and the order of the flat
    buffer.  Matrices are [out, in], row-major."""
    qd = s.n_heads * s.d_head
    kvd = s.n_kv_heads * s.d_head
    specs = [("embed", (s.vocab, s.d_model), False)]
    for l in range(s.n_layers):
        specs += [
            (f"l{l}.attn_norm", (s.d_model,), True),
            (f"l{l}.wq", (qd, s.d_model), False),
            (f"l{l}.wk", (kvd, s.d_model), False),
            (f"l{l}.wv", (kvd, s.d_model), False),
            (f"l{l}.wo", (s.d_model, qd), False),
            (f"l{l}.ffn_norm", (s.d_model,), True),
            (f"l{l}.w_gate", (s.d_ffn, s.d_model), False),
            (f"l{l}.w_up", (s.d_ffn, s.d_model), False),
            (f"l{l}.w_down", (s.d_model, s.d_ffn), False),
        ]
    specs.append(("final_norm", (s.d_model,), True))
    return specs


WEIGHT_ORDER = "embed, then per layer: attn_norm wq wk wv wo ffn_norm w_gate w_up w_down, then final_norm"


def n_params(s: ModelShape) -> int:
    return sum(int(np.prod(shape)) for _, shape, _ in tensor_specs(s))


def _tensor_rng(seed: int, idx: int) -> np.random.Generator:
    return np.random.Generator(np.random.PCG64(np.random.SeedSequence([seed, idx])))


@functools.lru_cache(maxsize=4)
def weights(s: ModelShape, seed: int, std: float = 0.02):
    """Random-init FP32 weights as a dict name -> float32 array (read-only)."""
    out = {}
    for idx, (name, shape, is_gain) in enumerate(tensor_specs(s)):
        if is_gain:
            w = np.ones(shape, dtype=np.float32)
        else:
            w = _tensor_rng(seed, idx).normal(0.0, std, size=shape).astype(np.float32)
        w.setflags(write=False)
        out[name] = w
    return out


@functools.lru_cache(maxsize=4)
def flat_weights(s: ModelShape, seed: int) -> np.ndarray:
    """The flat little-endian FP32 buffer in ``tensor_specs`` order."""
    w = weights(s, seed)
    flat = np.concatenate([w[name].reshape(-1) for name, _, _ in tensor_specs(s)])
    flat.setflags(write=False)
    return flat


# ---------------------------------------------------------------- token streams

def splitmix64(x: int) -> int:
    """SplitMix64 finaliser (Steele, Lea, Flood 2014), used only as a seeded
    hash for the synthetic stream generator."""
    x = (x + 0x9E3779B97F4A7C15) & MASK64
    z = x
    z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & MASK64
    z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & MASK64
    return z ^ (z >> 31)


@functools.lru_cache(maxsize=8)
def _zipf_cdf(vocab: int, s: float) -> np.ndarray:
    ranks = np.arange(1, vocab + 1, dtype=np.float64)
    w = ranks ** (-s)
    c = np.cumsum(w)
    return c / c[-1]


@functools.lru_cache(maxsize=8)
def _rank_to_id(seed: int, vocab: int) -> np.ndarray:
    return _tensor_rng(seed, 0x5EED_0001).permutation(vocab).astype(np.int32)


SUCCESSOR_PROBS = (0.6, 0.25, 0.1, 0.05)


def token_stream(seed: int, stream_idx: int, n: int, vocab: int, zipf_s: float = 1.1,
                 beta: float = 0.5) -> np.ndarray:
    """One synthetic token stream of length ``n`` (int32 ids in [0, vocab)).

    With probability ``beta`` (and once two tokens exist) the next id is one
    of four successors of the context (t[i-2], t[i-1]); the successors are
    Zipf draws keyed by a hash of (seed, context) and are picked with
    probabilities SUCCESSOR_PROBS.  Otherwise the id is an i.i.d. Zipf draw.
    Zipf ranks map to ids through a seeded permutation.
    """
    cdf = _zipf_cdf(vocab, zipf_s)
    perm = _rank_to_id(seed, vocab)
    rng = _tensor_rng(seed, 0x57EA_0000 + stream_idx)
    iid = perm[np.minimum(np.searchsorted(cdf, rng.random(n), side="right"), vocab - 1)]
    u_branch = rng.random(n)
    u_pick = rng.random(n)
    pick_cdf = np.cumsum(SUCCESSOR_PROBS)
    out = np.empty(n, dtype=np.int32)
    succ_cache = {}
    seed_h = splitmix64(seed & MASK64)
    for i in range(n):
        if i >= 2 and u_branch[i] < beta:
            key = (int(out[i - 2]) << 20) | int(out[i - 1])
            succ = succ_cache.get(key)
            if succ is None:
                h = splitmix64(seed_h ^ key)
                succ = []
                for _ in range(4):
                    h = splitmix64(h)
                    u = (h >> 11) * (1.0 / (1 << 53))
                    r = min(int(np.searchsorted(cdf, u, side="right")), vocab - 1)
                    succ.append(int(perm[r]))
                succ_cache[key] = succ
            j = min(int(np.searchsorted(pick_cdf, u_pick[i], side="right")), 3)
            out[i] = succ[j]
        else:
            out[i] = iid[i]
    return out


def stream_lengths(seed: int, n_streams: int, lo: int, hi: int) -> np.ndarray:
    """Log-uniform integer lengths in [lo, hi]."""
    rng = _tensor_rng(seed, 0x1E46_0000)
    x = np.exp(rng.uniform(np.log(lo), np.log(hi + 1), size=n_streams))
    return np.clip(np.floor(x).astype(np.int64), lo, hi)


def streams(seed: int, n_streams: int, lengths, vocab: int):
    return [token_stream(seed, j, int(lengths[j]), vocab) for j in range(n_streams)]


def bytes_per_token(tokens) -> np.ndarray:
    """Synthetic ids carry no text; each id is assigned 1 + (splitmix64(id) mod 7)
    bytes (mean 4.0, within the 3-5 bytes/token of English BPE text)."""
    return np.array([1 + splitmix64(int(t)) % 7 for t in np.asarray(tokens).reshape(-1)],
                    dtype=np.int64)


def n_bytes(tokens) -> int:
    return int(bytes_per_token(tokens).sum())
