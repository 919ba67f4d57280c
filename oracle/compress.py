"""The compression loop of Algorithm 1 and its mirror-image decompression.

Per stream, for i = 1..n (Algorithm 1):
    z       = LLM(t_1..t_{i-1})      (BOS at position 0 feeds the first step)
    p_llm   = softmax(z / tau)                        (Sec. 3.2)
    p_tilde = softmax(log p_llm + b)                  (Sec. 3.6)
    p_ng    = N-gram prediction                        (Sec. 3.4)
    p       = p_ng when the confidence skip is on and H(p_ng) < 1.5 bits
              (Sec. 3.7, Algorithm 1); else p_tilde during warm-up
              (i <= 100), else w_llm p_tilde + w_ng p_ng (Sec. 3.5)
    cdf     = probs_to_cdf(binary32(p), 2^24)          (Sec. 3.3)
    encode t_i; then update head, mixer and N-gram with t_i (a skipped token
    updates the N-gram only: the LLM produced no distribution for the head
    and the mixer to learn from).
The LLM step still runs on a skipped token, so that the KV cache holds every
token (the paper evaluates skipped tokens later, in a batch; the cache is the
same).
The order "head acts on the LLM distribution, then the mix, then the
quantiser" follows the ablation's build-up (CDF-24, then head, then N-gram).

Update rules: 'paper' (head: b -= alpha (p_tilde - e); mixer: exponential
weights) or 'mixed_nll' (one SGD step of -log p_mix(t*) in b and the mixer
log-weights, both with rate alpha).
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np

from . import cdf as cdfmod
from . import container
from . import ans
from .coder import Decoder, Encoder
from .head import BiasHead, p_llm as llm_softmax
from .mixer import Mixer, mixed_nll_grad
from .ngram import NGram


@dataclass
class StepConfig:
    cdf_log2_total: int = 24
    floor: int = 1
    tau: float = 1.0
    alpha: float = 1e-3
    eta: float = 1.0
    w_llm: float = 0.85
    warmup: int = 100
    order: int = 3
    use_ngram: bool = True
    use_head: bool = True
    rule: str = "paper"          # or "mixed_nll"
    skip: bool = False           # confidence-based LLM skip (Sec. 3.7)
    coder: str = "arith"         # or "rans" (the ANS coder of Sec. 6)

    @property
    def T(self) -> int:
        return 1 << self.cdf_log2_total

    def flags(self) -> int:
        f = 0
        if self.use_ngram:
            f |= container.FLAG_NGRAM
        if self.use_head:
            f |= container.FLAG_HEAD
        if self.rule == "mixed_nll":
            f |= container.FLAG_MIXED_NLL
        if self.skip:
            f |= container.FLAG_SKIP
        if self.coder == "rans":
            f |= container.FLAG_RANS
        return f


SKIP_BITS = 1.5                   # the skip threshold on H(p_ng) in bits (Sec. 3.7)


def entropy_bits(p: np.ndarray) -> float:
    """Shannon entropy -sum p log2 p in bits, with 0 log 0 = 0."""
    q = p[p > 0]
    return float(-np.sum(q * np.log2(q)))


@dataclass
class StreamState:
    cfg: StepConfig
    model: object
    V: int
    cache: object = None
    head: BiasHead = None
    mixer: Mixer = None
    ngram: NGram = None
    theta: np.ndarray = None          # mixer log-weights under the mixed-NLL rule
    i: int = 0                        # tokens coded so far
    last: int = 0                     # token fed at the next step (BOS first)
    ideal_bits: float = 0.0
    skipped: int = 0                  # tokens coded by the N-gram alone
    records: list = field(default_factory=list)

    @classmethod
    def new(cls, model, cfg: StepConfig):
        V = model.s.vocab
        st = cls(cfg=cfg, model=model, V=V)
        st.cache = model.new_cache()
        st.head = BiasHead(V, cfg.alpha)
        st.mixer = Mixer(2, cfg.w_llm, cfg.eta, cfg.warmup)
        st.ngram = NGram(V, cfg.order)
        st.theta = st.mixer.logw.copy()
        st.last = model.BOS
        return st

    # ---------------------------------------------------------------- one step
    def predict(self, record: bool = False):
        """Distribution for token i+1: returns (p float64, p32, cdf)."""
        cfg = self.cfg
        i = self.i + 1
        z = self.model.step(self.cache, self.last)
        pl = llm_softmax(z, cfg.tau)
        pt = self.head.adjust(pl) if cfg.use_head else pl
        png = self.ngram.predict() if cfg.use_ngram else None
        self._skip = bool(cfg.skip and cfg.use_ngram and entropy_bits(png) < SKIP_BITS)
        if self._skip:
            p = png
        elif cfg.use_ngram and i > cfg.warmup:
            if cfg.rule == "mixed_nll":
                w = np.exp(self.theta - self.theta.max())
                w /= w.sum()
            else:
                w = self.mixer.weights()
            p = w[0] * pt + w[1] * png
        else:
            p = pt
        p32 = p.astype(np.float32)
        cdf = cdfmod.probs_to_cdf(p32, cfg.T, cfg.floor)
        self._cur = (z, pt, png, p)
        if record:
            self.records.append(dict(i=i, z=z, p_tilde=pt, p_ng=png, p=p, p32=p32, cdf=cdf))
        return p, p32, cdf

    def update(self, t: int):
        cfg = self.cfg
        z, pt, png, p = self._cur
        i = self.i + 1
        self.ideal_bits += -np.log2(p[t])
        warm = i <= cfg.warmup or not cfg.use_ngram
        if self._skip:
            self.skipped += 1
        elif cfg.rule == "mixed_nll":
            gb, gth = mixed_nll_grad(pt, png if png is not None else pt, self.theta, t, warm)
            if cfg.use_head:
                self.head.b -= cfg.alpha * gb
            self.theta = self.theta - cfg.alpha * gth
        else:
            if cfg.use_head:
                self.head.update(pt, t)
            if cfg.use_ngram:
                self.mixer.update([pt[t], png[t]], i)
        if cfg.use_ngram:
            self.ngram.update(t)
        self.i = i
        self.last = int(t)


def compress_stream(model, tokens, cfg: StepConfig, record_steps: int = 0):
    st = StreamState.new(model, cfg)
    enc = Encoder(cfg.T)
    intervals = []
    for k, t in enumerate(np.asarray(tokens)):
        _, _, cdf = st.predict(record=k < record_steps)
        intervals.append((int(cdf[int(t)]), int(cdf[int(t) + 1])))
        enc.encode(cdf, int(t))
        st.update(int(t))
    payload, nbits = enc.finish()
    if cfg.coder == "rans":                       # the same intervals, coded in reverse by rANS
        payload = ans.encode(intervals, cfg.cdf_log2_total)
        nbits = 8 * len(payload)
    return dict(payload=payload, nbits=nbits, ideal_bits=st.ideal_bits,
                records=st.records, min_range=enc.min_range, slides=st.cache.slides, skipped=st.skipped)


def decompress_stream(model, payload: bytes, nbits: int, n: int, cfg: StepConfig):
    st = StreamState.new(model, cfg)
    dec = ans.Decoder(payload, cfg.cdf_log2_total) if cfg.coder == "rans" else Decoder(payload, nbits, cfg.T)
    out = np.empty(n, dtype=np.int32)
    for k in range(n):
        _, _, cdf = st.predict()
        t = dec.decode(cdf)
        out[k] = t
        st.update(t)
    return out


def compress(model, streams, cfg: StepConfig, path_byte: int = 0) -> bytes:
    recs, pays = [], []
    for toks in streams:
        r = compress_stream(model, toks, cfg)
        recs.append((len(toks), r["nbits"], len(r["payload"])))
        pays.append(r["payload"])
    return container.pack(cfg.flags(), cfg.tau, path_byte, recs, pays)


def decompress(model, buf: bytes, cfg: StepConfig):
    flags, tau, _, recs, pays = container.unpack(buf)
    if flags != cfg.flags() or np.float16(tau) != np.float16(cfg.tau):
        raise container.ContainerError("container features differ from the configuration")
    return [decompress_stream(model, p, nbits, ntok, cfg)
            for (ntok, nbits, _), p in zip(recs, pays)]
