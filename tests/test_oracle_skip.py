"""Pins for the confidence-based LLM skip (Sec. 3.7, Algorithm 1): a token
whose N-gram distribution has Shannon entropy below 1.5 bits is coded with
p = p_ng; only the N-gram learns from it."""
import math

import numpy as np
import pytest

import synthetic as S
from oracle.compress import SKIP_BITS, StepConfig, StreamState, compress, compress_stream, decompress, \
    decompress_stream, entropy_bits
from oracle import container
from oracle.model import Model

TINY = S.ModelShape(n_layers=2, d_model=32, n_heads=4, n_kv_heads=2, d_ffn=48,
                    vocab=97, ctx_len=16, slide=4)


def test_entropy_closed_forms():
    assert entropy_bits(np.full(97, 1 / 97)) == pytest.approx(math.log2(97), abs=1e-12)
    assert entropy_bits(np.array([0.5, 0.5])) == pytest.approx(1.0, abs=1e-15)
    assert entropy_bits(np.array([0.25] * 4)) == pytest.approx(2.0, abs=1e-15)
    one_hot = np.zeros(10)
    one_hot[3] = 1.0
    assert entropy_bits(one_hot) == 0.0
    # (1/2, 1/4, 1/8, 1/8): 1/2 + 2/4 + 3/8 + 3/8 = 1.75 bits
    assert entropy_bits(np.array([0.5, 0.25, 0.125, 0.125])) == pytest.approx(1.75, abs=1e-15)
    assert SKIP_BITS == 1.5


def periodic(period, reps, vocab, seed):
    base = np.random.default_rng(seed).choice(vocab, size=period, replace=False)
    return np.tile(base, reps).astype(np.int32)


@pytest.mark.parametrize("rule", ["paper", "mixed_nll"])
def test_skip_rule_and_state(rule):
    """A periodic stream makes the N-gram confident: skipped steps code
    p = p_ng exactly and leave the head and the mixer unchanged; other
    steps follow the unskipped rule."""
    m = Model(TINY, S.weights(TINY, 21))
    toks = periodic(5, 30, TINY.vocab, 21)
    st = StreamState.new(m, StepConfig(warmup=10, rule=rule, skip=True))
    ref = StreamState.new(m, StepConfig(warmup=10, rule=rule, skip=False))
    n_skip = 0
    for t in toks:
        b0 = st.head.b.copy()
        w0 = st.mixer.logw.copy()
        th0 = st.theta.copy()
        n0 = st.ngram.N
        p, _, _ = st.predict()
        z, pt, png, _ = st._cur
        h = entropy_bits(png)
        if h < SKIP_BITS:
            n_skip += 1
            assert st._skip and np.array_equal(p, png)
        else:
            assert not st._skip
        st.update(int(t))
        if h < SKIP_BITS:
            assert np.array_equal(st.head.b, b0) and np.array_equal(st.mixer.logw, w0)
            assert np.array_equal(st.theta, th0)
        assert st.ngram.N == n0 + 1
        ref.predict()
        ref.update(int(t))
    assert n_skip > 50 and st.skipped == n_skip
    assert ref.skipped == 0


def test_skip_before_any_context_is_never_taken():
    """At i = 1 the N-gram is the Laplace uniform 1/V: H = log2 V > 1.5."""
    m = Model(TINY, S.weights(TINY, 22))
    st = StreamState.new(m, StepConfig(skip=True))
    st.predict()
    assert not st._skip and entropy_bits(st._cur[2]) == pytest.approx(math.log2(TINY.vocab), abs=1e-9)


def test_skip_roundtrip_and_gain():
    """Lossless with the skip.  With the mixer held in warm-up (LLM alone,
    random weights) the skip is the only channel of the N-gram, and on a
    repetitive stream it codes in far fewer bits; the container flags it."""
    m = Model(TINY, S.weights(TINY, 23))
    toks = periodic(7, 25, TINY.vocab, 23)
    on = compress_stream(m, toks, StepConfig(warmup=10_000, skip=True))
    off = compress_stream(m, toks, StepConfig(warmup=10_000, skip=False))
    assert on["skipped"] > 100 and on["nbits"] < 0.5 * off["nbits"]
    out = decompress_stream(m, on["payload"], on["nbits"], len(toks), StepConfig(warmup=10_000, skip=True))
    assert np.array_equal(out, toks)
    buf = compress(m, [toks[:40]], StepConfig(warmup=5, skip=True))
    flags = container.unpack(buf)[0]
    assert flags & container.FLAG_SKIP
    with pytest.raises(container.ContainerError):
        decompress(m, buf, StepConfig(warmup=5, skip=False))
