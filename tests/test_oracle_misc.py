"""Pins for the number formats, the NC05-style container (Sec. 3.12) and the
whole compression loop (Algorithm 1): lossless round trip and the coded size
against the quantised code length and the coder's bound."""
import json
import math
import os

import numpy as np
import pytest

import synthetic as S
from oracle import cdf as Q
from oracle import container, numerics
from oracle.coder import QTR
from oracle.compress import StepConfig, compress, compress_stream, decompress, decompress_stream
from oracle.model import Model

GOLD = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "paper_values.json")))
TINY = S.ModelShape(n_layers=2, d_model=32, n_heads=4, n_kv_heads=2, d_ffn=48,
                    vocab=97, ctx_len=16, slide=4)


def test_bf16_rounding_examples():
    x = np.array([1 + 2 ** -8, 1 + 3 * 2 ** -8, -2.5, 3.0e38, 1e-40], dtype=np.float32)
    got = numerics.bf16_round(x)
    assert got[0] == 1.0                      # tie -> even
    assert got[1] == 1 + 2 ** -6              # tie -> even (upwards)
    assert got[2] == -2.5
    assert np.isfinite(got[3])
    assert np.all(got.view(np.uint32) & 0xFFFF == 0)   # every result is a bf16 value


def test_e4m3_rounding_examples():
    got = numerics.e4m3_round(np.array([0.3, 17.0, 19.0, 500.0, -448.0, 2.0 ** -9, 2.0 ** -11, 0.0]))
    assert list(got) == [0.3125, 16.0, 20.0, 448.0, -448.0, 2.0 ** -9, 0.0, 0.0]
    grid = numerics._GRID
    assert grid[-1] == 448.0 and len(grid) == 127
    assert np.array_equal(numerics.e4m3_round(grid), grid)


def test_container_layout_and_errors():
    recs = [(10, 33, 5), (3, 8, 1)]
    pays = [b"\x01\x02\x03\x04\x05", b"\xff"]
    buf = container.pack(container.FLAG_NGRAM | container.FLAG_HEAD, 1.0, 0x21, recs, pays)
    assert buf[:4] == b"NC05"
    assert GOLD["nc05_header_bytes"]["value"] == 4 + 1 + 2 + 2 == container.HEADER
    assert GOLD["nc05_record_bytes"]["value"] == 12 == container.RECORD
    assert len(buf) == 9 + 1 + 12 * 2 + 6
    flags, tau, pb, r2, p2 = container.unpack(buf)
    assert flags == 3 and tau == 1.0 and pb == 0x21 and r2 == recs and p2 == pays
    for bad in (buf[:-1], buf + b"\x00", b"NC06" + buf[4:], buf[:12]):
        with pytest.raises(container.ContainerError):
            container.unpack(bad)


@pytest.mark.parametrize("rule", ["paper", "mixed_nll"])
def test_loop_roundtrip_and_size_bound(rule):
    w = S.weights(TINY, 11)
    m = Model(TINY, w)
    cfg = StepConfig(warmup=10, rule=rule)
    toks = S.token_stream(11, 0, 60, TINY.vocab)   # crosses several slides (L=16, C=4)
    r = compress_stream(m, toks, cfg, record_steps=60)
    assert r["slides"] > 0
    # coded size within the coder bound of the quantised code length
    qbits, slack = 0.0, 0.0
    for rec, t in zip(r["records"], toks):
        c = int(rec["cdf"][t + 1] - rec["cdf"][t])
        qbits += -math.log2(c / cfg.T)
        slack += -math.log2(1 - cfg.T / (QTR * c))
    assert r["nbits"] <= qbits + slack + 2
    assert r["nbits"] >= qbits - 1e-6 - 32
    out = decompress_stream(m, r["payload"], r["nbits"], len(toks), cfg)
    assert np.array_equal(out, toks)
    assert r["min_range"] > QTR


def test_multi_stream_container_roundtrip():
    w = S.weights(TINY, 12)
    m = Model(TINY, w)
    cfg = StepConfig(warmup=5)
    streams = [S.token_stream(12, j, n, TINY.vocab) for j, n in enumerate([1, 7, 30])]
    buf = compress(m, streams, cfg, path_byte=0)
    out = decompress(m, buf, cfg)
    for a, b in zip(streams, out):
        assert np.array_equal(a, b)
    with pytest.raises(container.ContainerError):
        decompress(m, buf, StepConfig(warmup=5, use_ngram=False))


def test_rans_container_roundtrip_and_size():
    """The loop with the rANS coder (the ANS coder of Sec. 6): lossless, flagged
    in the container, and within 96 bits plus 0.02 bit per token of the
    arithmetic coder's stream on the same CDFs."""
    w = S.weights(TINY, 13)
    m = Model(TINY, w)
    cfg = StepConfig(warmup=5, coder="rans")
    streams = [S.token_stream(13, j, n, TINY.vocab) for j, n in enumerate([0, 9, 60])]
    buf = compress(m, streams, cfg, path_byte=0)
    flags = container.unpack(buf)[0]
    assert flags & container.FLAG_RANS
    for a, b in zip(streams, decompress(m, buf, cfg)):
        assert np.array_equal(a, b)
    with pytest.raises(container.ContainerError):
        decompress(m, buf, StepConfig(warmup=5))
    for toks in streams[1:]:
        r = compress_stream(m, toks, cfg)
        a = compress_stream(m, toks, StepConfig(warmup=5))
        assert abs(r["nbits"] - a["nbits"]) <= 96 + 0.02 * len(toks) + 32


def test_ideal_bits_match_quantised_bits_closely():
    """With V = 97 the floors cost log2(T / (T - V)) ~ 8e-6 bits per token at
    most, so quantised and ideal code lengths agree closely."""
    w = S.weights(TINY, 13)
    m = Model(TINY, w)
    cfg = StepConfig(warmup=5)
    toks = S.token_stream(13, 0, 40, TINY.vocab)
    r = compress_stream(m, toks, cfg, record_steps=40)
    qbits = sum(Q.code_length_bits(rec["cdf"], t, cfg.T) for rec, t in zip(r["records"], toks))
    assert abs(qbits - r["ideal_bits"]) < 40 * 1e-3
