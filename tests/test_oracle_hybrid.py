"""NC06 hybrid segmentation and container (oracle/hybrid.py, Sec. 3.10, Sec.
3.12) against what the four rules fix: hand-worked inputs for each rule,
uniformly random bytes staying binary (which fixes the order of rules 2
and 3), the character
classes of rule 1, and invariants on random structured inputs (the runs
cover the input and alternate, text runs hold at least 64 bytes, binary runs
under 64 bytes only without text, and splitting then joining gives the
input back); the blob's size rule and the container layout round trip."""
import gzip
import lzma

import numpy as np

from oracle import hybrid as H

T, B = H.TEXT, H.BINARY


def txt(n):
    return b"a" * n


def bin_(n):
    return b"\x00" * n


def test_rule_1_classes():
    assert all(H.is_text_byte(b) for b in range(32, 127))
    assert all(H.is_text_byte(b) for b in (9, 10, 13))
    assert not any(H.is_text_byte(b) for b in (0, 8, 11, 12, 14, 31, 127, 128, 255))
    assert H.segment(b"\t\n\r" + txt(61)) == [(T, 64)]


def test_rule_2_short_text_demoted():
    assert H.segment(txt(64)) == [(T, 64)]
    assert H.segment(txt(63)) == [(B, 63)]
    assert H.segment(bin_(200) + txt(30) + bin_(200)) == [(B, 430)]


def test_rule_3_gaps_after_demotion():
    # gaps of up to 8 bytes join text runs that rule 2 kept
    assert H.segment(txt(64) + bin_(8) + txt(64)) == [(T, 136)]
    assert H.segment(txt(100) + b"\x7f" + txt(100)) == [(T, 201)]
    # text runs too short for rule 2 are binary before any gap is bridged
    assert H.segment(txt(40) + bin_(8) + txt(40)) == [(B, 88)]
    assert H.segment(txt(32) + b"\x7f" + txt(31)) == [(B, 64)]
    # a gap at either end is not between two text runs
    assert H.segment(bin_(3) + txt(10)) == [(B, 13)]


def test_random_bytes_stay_binary():
    # uniform bytes are text-like with probability 98/256 but hold no text-like
    # run of 64; bridging their gaps first would call most of them text
    for seed in range(4):
        data = bytes(np.random.default_rng(seed).integers(0, 256, 5000, dtype=np.uint8))
        assert H.segment(data) == [(B, 5000)]


def test_rule_4_small_binary_absorbed():
    assert H.segment(bin_(10) + txt(100) + bin_(10)) == [(T, 120)]
    assert H.segment(txt(100) + bin_(63) + txt(100)) == [(T, 263)]
    assert H.segment(txt(100) + bin_(64) + txt(100)) == [(T, 100), (B, 64), (T, 100)]
    assert H.segment(bin_(64) + txt(100)) == [(B, 64), (T, 100)]
    assert H.segment(bin_(5)) == [(B, 5)]                   # no text to be absorbed into
    assert H.segment(b"") == []


def _random_input(rng, n_runs):
    parts = []
    for _ in range(n_runs):
        n = int(rng.integers(1, 120))
        if rng.random() < 0.5:
            parts.append(bytes(rng.choice(np.r_[9, 10, 13, 32:127], n).astype(np.uint8)))
        else:
            parts.append(bytes(rng.choice(np.r_[0:9, 11, 12, 14:32, 127:256], n).astype(np.uint8)))
    return b"".join(parts)


def test_invariants_random():
    rng = np.random.default_rng(5)
    for trial in range(400):
        data = _random_input(rng, int(rng.integers(0, 12)))
        runs = H.segment(data)
        assert sum(n for _, n in runs) == len(data)
        assert all(n > 0 for _, n in runs)
        assert all(runs[i][0] != runs[i + 1][0] for i in range(len(runs) - 1))
        assert all(n >= H.MIN_TEXT for k, n in runs if k == T)
        assert all(n >= H.MIN_BINARY or len(runs) == 1 for k, n in runs if k == B)
        texts, blob = H.split(data, runs)
        assert H.join(runs, texts, blob) == data
        assert len(blob) == sum(n for k, n in runs if k == B)
        # all text-like input: one text run, or one binary run when short
        if data and all(H.is_text_byte(b) for b in data):
            assert runs == [(T if len(data) >= 64 else B, len(data))]


def test_blob_size_rule():
    small = b"ab" * 2000                                     # 4,000 bytes: gzip
    m, s = H.pack_blob(small)
    assert m == H.GZIP and gzip.decompress(s) == small
    big = b"ab" * 2048                                       # 4,096 bytes: LZMA
    m, s = H.pack_blob(big)
    assert m == H.LZMA and lzma.decompress(s) == big
    noise = bytes(np.random.default_rng(1).integers(0, 256, 5000, dtype=np.uint8))
    assert H.pack_blob(noise) == (H.RAW, noise)              # compression does not help
    assert H.pack_blob(b"") == (H.RAW, b"")
    for blob in (small, big, noise, b""):
        assert H.unpack_blob(*H.pack_blob(blob)) == blob


def test_container_round_trip():
    data = bin_(100) + txt(300) + bin_(70) + txt(80)
    runs = H.segment(data)
    texts, blob = H.split(data, runs)
    m, s = H.pack_blob(blob)
    text = b"NC05" + bytes([3]) + (0x3A66).to_bytes(2, "little") + b"\x02\x00rest"   # flags 3, tau 0.8
    buf = H.pack(runs, m, s, text)
    assert buf[:4] == b"NC06" and buf[4] == 1 and buf[5] == 3 and buf[6:8] == bytes([0x66, 0x3A])
    assert len(buf) == 12 + 5 * len(runs) + 5 + len(s) + len(text)
    flags, tau, runs2, m2, s2, tc = H.unpack(buf)
    assert (flags, tau, runs2, m2, s2, tc) == (3, 0x3A66, runs, m, s, text)
    assert H.join(runs2, texts, H.unpack_blob(m2, s2)) == data
    # no text run: flags 0 and tau 1.0, nothing after the blob
    runs = H.segment(bin_(20))
    buf = H.pack(runs, H.RAW, bin_(20), b"")
    assert H.unpack(buf) == (0, 0x3C00, [(B, 20)], H.RAW, bin_(20), b"")
