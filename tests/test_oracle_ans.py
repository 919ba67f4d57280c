"""rANS oracle (oracle/ans.py) against what its definition fixes: the state
maps' closed forms on hand-worked values, brute force over every short
sequence of a small alphabet (round trip and injectivity), the final state,
and the information content (-sum log2 f / M) up to the bounded slack of the
renormalisation."""
import itertools
import math

import numpy as np
import pytest

from oracle import ans


def test_single_symbol_closed_form():
    # uniform over 256 symbols at M = 2^24 (f = 2^16), from x = L = 2^31:
    # no word moves out (x_max = 2^39 f), and C(s, 2^31) = (2^31 / 2^16) 2^24 + 0 + s 2^16
    for s in (0, 1, 77, 255):
        out = ans.encode([(s << 16, (s + 1) << 16)], 24)
        assert out == ((1 << 39) + (s << 16)).to_bytes(8, "little")


def test_two_symbols_by_hand():
    # M = 16, f = (8, 5, 3): code (s=1) then (s=2); the encoder runs them in reverse.
    # x = 2^31: C(2, x) = floor(2^31 / 3) * 16 + (2^31 mod 3) + 13
    x = (1 << 31)
    x = (x // 3) * 16 + (x % 3) + 13
    # x_max for f = 5 is (2^31 / 16) 2^32 5 = 5 * 2^59 > x: no word moves out
    x = (x // 5) * 16 + (x % 5) + 8
    assert ans.encode([(8, 13), (13, 16)], 4) == x.to_bytes(8, "little")


def test_brute_force_small_alphabet():
    cdf = [0, 8, 13, 16]                                   # M = 16, f = 8, 5, 3
    seen = {}
    for n in range(0, 6):
        for seq in itertools.product(range(3), repeat=n):
            data = ans.encode([(cdf[s], cdf[s + 1]) for s in seq], 4)
            d = ans.Decoder(data, 4)
            assert [d.decode(cdf) for _ in seq] == list(seq)
            assert d.finished()
            assert (data, n) not in seen                    # injective for a given length
            seen[(data, n)] = seq


def test_renormalisation_round_trip_and_size():
    rng = np.random.default_rng(5)
    for log2M, V, n in ((24, 1000, 4000), (16, 37, 3000), (31, 5, 2000), (24, 2, 5000)):
        M = 1 << log2M
        ivs, cdfs = [], []
        info = 0.0
        for _ in range(n):
            c = rng.multinomial(M - V, rng.dirichlet(np.full(V, 0.3))) + 1
            cdf = np.concatenate([[0], np.cumsum(c)]).astype(np.int64)
            s = int(rng.integers(V))
            ivs.append((int(cdf[s]), int(cdf[s + 1])))
            cdfs.append(cdf)
            info += math.log2(M / (cdf[s + 1] - cdf[s]))
        data = ans.encode(ivs, log2M)
        d = ans.Decoder(data, log2M)
        assert [d.decode(c) for c in cdfs] == [int(np.searchsorted(c, lo, side="right") - 1) for c, (lo, _) in
                                               zip(cdfs, ivs)]
        assert d.finished()
        bits = 8 * len(data)
        # each step multiplies x by M / f within a relative M / x <= M / 2^31; the
        # final state holds at most 64 bits and the start 31
        slack = n * math.log2(1 + M / 2 ** 31) + 64 + 32
        assert info - slack <= bits - 31 <= info + slack


def test_decoder_state_detects_a_wrong_cdf():
    cdf = [0, 8, 13, 16]
    data = ans.encode([(0, 8), (8, 13), (13, 16)] * 20, 4)
    d = ans.Decoder(data, 4)
    other = [0, 5, 13, 16]
    for _ in range(60):
        d.decode(other)
    assert not d.finished()


def test_rejects_bad_input():
    with pytest.raises(ans.AnsError):
        ans.encode([(5, 5)], 8)
    with pytest.raises(ans.AnsError):
        ans.encode([(0, 257)], 8)
    with pytest.raises(ans.AnsError):
        ans.Decoder(b"\x00" * 9, 8)
