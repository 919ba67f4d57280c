"""CPU tests of the C ABI: the library loads and exports every declared
entry point, host-only calls (coder, container parsing, argument checks)
agree with the oracle, and nothing here touches a GPU."""
import os
import re

import numpy as np
import pytest

import synthetic as S
from oracle.coder import Decoder, Encoder

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def nc24():
    from paper_2602_19626_gb300 import build
    build.build()
    from paper_2602_19626_gb300 import nc24 as m
    return m


def declared_symbols():
    hdr = open(os.path.join(ROOT, "include", "nc24.h")).read()
    hdr = re.sub(r"/\*.*?\*/", "", hdr, flags=re.S)
    return sorted(set(re.findall(r"\b(nc_[a-z0-9_]+)\s*\(", hdr)))


def test_exports_every_declared_symbol(nc24):
    decl = declared_symbols()
    assert len(decl) >= 20
    for name in decl:
        assert hasattr(nc24.lib, name), name
    assert sorted(nc24.EXPORTED) == decl


def test_config_default_and_status(nc24):
    c = nc24.nc_config_default()
    assert (c.n_layers, c.d_model, c.n_heads, c.n_kv_heads, c.d_ffn, c.vocab) == (30, 576, 9, 3, 1536, 49152)
    assert (c.ctx_len, c.slide, c.cdf_log2_total, c.floor, c.warmup) == (2048, 512, 24, 1, 100)
    assert abs(c.bias_lr - 1e-3) < 1e-9 and abs(c.w_llm_init - 0.85) < 1e-7
    assert (c.prefill_rows, c.skip, c.coder) == (0, 0, nc24.NC_CODER_ARITH)
    assert nc24.nc_status_str(nc24.NC_ENUMERIC) == "NC_ENUMERIC"


def test_ctx_create_rejects_bad_config_without_gpu(nc24):
    import ctypes as C
    c = nc24.nc_config_default()
    w = np.zeros(4, dtype=np.float32)
    h = C.c_void_p()
    assert nc24.lib.nc_ctx_create(C.byref(c), w.ctypes.data, w.nbytes, C.byref(h)) == nc24.NC_EINVAL
    c.d_model = 100
    assert nc24.lib.nc_ctx_create(C.byref(c), w.ctypes.data, w.nbytes, C.byref(h)) == nc24.NC_EINVAL
    c = nc24.nc_config_default()
    c.coder = 7
    assert nc24.lib.nc_ctx_create(C.byref(c), w.ctypes.data, w.nbytes, C.byref(h)) == nc24.NC_EINVAL
    assert not h.value


@pytest.mark.parametrize("log2T", [8, 16, 24])
def test_host_coder_matches_oracle(nc24, log2T):
    T = 1 << log2T
    rng = np.random.default_rng(log2T)
    n = 3000
    lo = np.empty(n, np.uint32)
    hi = np.empty(n, np.uint32)
    V = 37
    cdfs = np.empty((n, V + 1), np.uint32)
    for i in range(n):
        c = rng.multinomial(T - V, rng.dirichlet(np.full(V, 0.2))) + 1
        cdf = np.concatenate([[0], np.cumsum(c)]).astype(np.uint32)
        s = int(rng.integers(V))
        cdfs[i] = cdf
        lo[i], hi[i] = cdf[s], cdf[s + 1]
    data, nbits = nc24.nc_ac_encode(lo, hi, log2T)
    enc = Encoder(T)
    for a, b in zip(lo, hi):
        enc.encode_interval(int(a), int(b))
    ref, ref_bits = enc.finish()
    assert nbits == ref_bits and data == ref
    sym = nc24.nc_ac_decode(data, nbits, cdfs, log2T)
    dec = Decoder(ref, ref_bits, T)
    ref_sym = [dec.decode(c) for c in cdfs]
    assert list(sym) == ref_sym
    assert np.all(cdfs[np.arange(n), sym] == lo)


def test_host_coder_rejects_bad_input(nc24):
    with pytest.raises(nc24.NcError):
        nc24.nc_ac_encode(np.array([5], np.uint32), np.array([5], np.uint32), 8)
    with pytest.raises(nc24.NcError):
        nc24.nc_ac_encode(np.array([0], np.uint32), np.array([257], np.uint32), 8)
    bad = np.array([[0, 3, 2, 256]], np.uint32)
    with pytest.raises(nc24.NcError):
        nc24.nc_ac_decode(b"\x00", 8, np.array([[0, 3, 3, 255]], np.uint32), 8)


@pytest.mark.parametrize("log2T", [24, 16, 31])
def test_host_rans_matches_oracle(nc24, log2T):
    """The C++ rANS coder writes the oracle's bytes and decodes its symbols."""
    from oracle import ans
    T = 1 << log2T
    rng = np.random.default_rng(100 + log2T)
    n, V = 2500, 29
    lo = np.empty(n, np.uint32)
    hi = np.empty(n, np.uint32)
    cdfs = np.empty((n, V + 1), np.uint32)
    for i in range(n):
        c = rng.multinomial(T - V, rng.dirichlet(np.full(V, 0.2))) + 1
        cdf = np.concatenate([[0], np.cumsum(c)]).astype(np.uint64)
        s = int(rng.integers(V))
        cdfs[i] = cdf
        lo[i], hi[i] = cdf[s], cdf[s + 1]
    data = nc24.nc_ans_encode(lo, hi, log2T)
    ref = ans.encode(zip(lo.tolist(), hi.tolist()), log2T)
    assert data == ref
    sym = nc24.nc_ans_decode(data, cdfs, log2T)
    assert np.all(cdfs[np.arange(n), sym] == lo)
    assert len(nc24.nc_ans_encode(lo[:0], hi[:0], log2T)) == 8          # the initial state alone


def test_host_rans_rejects_bad_input(nc24):
    with pytest.raises(nc24.NcError):
        nc24.nc_ans_encode(np.array([5], np.uint32), np.array([5], np.uint32), 8)
    with pytest.raises(nc24.NcError):
        nc24.nc_ans_encode(np.array([0], np.uint32), np.array([257], np.uint32), 8)
    cdf = np.array([[0, 100, 200, 256]], np.uint32)
    data = nc24.nc_ans_encode(np.array([100], np.uint32), np.array([200], np.uint32), 8)
    with pytest.raises(nc24.NcError):                                  # not 8 + 4k bytes
        nc24.nc_ans_decode(data + b"\x00", cdf, 8)
    with pytest.raises(nc24.NcError):                                  # one symbol too many
        nc24.nc_ans_decode(data, np.repeat(cdf, 2, axis=0), 8)
    assert list(nc24.nc_ans_decode(data, cdf, 8)) == [1]


def test_split_chunks_matches_oracle(nc24):
    """File-level chunking (Sec. 3.11): the library's cuts are the oracle's."""
    from oracle import chunking
    rng = np.random.default_rng(7)
    V = 300
    bnd = (rng.random(V) < 0.05).astype(np.uint8)
    for n, N in ((0, 4), (1, 8), (37, 3), (5000, 8), (5000, 1), (999, 16)):
        toks = rng.integers(0, V, n).astype(np.int32)
        got = nc24.nc_split_chunks(toks, bnd, N)
        assert list(got) == chunking.split_points(toks, bnd, N)
    with pytest.raises(nc24.NcError):
        nc24.nc_split_chunks(np.array([V], np.int32), bnd, 2)           # id out of range
    with pytest.raises(nc24.NcError):
        nc24.nc_split_chunks(np.array([1], np.int32), bnd, 0)


def test_container_parse(nc24):
    import ctypes as C
    from oracle import container
    buf = container.pack(3, 1.0, 1, [(10, 33, 5), (0, 1, 1)], [b"abcde", b"\x80"])
    arr = np.frombuffer(buf, np.uint8).copy()
    n = C.c_int(0)
    assert nc24.lib.nc_container_streams(arr.ctypes.data, arr.size, C.byref(n)) == 0 and n.value == 2
    for cut in (arr[:-1], arr[:9], np.concatenate([arr, [0]]).astype(np.uint8)):
        cut = np.ascontiguousarray(cut)
        assert nc24.lib.nc_container_streams(cut.ctypes.data, cut.size, C.byref(n)) == nc24.NC_ECORRUPT


def _hybrid_inputs():
    """Byte strings for the NC06 segmentation: each rule's edges, and random
    mixes of text-like and binary runs of 1..150 bytes."""
    t, b = b"x", b"\x00"
    yield from (b"", t * 63, t * 64, b * 5, t * 40 + b * 8 + t * 40, t * 40 + b * 9 + t * 40,
                b * 10 + t * 100 + b * 10, t * 100 + b * 63 + t * 100, t * 100 + b * 64 + t * 100,
                b"\t\n\r" + t * 61, t * 32 + b"\x7f" + t * 31)
    rng = np.random.default_rng(11)
    text_bytes = np.r_[9, 10, 13, 32:127].astype(np.uint8)
    bin_bytes = np.r_[0:9, 11, 12, 14:32, 127:256].astype(np.uint8)
    for _ in range(300):
        parts = [rng.choice(text_bytes if rng.random() < 0.5 else bin_bytes, int(rng.integers(1, 150)))
                 for _ in range(int(rng.integers(1, 16)))]
        yield np.concatenate(parts).tobytes()


def test_hybrid_segments_match_oracle(nc24):
    """NC06 segmentation (Sec. 3.10): the library's runs are the oracle's."""
    from oracle import hybrid
    for data in _hybrid_inputs():
        kinds, lens = nc24.nc_hybrid_segments(data)
        assert list(zip(kinds.tolist(), lens.tolist())) == hybrid.segment(data)


def test_hybrid_container_matches_oracle(nc24):
    """NC06 layout: the library's container is the oracle's byte for byte, and
    its parse gives back the runs and sections."""
    from oracle import hybrid
    rng = np.random.default_rng(12)
    text = b"NC05" + bytes([7]) + (0x3B33).to_bytes(2, "little") + bytes(rng.integers(0, 256, 40, dtype=np.uint8))
    for data in list(_hybrid_inputs())[:60]:
        runs = hybrid.segment(data)
        if not runs:
            continue
        texts, blob = hybrid.split(data, runs)
        method, stored = hybrid.pack_blob(blob)
        tc = text if texts else b""
        kinds = np.array([k for k, _ in runs], np.uint8)
        lens = np.array([n for _, n in runs], np.int64)
        buf = nc24.nc_hybrid_pack(kinds, lens, method, stored, tc)
        assert buf == hybrid.pack(runs, method, stored, tc)
        k2, l2, m2, so, sl, to = nc24.nc_hybrid_parse(buf)
        assert list(zip(k2.tolist(), l2.tolist())) == runs and m2 == method
        assert buf[so:so + sl] == stored and buf[to:] == tc


def test_hybrid_rejects_bad_input(nc24):
    good = nc24.nc_hybrid_pack(np.array([1], np.uint8), np.array([3], np.int64), 0, b"abc", b"")
    assert nc24.nc_hybrid_parse(good)[:3][2] == 0
    for bad in (good[:-1], b"NC07" + good[4:], good[:4] + b"\x02" + good[5:], good[:12] + b"\x02" + good[13:]):
        with pytest.raises(nc24.NcError) as e:
            nc24.nc_hybrid_parse(bad)
        assert e.value.status == nc24.NC_ECORRUPT
    with pytest.raises(nc24.NcError):
        nc24.nc_hybrid_pack(np.array([2], np.uint8), np.array([3], np.int64), 0, b"abc", b"")      # kind
    with pytest.raises(nc24.NcError):
        nc24.nc_hybrid_pack(np.array([0], np.uint8), np.array([0], np.int64), 0, b"", b"")         # length 0
    with pytest.raises(nc24.NcError):
        nc24.nc_hybrid_pack(np.array([0], np.uint8), np.array([3], np.int64), 3, b"", b"")         # method
    with pytest.raises(nc24.NcError):
        nc24.nc_hybrid_pack(np.array([0], np.uint8), np.array([3], np.int64), 0, b"", b"not NC05")  # text


def test_launch_chain_floor_rejects_bad_arguments(nc24):
    """The launch-floor diagnostic checks its arguments before touching a device."""
    for args in ((0, 0, 152, 256, 1), (0, 16, 0, 256, 1), (0, 16, 152, 33, 1), (0, 16, 152, 256, 0),
                 (0, 5000, 152, 256, 1)):
        with pytest.raises(nc24.NcError) as e:
            nc24.nc_launch_chain_floor(*args)
        assert e.value.status == nc24.NC_EINVAL


def test_hybrid_blob_errors_are_corrupt_containers(nc24):
    """A damaged compressed binary section reads as a corrupt container."""
    import gzip
    for method, stored in ((1, b"not gzip"), (2, b"not xz"), (1, gzip.compress(b"abc")[:-3])):
        with pytest.raises(nc24.NcError) as e:
            nc24._blob_unpack(method, stored)
        assert e.value.status == nc24.NC_ECORRUPT
    assert nc24._blob_unpack(*nc24._blob_pack(b"y" * 5000)) == b"y" * 5000
