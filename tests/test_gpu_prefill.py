"""GPU tests of the encoder's chunked prefill, through the C ABI.

With prefill_rows set, the encoder runs the model over m positions of every
stream in one forward pass (between window slides) and then the per-token
vocabulary passes in order.  Every row's arithmetic is the decode step's, so
the coder intervals must equal, bit for bit, those of one position per step,
and a container written with prefill must decode one position per step.
"""
import dataclasses

import numpy as np
import pytest
import torch

import synthetic as S

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def nc(gpu_lib):
    return gpu_lib


def intervals(nc, shape, w, fmt, path, toks, prefill_rows, max_streams, rule="paper"):
    lens = np.array([len(t) for t in toks], dtype=np.int64)
    offs = np.concatenate([[0], np.cumsum(lens)[:-1]]).astype(np.int64)
    flat = torch.from_numpy(np.concatenate(toks).astype(np.int32)).cuda()
    stride = max(int(lens.max()), 1)
    ctx = nc.Context(nc.make_config(shape, fmt=fmt, path=path, warmup=20, max_streams=max_streams,
                                    prefill_rows=prefill_rows, rule=rule), w)
    iv = torch.full((len(toks), stride, 2), -1, dtype=torch.int32, device="cuda")
    ctx.encode_intervals(flat, offs, lens, iv, stride)
    out = iv.cpu().numpy()
    ctx.close()
    return out


@pytest.mark.parametrize("fmt,path", [("fp32", "gemv"), ("bf16", "gemv"), ("bf16", "tc"), ("fp8", "tc")])
def test_prefill_intervals_equal_decode(nc, fmt, path):
    """Small model (window 512, slide 128): three ragged streams, one
    crossing four slides; prefill chunks of 64 positions (3 streams, 256
    rows) and of 128 (1 stream) give the decode intervals exactly."""
    shape, seed = S.SMALL, 6
    w = S.flat_weights(shape, seed)
    toks = [S.token_stream(seed, j, n, shape.vocab) for j, n in enumerate([1000, 130, 1])]
    ref = intervals(nc, shape, w, fmt, path, toks, 0, 3)
    got = intervals(nc, shape, w, fmt, path, toks, 256, 3)
    assert np.array_equal(got, ref)
    one = intervals(nc, shape, w, fmt, path, toks[:1], 1024, 1)
    assert np.array_equal(one[0], ref[0])


@pytest.mark.parametrize("path", ["gemv", "tc"])
def test_prefill_mixed_nll_equals_decode(nc, path):
    """The mixed-NLL update rule (its head step waits for the mixer, so the
    prefill loop takes a second barrier per position): prefill chunks give the
    decode intervals exactly."""
    shape, seed = S.SMALL, 9
    w = S.flat_weights(shape, seed)
    toks = [S.token_stream(seed, j, n, shape.vocab) for j, n in enumerate([600, 97])]
    ref = intervals(nc, shape, w, "bf16", path, toks, 0, 2, rule="mixed_nll")
    got = intervals(nc, shape, w, "bf16", path, toks, 256, 2, rule="mixed_nll")
    assert np.array_equal(got, ref)


@pytest.mark.parametrize("path", ["gemv", "tc"])
def test_prefill_full_model_single_stream(nc, path):
    """Full-size BF16 model, one 700-token stream: a 512-position prefill
    chunk then a partial one give the decode intervals exactly, on the
    CUDA-core and the tensor-core paths."""
    shape, seed = S.FULL, 1
    w = S.flat_weights(shape, seed)
    toks = [S.token_stream(seed, 0, 700, shape.vocab)]
    ref = intervals(nc, shape, w, "bf16", path, toks, 0, 1)
    got = intervals(nc, shape, w, "bf16", path, toks, 4096, 1)
    assert np.array_equal(got, ref)


def test_prefill_container_decodes_per_position(nc):
    """A container written with prefill decodes, one position per step, to
    the original streams; it is byte-identical to the one written without."""
    shape, seed = dataclasses.replace(S.SMALL, ctx_len=256, slide=64), 7
    w = S.flat_weights(shape, seed)
    streams = [S.token_stream(seed, 20 + j, n, shape.vocab) for j, n in enumerate([400, 0, 65, 3])]
    enc = nc.Context(nc.make_config(shape, fmt="bf16", warmup=10, max_streams=4, prefill_rows=128), w)
    blob = enc.encode(streams)
    enc.close()
    dec = nc.Context(nc.make_config(shape, fmt="bf16", warmup=10, max_streams=4), w)
    plain = dec.encode(streams)
    back = dec.decode(blob)
    dec.close()
    assert blob == plain
    for a, b in zip(streams, back):
        assert np.array_equal(a, b)


@pytest.mark.parametrize("fmt,path,split", [("bf16", "gemv", "0"), ("bf16", "tc", "0"), ("fp32", "gemv", "0"),
                                            ("fp32", "gemv", "1"), ("fp32", "gemv", "2"), ("fp32", "gemv", "4"),
                                            ("fp32", "gemv", "8")])
def test_prefill_attention_split(nc, monkeypatch, fmt, path, split):
    """Windows up to 2,048 positions (8 chunks of 256) with a slide: the
    prefill's attention gives the decode intervals exactly.  BF16 cache: the
    tensor-core attention (rows of 512-position prefill chunks in tiles of
    42 rows).  FP32 cache: the CUDA-core row kernel with 1, 2, 4 or 8 CTAs
    per row group ("0": picked from the rows)."""
    shape, seed = dataclasses.replace(S.SMALL, ctx_len=2048, slide=512), 8
    w = S.flat_weights(shape, seed)
    toks = [S.token_stream(seed, j, n, shape.vocab) for j, n in enumerate([2300, 700])]
    ref = intervals(nc, shape, w, fmt, path, toks, 0, 2)
    monkeypatch.setenv("NC24_ATTN_CLUSTER", split)
    got = intervals(nc, shape, w, fmt, path, toks, 1024, 2)
    assert np.array_equal(got, ref)


@pytest.mark.parametrize("path,ctx_len,slide", [("tc", 256, 40), ("gemv", 256, 40), ("tc", 32, 8)])
def test_bf16_cache_ring_wrap_windows(nc, path, ctx_len, slide):
    """BF16 KV cache with windows whose 64-position attention blocks wrap
    around the ring (a slide of 40: the window starts at multiples of 40) and
    with a ring shorter than one block (window 32): the per-token step's
    logits against the oracle on the dequantised BF16 weights (Sec. 3.9
    window, slides included), and the prefill's intervals equal the
    per-token step's bit for bit."""
    from oracle.model import Model

    shape, seed = dataclasses.replace(S.SMALL, ctx_len=ctx_len, slide=slide), 11
    w = S.flat_weights(shape, seed)
    n = 2 * ctx_len + 3 * slide + 5
    toks = S.token_stream(seed, 0, n, shape.vocab)
    ctx = nc.Context(nc.make_config(shape, fmt="bf16", path=path, warmup=20), w)
    z = torch.empty(1, shape.vocab, device="cuda")
    ctx.stream_open(0, n)
    m = Model(shape, S.weights(shape, seed), "bf16")
    cache = m.new_cache()
    last = Model.BOS
    err = 0.0
    for t in toks:
        ctx.step_probe([0], z=z)
        ref = m.step(cache, last)
        err = max(err, float(np.max(np.abs(z[0].cpu().numpy() - ref))))
        ctx.update_bias([0], [int(t)])
        last = int(t)
    ctx.close()
    assert cache.slides >= 3
    print(f"{path} window {ctx_len} slide {slide}: logits max abs err {err:.3e}")
    assert err <= 1.5e-2
    ref_iv = intervals(nc, shape, w, "bf16", path, [toks], 0, 1)
    got_iv = intervals(nc, shape, w, "bf16", path, [toks], 4 * slide, 1)
    assert np.array_equal(got_iv, ref_iv)


_M64 = (1 << 64) - 1


def _mix64(x: int) -> int:
    """The N-gram index's home-slot hash (a 64-bit finaliser), to build keys
    whose home slots crowd together."""
    x ^= x >> 33
    x = (x * 0xFF51AFD7ED558CCD) & _M64
    x ^= x >> 33
    x = (x * 0xC4CEB9FE1A85EC53) & _M64
    x ^= x >> 33
    return x


@pytest.mark.parametrize("fmt,path", [("fp32", "gemv"), ("bf16", "tc")])
def test_prefill_ngram_long_probes(nc, fmt, path):
    """The prefill's N-gram pass reads 32 index slots per load; a key whose
    probe runs past them takes the one-slot-at-a-time walk (look-up and
    insert).  48 distinct tokens whose order-1 keys (the token ids) home in
    4 neighbouring slots of the stream's 1,024-slot index fill a run of 48
    slots, so inserting or finding the later ones probes past 32 slots; the
    intervals still equal those of one update per step."""
    shape, seed = S.SMALL, 12
    n = 300
    cap = 1 << (2 * n - 1).bit_length()          # the index capacity for an n-token stream
    assert cap == 1024
    home = 100
    crowd = [t for t in range(1, shape.vocab) if home <= (_mix64(t) & (cap - 1)) < home + 4][:48]
    assert len(crowd) == 48
    # linear probing in insertion order: some key sits more than 32 slots past its home
    used, far = set(), 0
    for t in crowd:
        h = _mix64(t) & (cap - 1)
        d = 0
        while (h + d) % cap in used:
            d += 1
        used.add((h + d) % cap)
        far = max(far, d)
    assert far > 32
    toks = np.array((crowd * (n // len(crowd) + 1))[:n], dtype=np.int32)
    w = S.flat_weights(shape, seed)
    ref = intervals(nc, shape, w, fmt, path, [toks], 0, 1)
    got = intervals(nc, shape, w, fmt, path, [toks], 256, 1)
    assert np.array_equal(got, ref)
