"""GPU tests of the NC06 hybrid binary format (Sec. 3.10), through the C ABI.

A seeded synthetic binary file mixes text regions, binary regions, short
text islands inside binary data and short binary gaps inside text.  The
container's run table and binary section must equal the oracle's byte for
byte (segmentation and the blob rule), its text runs are coded on the GPU as
the streams of one NC05 container, and decoding gives the file back.
"""
import numpy as np
import pytest

import synthetic as S
from oracle import hybrid

pytestmark = pytest.mark.gpu

TEXT = np.r_[9, 10, 13, 32:127].astype(np.uint8)
BINARY = np.r_[0:9, 11, 12, 14:32, 127:256].astype(np.uint8)


def synthetic_file(seed: int, n_regions: int) -> bytes:
    rng = np.random.default_rng(seed)
    parts = []
    for _ in range(n_regions):
        r = rng.random()
        if r < 0.4:                                     # a text region, with short gaps in it
            text = rng.choice(TEXT, int(rng.integers(80, 400)))
            for p in rng.integers(0, text.size, int(rng.integers(0, 3))):
                text = np.concatenate([text[:p], rng.choice(BINARY, int(rng.integers(1, 9))), text[p:]])
            parts.append(text)
        elif r < 0.7:                                   # a binary region, maybe a run of zeros
            if rng.random() < 0.3:
                parts.append(np.zeros(int(rng.integers(64, 3000)), np.uint8))
            else:
                parts.append(rng.integers(0, 256, int(rng.integers(10, 300))).astype(np.uint8))
        else:                                           # a short text island
            parts.append(rng.choice(TEXT, int(rng.integers(5, 60))))
    return np.concatenate(parts).astype(np.uint8).tobytes()


def context(nc, n_streams):
    shape = S.SMALL
    cfg = nc.make_config(shape, fmt="fp32", warmup=20, max_streams=max(n_streams, 1))
    return nc.Context(cfg, S.flat_weights(shape, 0))


@pytest.mark.parametrize("seed", [0, 1])
def test_hybrid_round_trip_and_layout(gpu_lib, seed):
    data = synthetic_file(seed, 14)
    runs = hybrid.segment(data)
    n_text = sum(k == hybrid.TEXT for k, _ in runs)
    assert n_text >= 2 and len(runs) > n_text               # both kinds present
    ctx = context(gpu_lib, n_text)
    buf = ctx.encode_hybrid(data)
    # the run table and the binary section are the oracle's
    _, blob = hybrid.split(data, runs)
    method, stored = hybrid.pack_blob(blob)
    head = len(hybrid.pack(runs, method, stored, b""))
    assert buf[:5] == b"NC06\x01" and buf[8:head] == hybrid.pack(runs, method, stored, b"")[8:]
    # the text runs' NC05 container follows; its flags and temperature are repeated in the header
    assert buf[head:head + 4] == b"NC05" and buf[5:8] == buf[head + 4:head + 7]
    assert ctx.decode_hybrid(buf) == data
    ctx.close()


def test_hybrid_one_kind_only(gpu_lib):
    rng = np.random.default_rng(3)
    binary = rng.integers(0, 256, 5000).astype(np.uint8).tobytes()
    text = rng.choice(TEXT, 300).tobytes()
    ctx = context(gpu_lib, 1)
    for data in (binary, text, b"\x00" * 10, b""):
        buf = ctx.encode_hybrid(data)
        assert ctx.decode_hybrid(buf) == data
    # all binary: no text section, flags 0 and tau 1.0 in the header
    buf = ctx.encode_hybrid(binary)
    assert buf == hybrid.pack(hybrid.segment(binary), *hybrid.pack_blob(binary), b"")
    ctx.close()
