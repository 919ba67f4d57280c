"""GPU tests of the confidence-based LLM skip (Sec. 3.7), through the C ABI:
the skip decision against the FP64 oracle's, p = p_ng on skipped steps, the
head and mixer left alone there, lossless round trips, and prefill equal to
one position per step."""
import numpy as np
import pytest
import torch

import synthetic as S
from oracle.compress import SKIP_BITS, StepConfig, StreamState, entropy_bits
from oracle.model import Model

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def nc(gpu_lib):
    return gpu_lib


def periodic(period, reps, vocab, seed):
    base = np.random.default_rng(seed).choice(vocab, size=period, replace=False)
    return np.tile(base, reps).astype(np.int32)


@pytest.mark.parametrize("rule", ["paper", "mixed_nll"])
def test_skip_decisions_and_state_vs_oracle(nc, rule):
    """Small FP32 model, a periodic stream (the N-gram grows confident):
    where the oracle's entropy is clear of the 1.5-bit threshold (1e-3), the
    GPU skips exactly when the oracle does; skipped steps give p = p_ng
    bit for bit; p and the head / mixer state follow the oracle."""
    shape, seed = S.SMALL, 0
    toks = periodic(6, 20, shape.vocab, 31)
    V = shape.vocab
    ctx = nc.Context(nc.make_config(shape, fmt="fp32", rule=rule, warmup=12, skip=True), S.flat_weights(shape, seed))
    ref = StreamState.new(Model(shape, S.weights(shape, seed), "fp32"), StepConfig(warmup=12, rule=rule, skip=True))
    bufs = {k: torch.empty(1, V, device="cuda") for k in ("z", "pt", "png", "p")}
    ctx.stream_open(1, len(toks))
    n_skip, clear, agree = 0, 0, True
    b_prev, _, _ = ctx.stream_state(1)
    for i, t in enumerate(toks):
        ctx.step_probe([1], z=bufs["z"], p_tilde=bufs["pt"], p_ng=bufs["png"], p=bufs["p"])
        p, png = bufs["p"][0].cpu().numpy(), bufs["png"][0].cpu().numpy()
        ref.predict()
        h = entropy_bits(ref._cur[2])
        ctx.update_bias([1], [int(t)])
        ref.update(int(t))
        b_now, _, _ = ctx.stream_state(1)
        gpu_skip = np.array_equal(b_now, b_prev)     # the head learns from every unskipped token
        b_prev = b_now
        if gpu_skip:
            assert np.array_equal(p, png)            # p = p_ng, bit for bit
        agree &= gpu_skip == (h < SKIP_BITS)
        if abs(h - SKIP_BITS) > 1e-3:
            clear += 1
            assert gpu_skip == (h < SKIP_BITS), (i, h)
            if agree:
                np.testing.assert_allclose(p, ref._cur[3], rtol=2e-4, atol=1e-9)
        n_skip += gpu_skip
    assert n_skip > 40 and clear >= len(toks) - 3
    b, th, n = ctx.stream_state(1)
    assert n == len(toks)
    if agree:   # the same decisions everywhere: the same updates were applied
        np.testing.assert_allclose(b, ref.head.b, rtol=0, atol=2e-6)
        logw = ref.theta if rule == "mixed_nll" else ref.mixer.logw
        np.testing.assert_allclose(th, logw, rtol=1e-4, atol=1e-4)
    ctx.close()


@pytest.mark.parametrize("fmt,path", [("fp32", "gemv"), ("bf16", "tc")])
def test_skip_roundtrip_and_prefill(nc, fmt, path):
    """Ragged streams mixing periodic and Zipf/Markov tokens: lossless with
    the skip, prefill intervals equal to one position per step, and a
    container flagged with the skip is refused by a context without it."""
    shape, seed = S.SMALL, 5
    w = S.flat_weights(shape, seed)
    streams = [np.concatenate([periodic(5, 40, shape.vocab, 40), S.token_stream(seed, 0, 300, shape.vocab)]),
               periodic(9, 30, shape.vocab, 41), S.token_stream(seed, 2, 77, shape.vocab)]
    plain = nc.Context(nc.make_config(shape, fmt=fmt, path=path, warmup=20, max_streams=3, skip=True), w)
    pre = nc.Context(nc.make_config(shape, fmt=fmt, path=path, warmup=20, max_streams=3, skip=True,
                                    prefill_rows=512), w)
    blob = pre.encode(streams)
    assert blob == plain.encode(streams)
    back = plain.decode(blob)
    for a, b in zip(streams, back):
        assert np.array_equal(a, b)
    off = nc.Context(nc.make_config(shape, fmt=fmt, path=path, warmup=20, max_streams=3), w)
    with pytest.raises(nc.NcError):
        off.decode(blob)
    for c in (plain, pre, off):
        c.close()
