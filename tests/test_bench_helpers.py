"""bench.py's reporting logic on CPU: the positions per forward it reports,
the dominant kernel it takes for the roofline (the largest share of the
trace, with the kinds that run beside it), and the bound chosen from the
arithmetic intensity."""
import bench


def kind(name, ms, launches=1, nbytes=1e6, flops=0.0):
    return {"name": name, "ms": ms, "launches": launches, "bytes": nbytes, "flops": flops}


def test_positions_per_forward():
    wl = bench.WORKLOADS["full_bf16_single"]
    assert bench.prefill_positions(wl, 1, 8192) == 512          # the slide of 512 bounds a chunk
    assert bench.prefill_positions(dict(wl, prefill_rows=0), 1, 8192) == 1
    assert bench.prefill_positions(wl, 1, 100) == 128           # doubles while below the longest stream


def test_dominant_kind_on_the_critical_path():
    wl = bench.WORKLOADS["full_bf16_single"]
    # the vocabulary loop paces the pass: the forwards and the N-gram pass run beside it
    trace = [kind("vocab", 26.0), kind("ngram_update", 8.0), kind("attn", 10.0), kind("gemv_gate_up", 8.0)]
    dom, beside = bench.dominant_kind(trace, wl, 1, 8192)
    assert dom["name"] == "vocab" and set(beside) == {"ngram_update", "attn", "gemv_gate_up"}
    # a forward kind that dominates: the loop and the N-gram pass run beside the forwards
    trace = [kind("vocab", 9.0), kind("ngram_update", 8.0), kind("attn", 22.0), kind("gemv_gate_up", 13.0)]
    dom, beside = bench.dominant_kind(trace, wl, 1, 8192)
    assert dom["name"] == "attn" and set(beside) == {"vocab", "ngram_update"}
    # one position per step: every kernel is on the chain
    dom, beside = bench.dominant_kind(trace, dict(wl, prefill_rows=0), 1, 8192)
    assert dom["name"] == "attn" and beside == []


def test_bound_from_intensity():
    attn = kind("attn", 0.045, launches=1, nbytes=4.3e6, flops=1.9e9)   # about 440 flop / byte
    r = bench.roofline_of(attn, "tc", "bf16", 152, 2070.0)
    assert r["bound"] == "tensor" and r["unit"] == "TFLOP/s"
    vocab = kind("vocab", 2.3, nbytes=4.0e8)
    r = bench.roofline_of(vocab, "tc", "bf16", 152, 2070.0)
    assert r["bound"] == "hbm" and r["unit"] == "GB/s"
    assert abs(r["achieved"] - 4.0e8 / 2.3e-3 / 1e9) < 1e-6
