"""Coded size against the FP64 oracle at full model size (the 0.5% bar).

The GPU compresses a prefix of a workload's stream through the public ABI
(nc_encode); the oracle compresses the same tokens with the FP64 model on the
same dequantised weights; the container's bit count must be within 0.5% of
the oracle's.  The GPU round trip must be lossless.
"""
import numpy as np
import pytest

import synthetic as S
from oracle.compress import StepConfig, compress_stream
from oracle.model import Model

pytestmark = pytest.mark.gpu


def gpu_bits(blob, n_streams):
    off = 10
    return [int.from_bytes(blob[off + 12 * j + 4: off + 12 * j + 8], "little") for j in range(n_streams)]


@pytest.mark.parametrize("fmt,path,rule,n,tol,prefill_rows", [
    ("bf16", "gemv", "paper", 512, 5e-3, 0),        # full model, single stream (first 512 tokens)
    ("bf16", "gemv", "mixed_nll", 300, 5e-3, 0),    # the differentiable update rule
    ("bf16", "tc", "paper", 300, 5e-3, 0),          # the tensor-core path
    ("bf16", "tc", "paper", 640, 5e-3, 4096),       # bench.py's configuration: prefill chunks of 512
    ("fp8", "tc", "paper", 300, None, 0),           # FP8 E4M3: reported
])
def test_full_model_bits_vs_oracle(gpu_lib, fmt, path, rule, n, tol, prefill_rows):
    nc = gpu_lib
    shape, seed = S.FULL, 1
    toks = S.token_stream(seed, 0, n, shape.vocab)
    ctx = nc.Context(nc.make_config(shape, fmt=fmt, rule=rule, path=path, prefill_rows=prefill_rows),
                     S.flat_weights(shape, seed))
    blob = ctx.encode([toks])
    back = ctx.decode(blob)
    assert np.array_equal(back[0], toks)
    ctx.close()
    got = gpu_bits(blob, 1)[0]
    ref = compress_stream(Model(shape, S.weights(shape, seed), fmt), toks, StepConfig(rule=rule))
    rel = (got - ref["nbits"]) / ref["nbits"]
    print(f"{fmt}/{path}/{rule}: gpu {got / n:.4f} bits/token, oracle {ref['nbits'] / n:.4f}, "
          f"ideal {ref['ideal_bits'] / n:.4f}, rel {rel:+.2e}")
    if tol is not None:
        assert abs(rel) <= tol
