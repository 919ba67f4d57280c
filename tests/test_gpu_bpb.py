"""Coded size against the FP64 oracle at full model size (the 0.5% bar), and
the bits-per-byte cost of each weight format.

The GPU compresses a prefix of a workload's stream through the public ABI
(nc_encode); the oracle compresses the same tokens with the FP64 model.  Per
case the container's bit count must be within 0.5% of the oracle's on the
same dequantised weights (the GPU's own arithmetic) and within 0.5% of the
oracle's on the FP32 weights (the format's cost).  The GPU round trip must
be lossless.  LLM-only cases (N-gram and mixer off, p = p_tilde) show the
format's cost where the mixer cannot hide it behind the N-gram.
"""
import numpy as np
import pytest

import synthetic as S
from oracle.compress import StepConfig

import oracle_jobs

pytestmark = pytest.mark.gpu

SEED = 1
# fmt, path, rule, tokens, N-gram order (0: LLM only)
CASES = [
    ("bf16", "gemv", "paper", 512, 3),
    ("bf16", "gemv", "mixed_nll", 300, 3),
    ("bf16", "tc", "paper", 300, 3),
    ("fp8", "tc", "paper", 300, 3),
    ("fp32", "gemv", "paper", 300, 0),
    ("bf16", "tc", "paper", 300, 0),
    ("fp8", "tc", "paper", 300, 0),
]


def _cfg(rule, order):
    return StepConfig(rule=rule, order=order, use_ngram=order > 0)


@pytest.fixture(scope="module")
def oracle_bits():
    """Every oracle run of this module, started in spawned workers before the
    module's first GPU call: (case, weights) -> result."""
    pool = oracle_jobs.OraclePool(4)
    futs = {}
    for fmt, _, rule, n, order in CASES:
        toks = S.token_stream(SEED, 0, n, S.FULL.vocab)
        for wf in {fmt, "fp32"}:
            key = (wf, rule, n, order)
            if key not in futs:
                futs[key] = pool.submit(oracle_jobs.compress_recorded, S.FULL, SEED, wf, toks, (), _cfg(rule, order))
    yield futs
    pool.close()


def gpu_bits(blob, n_streams):
    off = 10
    return [int.from_bytes(blob[off + 12 * j + 4: off + 12 * j + 8], "little") for j in range(n_streams)]


@pytest.mark.parametrize("fmt,path,rule,n,order", CASES)
def test_full_model_bits_vs_oracle(gpu_lib, oracle_bits, fmt, path, rule, n, order):
    nc = gpu_lib
    shape = S.FULL
    toks = S.token_stream(SEED, 0, n, shape.vocab)
    ctx = nc.Context(nc.make_config(shape, fmt=fmt, rule=rule, path=path, ngram_order=order),
                     S.flat_weights(shape, SEED))
    blob = ctx.encode([toks])
    back = ctx.decode(blob)
    assert np.array_equal(back[0], toks)
    ctx.close()
    got = gpu_bits(blob, 1)[0]
    same = oracle_bits[(fmt, rule, n, order)].result()
    w32 = oracle_bits[("fp32", rule, n, order)].result()
    rel = (got - same["nbits"]) / same["nbits"]
    cost = (got - w32["nbits"]) / w32["nbits"]
    print(f"{fmt}/{path}/{rule}/order {order}: gpu {got / n:.4f} bits/token; oracle on {fmt} weights "
          f"{same['nbits'] / n:.4f} (rel {rel:+.2e}); on fp32 weights {w32['nbits'] / n:.4f} "
          f"(format cost {cost:+.2e}); ideal {same['ideal_bits'] / n:.4f}")
    assert abs(rel) <= 5e-3
    assert abs(cost) <= 5e-3
