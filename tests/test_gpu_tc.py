"""GPU tests of the tensor-core (tcgen05) path, through the C ABI.

* the GEMM against an FP64 product of the same BF16 / E4M3 operands;
* results independent of the batch tile and of the batch size (bit-exact);
* the whole step on the tensor-core path: logits against the FP64 oracle,
  batch invariance, and a lossless round trip.
"""
import numpy as np
import pytest
import torch

import synthetic as S
from oracle import numerics
from oracle.compress import StepConfig, StreamState
from oracle.model import Model

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def nc(gpu_lib):
    return gpu_lib


def bf16_bits(a32):
    """float32 -> bfloat16 bit patterns (oracle rounding) as int16 numpy."""
    r = numerics.bf16_round(a32)
    return (r.view(np.uint32) >> 16).astype(np.uint16).view(np.int16), r.astype(np.float64)


def e4m3_bytes(q):
    """Exact E4M3 values -> their byte codes."""
    grid = numerics._GRID
    idx = np.searchsorted(grid, np.abs(q))
    assert np.all(grid[idx] == np.abs(q))
    return (idx | np.where(q < 0, 0x80, 0)).astype(np.uint8)


@pytest.mark.parametrize("M,K", [(960, 576), (384, 688), (128, 1536)])
@pytest.mark.parametrize("N", [1, 7, 64, 300])
def test_gemm_bf16_vs_fp64(nc, M, K, N):
    rng = np.random.default_rng(M * 7 + N)
    Wb, W64 = bf16_bits(rng.normal(0, 0.02, (M, K)).astype(np.float32))
    Xb, X64 = bf16_bits(rng.normal(0, 1.0, (N, K)).astype(np.float32))
    W = torch.from_numpy(Wb).cuda().view(torch.bfloat16)
    X = torch.from_numpy(Xb).cuda().view(torch.bfloat16)
    ref = X64 @ W64.T
    outs = []
    for bn in (32, 64, 128, 256):
        Y = torch.full((N, M), float("nan"), device="cuda")
        assert nc.nc_gemm_tc(W, X, Y, bn=bn) == nc.NC_OK
        outs.append(Y.cpu().numpy())
    np.testing.assert_allclose(outs[0], ref, rtol=1e-4, atol=1e-4 * np.abs(ref).max())
    for o in outs[1:]:
        assert np.array_equal(o, outs[0])           # the batch tile never changes a result
    # a row computed alone equals the same row inside the batch
    Y1 = torch.empty((1, M), device="cuda")
    assert nc.nc_gemm_tc(W, X[N - 1:N].contiguous(), Y1, bn=32) == nc.NC_OK
    assert np.array_equal(Y1.cpu().numpy()[0], outs[0][N - 1])


@pytest.mark.parametrize("N", [3, 130])
def test_gemm_fp8_vs_fp64(nc, N):
    M, K = 576, 1536
    rng = np.random.default_rng(N)
    qw, sw = numerics.fp8_rowwise(rng.normal(0, 0.02, (M, K)).astype(np.float32))
    qx, sx = numerics.fp8_rowwise(rng.normal(0, 1.0, (N, K)).astype(np.float32))
    W = torch.from_numpy(e4m3_bytes(qw)).cuda()
    X = torch.from_numpy(e4m3_bytes(qx)).cuda()
    Y = torch.empty((N, M), device="cuda")
    assert nc.nc_gemm_tc(W, X, Y, bn=64, w_scale=torch.from_numpy(sw).cuda(),
                         x_scale=torch.from_numpy(sx).cuda(), fp8=True) == nc.NC_OK
    ref = (qx @ qw.T) * sx.astype(np.float64)[:, None] * sw.astype(np.float64)[None, :]
    np.testing.assert_allclose(Y.cpu().numpy(), ref, rtol=1e-4, atol=1e-4 * np.abs(ref).max())


def test_tc_path_logits_full_model(nc):
    """Full model on the tensor-core path (BF16 weights, BF16 activations
    into each GEMM): logits of the first steps within 3e-2 of the FP64
    oracle on the FP32 weights."""
    shape, seed = S.FULL, 1
    toks = S.token_stream(seed, 0, 4, shape.vocab)
    ctx = nc.Context(nc.make_config(shape, fmt="bf16", path="tc"), S.flat_weights(shape, seed))
    z = torch.empty(1, shape.vocab, device="cuda")
    ctx.stream_open(0, 4)
    ref = StreamState.new(Model(shape, S.weights(shape, seed), "fp32"), StepConfig())
    err = 0.0
    for t in toks:
        ctx.step_probe([0], z=z)
        ref.predict()
        err = max(err, float(np.max(np.abs(z[0].cpu().numpy() - ref._cur[0]))))
        ctx.update_bias([0], [int(t)])
        ref.update(int(t))
    print(f"tc bf16 logits vs oracle(fp32) max abs err {err:.3e}")
    assert err <= 3e-2
    ctx.close()


@pytest.mark.parametrize("fmt", ["bf16", "fp8"])
def test_tc_path_batch_invariance_and_roundtrip(nc, fmt):
    """Streams stepped together on the tensor-core path give bit-identical
    CDFs to each stream stepped alone (different max_streams, so also a
    different tuned batch tile); encode / decode of ragged streams is
    lossless."""
    shape, seed = S.SMALL, 4
    streams = [S.token_stream(seed, j, 12, shape.vocab) for j in range(3)]
    w = S.flat_weights(shape, seed)
    ctxB = nc.Context(nc.make_config(shape, fmt=fmt, warmup=4, max_streams=40, path="tc"), w)
    for j in range(3):
        ctxB.stream_open(j, 12)
    batched = []
    for k in range(12):
        batched.append(ctxB.step_cdf(np.arange(3)).copy())
        ctxB.update_bias(np.arange(3), [int(s[k]) for s in streams])
    for j in range(3):
        ctxB.stream_close(j)
    ctx1 = nc.Context(nc.make_config(shape, fmt=fmt, warmup=4, max_streams=1, path="tc"), w)
    for j in range(3):
        ctx1.stream_open(0, 12)
        for k in range(12):
            c = ctx1.step_cdf([0])
            assert np.array_equal(c[0], batched[k][j]), (j, k)
            ctx1.update_bias([0], [int(streams[j][k])])
        ctx1.stream_close(0)
    ctx1.close()
    ragged = [S.token_stream(seed, 10 + j, n, shape.vocab) for j, n in enumerate([50, 3, 17])]
    blob = ctxB.encode(ragged)
    back = ctxB.decode(blob)
    for a, b in zip(ragged, back):
        assert np.array_equal(a, b)
    ctxB.close()
