"""Failure detection without a GPU fault.

* A bounded device wait that gives up (an mbarrier nothing arrives on, with a
  short poll limit) is reported as NC_ETIMEOUT and poisons the context; later
  calls return NC_ESTATE; the device stays usable for a new context.
* Device allocations that fail (the NC24_FAIL_ALLOC_AFTER test hook makes the
  n-th allocation fail as an out-of-memory device would) return NC_ENOMEM
  from context creation and from stream opening, and release every byte they
  held: the device's free memory returns to where it was.
"""
import numpy as np
import pytest
import torch

import synthetic as S

pytestmark = pytest.mark.gpu


def test_bounded_wait_times_out_and_poisons(gpu_lib):
    nc = gpu_lib
    shape = S.SMALL
    w = S.flat_weights(shape, 0)
    ctx = nc.Context(nc.make_config(shape, fmt="bf16", path="tc"), w)
    for polls in (0, 1000):
        if polls:
            ctx = nc.Context(nc.make_config(shape, fmt="bf16", path="tc"), w)
        with pytest.raises(nc.NcError) as e:
            ctx.selftest_wait(polls)
        assert e.value.status == nc.NC_ETIMEOUT
        with pytest.raises(nc.NcError) as e:
            ctx.stream_open(0, 8)
        assert e.value.status == nc.NC_ESTATE
        ctx.close()
    # the device is still usable: a fresh context codes and decodes
    ctx = nc.Context(nc.make_config(shape, fmt="bf16", path="tc"), w)
    toks = S.token_stream(0, 0, 40, shape.vocab)
    assert np.array_equal(ctx.decode(ctx.encode([toks]))[0], toks)
    ctx.close()


def _free_bytes():
    torch.cuda.synchronize()
    return torch.cuda.mem_get_info()[0]


@pytest.mark.parametrize("fail_after", [0, 1, 3, 17, 40, 70])
def test_allocation_failure_returns_enomem_without_leak(gpu_lib, monkeypatch, fail_after):
    nc = gpu_lib
    shape = S.SMALL
    w = S.flat_weights(shape, 0)
    cfg = nc.make_config(shape, fmt="bf16", path="tc", prefill_rows=256, max_streams=8)
    # a successful creation first (every kernel it launches is then loaded)
    ctx = nc.Context(cfg, w)
    ctx.close()
    torch.cuda.empty_cache()
    before = _free_bytes()
    monkeypatch.setenv("NC24_FAIL_ALLOC_AFTER", str(fail_after))
    try:
        ctx = nc.Context(cfg, w)
    except nc.NcError as e:
        assert e.status == nc.NC_ENOMEM
    else:
        # creation needed fewer allocations: the next ones (the streams'
        # buffers, 13 per stream) fail
        with pytest.raises(nc.NcError) as e:
            for sid in range(8):
                ctx.stream_open(sid, 1000)
        assert e.value.status == nc.NC_ENOMEM
        ctx.close()
    monkeypatch.delenv("NC24_FAIL_ALLOC_AFTER")
    assert _free_bytes() == before
    # and the device still works
    ctx = nc.Context(cfg, w)
    toks = S.token_stream(0, 1, 30, shape.vocab)
    assert np.array_equal(ctx.decode(ctx.encode([toks]))[0], toks)
    ctx.close()
