"""The quantiser entry point that allocates nothing (nc_probs_to_cdf_noalloc).

Callers that cannot let a library call cudaMalloc use it (all HBM already
reserved by their own allocator, or no device synchronisation allowed in the
loop).  Its per-row status words sit in a fixed device array shared by all
calls, so this file runs last and checks two calls in a row against the
allocating entry point, bit for bit (the quantiser's bar: exact integers).
"""
import numpy as np
import pytest
import torch

pytestmark = pytest.mark.gpu


def _rows(V, n, seed):
    rng = np.random.default_rng(seed)
    P = rng.dirichlet(np.full(V, 0.05), size=n).astype(np.float32)
    P[0] = np.float32(1.0) / np.float32(V)                  # uniform: residual to index 0
    P[-1] = 0.0
    P[-1, V // 2] = 1.0                                      # one-hot
    return torch.from_numpy(P).cuda()


@pytest.mark.parametrize("V,n", [(49152, 6), (1003, 33)])
def test_noalloc_matches_allocating_entry_point_twice(gpu_lib, V, n):
    nc = gpu_lib
    for call in range(2):
        p = _rows(V, n, 100 * call + V)
        want = torch.empty(n, V + 1, dtype=torch.int32, device="cuda")
        got = torch.full((n, V + 1), -1, dtype=torch.int32, device="cuda")
        assert nc.nc_probs_to_cdf(p, want, 24, 1) == nc.NC_OK
        assert nc.nc_probs_to_cdf_noalloc(p, got, 24, 1) == nc.NC_OK
        assert torch.equal(got, want), f"call {call}"


def test_noalloc_status_words_are_cleared_between_calls(gpu_lib):
    nc = gpu_lib
    V, n = 4096, 4
    bad = _rows(V, n, 7)
    bad[2, 5] = float("nan")
    cdf = torch.empty(n, V + 1, dtype=torch.int32, device="cuda")
    assert nc.nc_probs_to_cdf_noalloc(bad, cdf, 24, 1) == nc.NC_ENUMERIC
    good = _rows(V, n, 8)
    want = torch.empty_like(cdf)
    assert nc.nc_probs_to_cdf(good, want, 24, 1) == nc.NC_OK
    assert nc.nc_probs_to_cdf_noalloc(good, cdf, 24, 1) == nc.NC_OK
    assert torch.equal(cdf, want)


def test_noalloc_rejects_more_rows_than_its_array(gpu_lib):
    nc = gpu_lib
    n = nc.NC_NOALLOC_MAX_ROWS + 1
    p = torch.full((n, 16), 1.0 / 16, device="cuda")
    cdf = torch.empty(n, 17, dtype=torch.int32, device="cuda")
    assert nc.nc_probs_to_cdf_noalloc(p, cdf, 24, 1) == nc.NC_EINVAL
