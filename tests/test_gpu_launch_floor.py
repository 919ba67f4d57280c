"""GPU test of the launch-floor diagnostic: a captured chain of empty kernels
with programmatic dependent launch, the floor under the decode step's chain
of dependent kernels."""
import pytest

pytestmark = pytest.mark.gpu


def test_launch_chain_floor(gpu_lib):
    short = gpu_lib.nc_launch_chain_floor(0, 16, 152, 256, 5)
    long = gpu_lib.nc_launch_chain_floor(0, 216, 152, 256, 5)
    for us in (short, long):
        assert 0.05 < us < 200.0                 # microseconds per link
