"""Measurement hooks of the library on the GPU: the FP32 FMA microbenchmark
that gives the all-pairs kernels' roofline its peak."""
import pytest

from gpu_helpers import library

pytestmark = pytest.mark.gpu


def test_fma_peak_counts_and_rate():
    """npsim_fma_peak reports the flops of its launch exactly (CTAs x 256
    threads x iterations x 8 chains x 2 or 4 flops) and a rate of the order of
    the SMs' FP32 lanes x 2 x clock: not far below it (the chains hide the FMA
    latency) and not above what two FMAs per lane per clock could give."""
    P = library()
    info = P.npsim_device_info()
    nominal = info["sm_count"] * 128 * 2 * 2.07e9
    iters = 1 << 14
    for packed, per_lane in ((True, 4), (False, 2)):
        fl, ms, grid = P.npsim_fma_peak(packed, iters)
        assert grid % info["sm_count"] == 0
        assert fl == grid * 256 * iters * 8 * per_lane
        rate = fl / (ms * 1e-3)
        assert 0.3 * nominal <= rate <= 2.2 * nominal, (packed, rate / nominal)
    with pytest.raises(P.NpsimError):
        P.npsim_fma_peak(True, 0)
