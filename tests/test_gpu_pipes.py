"""The pipe-throughput diagnostic (hxc_pipe_rate) that gives the measured
peaks of the arithmetic-bound rooflines: sane rates and clock, and the
relation between the pipes that B300 fixes (FP64 at a small fraction of
FP32; an FP64 add no faster than an FP64 fused multiply-add)."""
import pytest

from paper_1810_11482_b300 import hxc

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def dev():
    devs = hxc.get_all_devices(2, 0)
    assert devs
    return devs[0]


def test_pipe_rates(dev):
    f64, mhz64 = hxc.pipe_rate(dev, hxc.HXC_PIPE_F64_FMA)
    add, _ = hxc.pipe_rate(dev, hxc.HXC_PIPE_F64_ADD)
    f32, mhz32 = hxc.pipe_rate(dev, hxc.HXC_PIPE_F32_FMA)
    for mhz in (mhz64, mhz32):
        assert 300.0 < mhz < 2200.0
    # per SM and clock: at most the issue width of the pipe
    per_sm = lambda ops, mhz: ops / (dev.sm_count * mhz * 1e6)
    assert 0.5 < per_sm(f64, mhz64) <= 2.05
    assert 16.0 < per_sm(f32, mhz32) <= 128.5
    assert add <= f64 * 1.05
    assert f32 > 10 * f64


def test_pipe_rate_rejects_unknown_kind(dev):
    import ctypes
    L = hxc.lib()
    x = ctypes.c_double()
    assert L.hxc_pipe_rate(dev.h, 7, ctypes.byref(x), None) == hxc.HXC_E_INVALID
