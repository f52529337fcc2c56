"""The FMA-rate measurement behind the FP64 sweeps' arithmetic roofline."""
import pytest

import paper_1510_04995_gb300 as girih

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _build():
    import __graft_entry__
    __graft_entry__.build()


def test_fma_rates_are_plausible_and_fp32_far_above_fp64():
    """FP64: the GPU's DFMA rate per SM per clock is small on this part (a few per SM per clock
    at most); FP32: 128 FMA lanes per SM.  The measured rates must lie within those bounds at the
    device's SM count and maximum clock, and FP32 must exceed FP64 many times over."""
    import torch
    props = torch.cuda.get_device_properties(0)
    sms = props.multi_processor_count
    r64, s64 = girih.measure_fma_rate("f64")
    r32, s32 = girih.measure_fma_rate("f32")
    assert 0.02 < s64 < 1.0 and 0.02 < s32 < 1.0
    clk = 2.2e9  # above the maximum SM clock of the part
    assert 0.2 * sms * 1e9 < r64 < 64 * sms * clk
    assert r32 < 128 * sms * clk
    assert r32 > 10 * r64


def test_fma_rate_rejects_bad_arguments():
    import ctypes
    L = girih.lib()
    assert L.girih_measure_fma_rate(0, None, None, None) == 1
    x = ctypes.c_double()
    assert L.girih_measure_fma_rate(7, ctypes.byref(x), None, None) == 1
