"""The FMA-rate probe (include/dg_probe.h) that gives the FP64/FP32 pipe
peaks of the roofline: its rates must be positive and within a plausible
band of the rates the unit counts give (152 SMs, 2 FP64 and 128 FP32 FMA
lanes per SM per clock, at most 2070 MHz), and FP32 must be far faster
than FP64 on this part."""
import pytest

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")


def test_fma_rates_plausible():
    import torch
    import paper_2301_11238_gb300 as G
    sms = torch.cuda.get_device_properties(0).multi_processor_count
    f64 = G.fma_rate(G.PREC_FP64)
    f32 = G.fma_rate(G.PREC_FP32)
    nominal64 = sms * 2070e6 * 2 * 2
    nominal32 = sms * 2070e6 * 2 * 128
    assert 0.3 * nominal64 < f64 < 1.3 * nominal64, (f64, nominal64)
    assert 0.3 * nominal32 < f32 < 1.3 * nominal32, (f32, nominal32)
    assert f32 > 16 * f64
