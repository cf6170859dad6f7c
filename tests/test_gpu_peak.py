"""The FP32 FMA-chain rate the fused kernel's roofline is quoted against: it
must sit near the FP32 pipes' nominal rate at the clock it reports (SMs x 128
lanes x 2 FLOP x clock), well above any latency-bound figure."""
import pytest

from paper_2308_10674_gb300 import _binding as B

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


def test_fma_peak_is_near_the_nominal_rate_at_its_clock():
    tflops, mhz = B.epie_fp32_fma_peak(0, 2048)
    sms = torch.cuda.get_device_properties(0).multi_processor_count
    nominal = sms * 128 * 2 * mhz * 1e6 / 1e12
    assert 500 < mhz < 3000, mhz
    assert 0.7 * nominal < tflops < 1.1 * nominal, (tflops, nominal, mhz)
