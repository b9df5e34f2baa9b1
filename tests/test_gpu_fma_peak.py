"""The FP32 FMA rate used as the CUDA-core comparator's roofline: measured
by pcc_measure_fp32_fma, it must be positive, repeatable and below what the
SMs' FP32 lanes can do at the highest SM clock of this part (2.07 GHz)."""
import pytest

pytestmark = pytest.mark.gpu


def test_fp32_fma_rate_is_plausible(pcc_gpu):
    import torch
    sms = torch.cuda.get_device_properties(0).multi_processor_count
    ceiling = sms * 128 * 2 * 2.07e9 / 1e12  # TFLOP/s
    a = pcc_gpu.pcc_measure_fp32_fma()
    b = pcc_gpu.pcc_measure_fp32_fma()
    print(f"FP32 FMA: {a:.1f} / {b:.1f} TFLOP/s (ceiling {ceiling:.1f})")
    for v in (a, b):
        assert 0.3 * ceiling < v <= 1.02 * ceiling
    assert abs(a - b) <= 0.2 * max(a, b)
