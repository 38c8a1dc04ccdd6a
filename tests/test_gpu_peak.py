"""The measured FP32 FMA peak that bench.py reports as the cluster loop's roofline denominator:
it must land near the unit-count figure (SMs x 128 FP32 lanes x 2 flops x SM clock), below it
by the loop overhead and any clock drop under load, never above it by more than timing noise."""
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def test_fma_peak_is_near_the_unit_count_figure():
    from paper_2602_13805_gb300 import build, pdf
    pdf.load(build.build())
    tf = pdf.pdf_fp32_fma_peak(5)
    sms = torch.cuda.get_device_properties(0).multi_processor_count
    upper = sms * 128 * 2 * 2.2e9 / 1e12          # above any SM clock this part runs at
    print("FP32 FMA peak", tf, "TFLOP/s; ceiling at 2.2 GHz", upper)
    assert 0.4 * upper < tf < 1.02 * upper
