"""The measured FMA peaks the ALU-bound rooflines divide by (adr_measure_peak)."""
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

from paper_2303_15861_gb300 import adr, build_lib  # noqa: E402

build_lib.build()
adr.load_library()


def test_fma_peaks_are_positive_and_ordered():
    fp64 = adr.adr_measure_peak("fp64_fma", 64)
    fp32 = adr.adr_measure_peak("fp32_fma", 1024)
    assert 0.0 < fp64 < fp32
    # 152 SMs x 128 FP32 lanes x 2 flops at up to 2.07 GHz is 80.5 TFLOP/s
    assert fp32 < 85.0
