"""The FMA microbenchmark behind the roofline's arithmetic ceilings (richm_fma_peak)."""
import pytest

from paper_2412_08076_gb300 import richm

pytestmark = pytest.mark.gpu


def test_fma_peaks_are_plausible_for_a_gb300_class_gpu():
    # nominal FP32: 152 SMs x 128 lanes x 2 flops x <= 2.07 GHz = 80.5 TFLOP/s; FP64 is
    # far lower. The bounds only catch a broken count or a kernel that does no work.
    f32 = richm.fma_peak(richm.FMA_F32)
    f32x2 = richm.fma_peak(richm.FMA_F32X2)
    f64 = richm.fma_peak(richm.FMA_F64)
    for v in (f32, f32x2):
        assert 5.0 < v < 120.0, (f32, f32x2)
    assert 0.05 < f64 < 120.0, f64
    with pytest.raises(richm.RichmError):
        richm.fma_peak(3)
