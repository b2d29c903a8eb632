"""The FMA-rate calibration behind the float64 roofline figure measures a
plausible rate on the device: float32 far above float64."""
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import paper_2412_05824_gb300 as tfl  # noqa: E402


def test_fma_peak_rates():
    f64 = tfl.fma_peak("complex128", 0.2)
    f32 = tfl.fma_peak("complex64", 0.2)
    assert 0.05 < f64 < 200.0, f64
    assert 1.0 < f32 < 500.0, f32
    assert f32 > 4 * f64
