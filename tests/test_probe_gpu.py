"""The measured FMA peaks that the FP64 roofline is quoted against."""
import pytest

pytestmark = pytest.mark.gpu


def test_fma_rates_are_plausible(hydro_lib):
    f64 = hydro_lib.hydro_fma_rate(64)
    f32 = hydro_lib.hydro_fma_rate(32)
    # a GB300 has O(1) TFLOP/s of FP64 FMA and O(10-100) TFLOP/s of FP32 FMA
    assert 0.05 < f64 < 50.0, f64
    assert 5.0 < f32 < 500.0, f32
    assert f32 > 4.0 * f64


def test_fma_rate_rejects_bad_precision(hydro_lib):
    with pytest.raises(hydro_lib.HydroError):
        hydro_lib.hydro_fma_rate(16)
