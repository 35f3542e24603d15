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


def test_bounded_wait_expires_and_reports_timeout(hydro_lib):
    """A device wait whose barrier nothing completes gives up after its bound
    and reports HYDRO_ERR_TIMEOUT; the context stays usable afterwards (the
    failure is detected without a fault, as the batched kernel's waits on its
    bulk copies would report one)."""
    import numpy as np
    from paper_2503_04428_gb300 import workloads as wl
    st, secs = hydro_lib.hydro_wait_probe()
    assert st == hydro_lib.HYDRO_ERR_TIMEOUT
    assert 0.0 < secs < 60.0, secs
    w = wl.tubes(4, seed=3, lo=256, hi=600)
    b = hydro_lib.Batch(w["lengths"], w["gamma"], precision=32)
    b.set_state(w["U"])
    b.run(2, 0.8)
    assert np.isfinite(b.get_state()).all()
