"""The FMA-peak probe that serves as the FP64 kernels' roofline denominator."""

import pytest

pytestmark = pytest.mark.gpu


def test_alu_peaks_are_plausible():
    import paper_2303_08609_gb300 as weo

    f64 = weo.wilson_eo_alu_peak("f64")
    f32 = weo.wilson_eo_alu_peak("f32")
    # somewhere between a tenth of a TFlop/s and the FP32 rate; FP32 well above FP64
    assert 1e11 < f64 < f32
    assert 1e12 < f32 < 2e14
    # repeatable to a few percent
    again = weo.wilson_eo_alu_peak("f64")
    assert abs(again - f64) / f64 < 0.1
