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


def test_l2_read_bandwidth_is_plausible():
    """The L2 -> SM read probe: above the HBM copy bandwidth's order of magnitude
    floor and below any plausible on-chip rate, and repeatable."""
    import paper_2303_08609_gb300 as weo

    bw = weo.wilson_eo_l2_peak()
    assert 1e12 < bw < 1e14
    again = weo.wilson_eo_l2_peak()
    assert abs(again - bw) / bw < 0.15
