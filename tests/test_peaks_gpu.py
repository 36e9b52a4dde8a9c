"""Measured FMA throughput (the direct form's and the fit's roofline denominators)."""
import pytest

import paper_1209_5823_gb300 as svk

pytestmark = pytest.mark.gpu


def test_fma_peaks_are_plausible():
    fp32 = svk.svk_measure_fma_peak(False)
    fp64 = svk.svk_measure_fma_peak(True)
    # 152 SMs x 128 FP32 lanes x 2 FLOP at up to 2.07 GHz is 80.5 TFLOP/s; FP64 is a small
    # fraction of that on this part
    assert 20e12 < fp32 < 90e12
    assert 0.1e12 < fp64 < fp32
