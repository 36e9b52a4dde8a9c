"""Measured FMA throughput (the direct form's and the fit's roofline denominators)."""
import pytest

import paper_1209_5823_gb300 as svk

pytestmark = pytest.mark.gpu


def test_fma_peaks_are_plausible():
    fp32 = svk.svk_measure_fma_peak(svk.SVK_FMA_FP32)
    fp32x2 = svk.svk_measure_fma_peak(svk.SVK_FMA_FP32X2)
    fp64 = svk.svk_measure_fma_peak(svk.SVK_FMA_FP64)
    # 152 SMs x 128 FP32 lanes x 2 FLOP at up to 2.07 GHz is 80.5 TFLOP/s, scalar or packed
    # (the packed form drives the same lanes); FP64 is a small fraction of that on this part
    assert 20e12 < fp32 < 90e12
    assert 20e12 < fp32x2 < 90e12
    assert 0.1e12 < fp64 < fp32
    # the old boolean form still selects FP32 / FP64
    assert 20e12 < svk.svk_measure_fma_peak(False) < 90e12
    with pytest.raises(svk.SvkError):
        svk.svk_measure_fma_peak(3)


def test_bounded_wait_gives_up_and_context_stays_usable():
    import torch
    for limit in (2_000_000, 20_000_000):  # 2 ms and 20 ms
        st, waited = svk.svk_selftest_bounded_wait(limit)
        assert st == svk.SVK_ERR_TIMEOUT
        assert limit <= waited < limit + 250_000_000  # sleep-hinted polls: coarse but bounded
    # the context still runs work afterwards
    B = svk.svk_build_basis(svk.SVK_BASIS_GAUSS, 7)
    assert torch.isfinite(B).all()


def test_bounded_wait_rejects_bad_limits():
    assert svk.svk_selftest_bounded_wait(10)[0] == svk.SVK_ERR_ARG


def test_device_status_stays_clear_after_normal_work():
    import numpy as np
    import torch
    assert svk.svk_device_status(reset=True) in (svk.SVK_OK, svk.SVK_ERR_TIMEOUT)
    assert svk.svk_device_status() == svk.SVK_OK
    R = torch.rand((70, 300), device="cuda") * 1000 + 1000
    I = torch.rand((70, 300), device="cuda") * 1000 + 1000
    B = svk.svk_build_basis(svk.SVK_BASIS_GAUSS, 19)
    c = torch.from_numpy(np.r_[np.ones((1, 6)), np.zeros((48, 6))].astype(np.float32)).cuda()
    for method, prec in [(svk.SVK_METHOD_BASIS, svk.SVK_PREC_BF16X3), (svk.SVK_METHOD_DIRECT, svk.SVK_PREC_FP32),
                         (svk.SVK_METHOD_TFORM, svk.SVK_PREC_BF16X3)]:
        svk.svk_difference(R, I, B, c, 2, method=method, precision=prec)
    # the self-test's timeout is its own: the library's status stays clear
    assert svk.svk_selftest_bounded_wait(1_000_000)[0] == svk.SVK_ERR_TIMEOUT
    assert svk.svk_device_status() == svk.SVK_OK
