"""svk_difference_noalloc: the difference image for callers that cannot allocate device
memory (their heap belongs to a host application, or allocation is forbidden once the
pipeline runs).  It must agree with svk_difference on the same inputs, and keep agreeing
on a second call that reuses its built-in scratch array with a different problem.

This file sorts last so that a run stopping at the first failure has run everything else.
"""
import numpy as np
import pytest
import torch

import paper_1209_5823_gb300 as svk
from _helpers import TOL_FP32, coeffs, star_pair

pytestmark = pytest.mark.gpu


def _dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


@pytest.mark.parametrize("prec", [svk.SVK_PREC_BF16X3, svk.SVK_PREC_FP16X3])
def test_noalloc_matches_workspace_entry_point_twice(prec):
    cases = [(300, 77, 19, 2, 11), (260, 40, 11, 1, 12)]  # two calls in a row, different plans
    for (W, H, L, d, seed) in cases:
        R, I = star_pair(W, H, W * H // 300, seed)
        B = svk.svk_build_basis(svk.SVK_BASIS_GAUSS, L)
        c = _dev(coeffs(B.shape[0], d, seed))
        Rt, It = _dev(R), _dev(I)
        ref = svk.svk_difference(Rt, It, B, c, d, method=svk.SVK_METHOD_BASIS, precision=prec)
        got = svk.svk_difference_noalloc(Rt, It, B, c, d, precision=prec)
        torch.cuda.synchronize()
        conv = ref.double() + It.double()  # R (x) K, the tolerance scale
        err = float((got.double() - ref.double()).abs().max() / conv.abs().max())
        assert err <= TOL_FP32


def test_noalloc_rejects_the_direct_form():
    R, I = star_pair(64, 32, 5, 3)
    B = svk.svk_build_basis(svk.SVK_BASIS_GAUSS, 7)
    c = _dev(coeffs(B.shape[0], 1, 3))
    with pytest.raises(svk.SvkError) as e:
        svk.svk_difference_noalloc(_dev(R), _dev(I), B, c, 1, precision=svk.SVK_PREC_FP32)
    assert e.value.status == svk.SVK_ERR_UNSUPPORTED
