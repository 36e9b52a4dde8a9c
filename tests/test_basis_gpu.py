"""Parity of the tensor-core basis form (tcgen05, implicit im2col) with the FP64 oracle."""
import numpy as np
import pytest
import torch

import paper_1209_5823_gb300 as svk
from _helpers import TOL_FP32, coeffs, oracle_conv, rel_err, star_pair

pytestmark = pytest.mark.gpu

SPLIT = [svk.SVK_PREC_BF16X3, svk.SVK_PREC_FP16X3]
# Plain BF16 operands (8-bit significands) with FP32 accumulation: the error bound is
# a measured number (2.2e-3 at 4096^2, L = 25); the test only guards against gross errors.
TOL_BF16 = 2e-2


def _dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def _run(W, H, L, d, N, prec, seed=0, pitch=None, kind=svk.SVK_BASIS_GAUSS, diff=False):
    R, I = star_pair(W, H, max(3, W * H // 300), 200 + seed + W + H)
    B = svk.svk_build_basis(kind, L)[:N].contiguous()
    c = coeffs(N, d, 11 + seed)
    ref = oracle_conv(R, B.cpu().numpy(), c, d)
    if pitch is None:
        Rt = _dev(R)
    else:
        Rt = torch.zeros((H, pitch), dtype=torch.float32, device="cuda")[:, :W]
        Rt[:] = _dev(R)
    if diff:
        out = svk.svk_difference(Rt, _dev(I), B, _dev(c), d, method=svk.SVK_METHOD_BASIS, precision=prec)
        got = out.cpu().numpy() + I
    else:
        out = svk.svk_convolve(Rt, B, _dev(c), d, method=svk.SVK_METHOD_BASIS, precision=prec)
        got = out.cpu().numpy()
    torch.cuda.synchronize()
    return rel_err(got, ref)


@pytest.mark.parametrize("prec", SPLIT)
@pytest.mark.parametrize("W,H,L,d,N", [
    (256, 256, 11, 1, 49),   # the 256x256 star-field case
    (300, 77, 19, 2, 49),    # ragged tiles, L = 19 (2-row blocks)
    (260, 40, 25, 3, 49),
    (130, 23, 31, 2, 49),    # largest kernel: 1-row blocks
    (140, 33, 9, 1, 20),     # packed tails of 1 tap, one full tap group per row
    (200, 41, 17, 2, 49),    # packed tails of 1 tap, two full groups
    (150, 61, 25, 2, 10),    # packed tails of 1 tap, three full groups (cross-row K step)
    (47, 38, 7, 3, 5),       # odd pitch, few stamps, 3+ rows per block
    (1, 1, 5, 2, 49),        # 1x1 frame
    (5, 300, 15, 1, 49),     # L > W
])
def test_split_precision_matches_oracle(W, H, L, d, N, prec):
    assert _run(W, H, L, d, N, prec) <= TOL_FP32


@pytest.mark.parametrize("prec", SPLIT)
@pytest.mark.parametrize("N,L,d", [
    (50, 9, 2),    # 5-row blocks, 52 exact accumulator slots per output row
    (52, 11, 3),   # 4-row blocks, 52 exact slots
    (53, 13, 1),   # four 16-column loads per output row
    (56, 9, 3),
])
def test_stamp_counts_50_to_56(N, L, d, prec):
    assert _run(230, 47, L, d, N, prec, seed=N, kind=svk.SVK_BASIS_DELTA) <= TOL_FP32


@pytest.mark.parametrize("prec", SPLIT)
@pytest.mark.parametrize("N", [100, 121])
def test_wide_delta_basis(N, prec):
    # 100 / 121 stamps of an 11 x 11 delta basis: 2-row and 1-row blocks
    assert _run(200, 50, 11, 2, N, prec, kind=svk.SVK_BASIS_DELTA) <= TOL_FP32


@pytest.mark.parametrize("prec", SPLIT)
def test_difference_fused_and_padded_pitch(prec):
    assert _run(333, 45, 19, 2, 49, prec, pitch=352, diff=True) <= TOL_FP32


def test_plain_bf16_error_is_bounded():
    err = _run(256, 256, 11, 1, 49, svk.SVK_PREC_BF16)
    assert err <= TOL_BF16


def test_delta_basis_paper_workload():
    # delta basis, L = 7 (N = 49), second-order polynomials: the paper's measured case
    assert _run(300, 60, 7, 2, 49, svk.SVK_PREC_BF16X3, kind=svk.SVK_BASIS_DELTA) <= TOL_FP32


def test_repeatable_bitwise():
    R, _ = star_pair(300, 90, 60, 1)
    B = svk.svk_build_basis(svk.SVK_BASIS_GAUSS, 19)
    c = _dev(coeffs(49, 2, 3))
    Rt = _dev(R)
    a = svk.svk_convolve(Rt, B, c, 2, method=svk.SVK_METHOD_BASIS, precision=svk.SVK_PREC_BF16X3)
    b = svk.svk_convolve(Rt, B, c, 2, method=svk.SVK_METHOD_BASIS, precision=svk.SVK_PREC_BF16X3)
    assert torch.equal(a, b)
