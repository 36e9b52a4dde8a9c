"""The difference image from host buffers (svk_difference_host): row bands copied in,
computed and copied out on three streams.  Its result must equal the device call bit for
bit (same blocks, same arithmetic) and the FP64 oracle within the parity bar."""
import numpy as np
import pytest
import torch

import paper_1209_5823_gb300 as svk
from _helpers import TOL_FP32, coeffs, oracle_conv, rel_err, star_pair

pytestmark = pytest.mark.gpu


def _inputs(W, H, L, d, N, seed=0):
    R, I = star_pair(W, H, max(3, W * H // 300), 900 + seed + W + H)
    B = svk.svk_build_basis(svk.SVK_BASIS_GAUSS, L)[:N].contiguous()
    c = coeffs(N, d, 21 + seed)
    return R, I, B, c


def _host(a, pitch=None, pinned=True):
    H, W = a.shape
    p = W if pitch is None else pitch
    t = torch.zeros((H, p), dtype=torch.float32, pin_memory=pinned)[:, :W]
    t.copy_(torch.from_numpy(a))
    return t


METHODS = [(svk.SVK_METHOD_BASIS, svk.SVK_PREC_BF16X3), (svk.SVK_METHOD_TFORM, svk.SVK_PREC_BF16X3),
           (svk.SVK_METHOD_DIRECT, svk.SVK_PREC_FP32), (svk.SVK_METHOD_BASIS, svk.SVK_PREC_FP16X3)]


@pytest.mark.parametrize("method,prec", METHODS)
@pytest.mark.parametrize("n_bands", [1, 3, 8, 16])
def test_host_bands_equal_device_call(method, prec, n_bands):
    W, H, L, d, N = 300, 173, 19, 2, 49
    R, I, B, c = _inputs(W, H, L, d, N)
    ct = torch.from_numpy(c).cuda()
    dev = svk.svk_difference(torch.from_numpy(R).cuda(), torch.from_numpy(I).cuda(), B, ct, d, method=method,
                             precision=prec)
    Dh = svk.svk_difference_host(_host(R), _host(I), B, ct, d, method=method, precision=prec, n_bands=n_bands)
    torch.cuda.synchronize()
    assert torch.equal(Dh, dev.cpu())


def test_host_matches_oracle_with_pitch_and_pageable_memory():
    W, H, L, d, N = 257, 61, 11, 1, 49
    R, I, B, c = _inputs(W, H, L, d, N, seed=1)
    ref = oracle_conv(R, B.cpu().numpy(), c, d)
    ct = torch.from_numpy(c).cuda()
    for pinned in (True, False):
        Rh, Ih = _host(R, pitch=272, pinned=pinned), _host(I, pitch=272, pinned=pinned)
        ws = torch.empty(svk.svk_host_workspace_size(svk.SVK_METHOD_BASIS, svk.SVK_PREC_BF16X3, W, H, N, L, d),
                         dtype=torch.uint8, device="cuda")
        Dh = svk.svk_difference_host(Rh, Ih, B, ct, d, n_bands=5, workspace=ws)
        torch.cuda.synchronize()
        assert rel_err(Dh.numpy() + I, ref) <= TOL_FP32


def test_host_tiny_frames_and_many_bands():
    for (W, H) in [(1, 1), (5, 3), (130, 7)]:
        R, I, B, c = _inputs(W, H, 7, 1, 20, seed=2)
        ct = torch.from_numpy(c).cuda()
        dev = svk.svk_difference(torch.from_numpy(R).cuda(), torch.from_numpy(I).cuda(), B, ct, 1,
                                 method=svk.SVK_METHOD_BASIS, precision=svk.SVK_PREC_BF16X3)
        Dh = svk.svk_difference_host(_host(R), _host(I), B, ct, 1, n_bands=16)
        torch.cuda.synchronize()
        assert torch.equal(Dh, dev.cpu())


def test_host_rejects_bad_arguments():
    R, I, B, c = _inputs(64, 32, 7, 1, 20)
    ct = torch.from_numpy(c).cuda()
    with pytest.raises(svk.SvkError):
        svk.svk_difference_host(_host(R), _host(I), B, ct, 1, n_bands=0)
    with pytest.raises(svk.SvkError):
        svk.svk_difference_host(_host(R), _host(I), B, ct, 1, method=svk.SVK_METHOD_DIRECT,
                                precision=svk.SVK_PREC_BF16X3)
