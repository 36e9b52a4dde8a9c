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
           (svk.SVK_METHOD_DIRECT, svk.SVK_PREC_FP32), (svk.SVK_METHOD_BASIS, svk.SVK_PREC_FP16X3),
           (svk.SVK_METHOD_TFORM, svk.SVK_PREC_FP32)]


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


def _batch_items(specs, pitch_pad=0, seed=0):
    """Host frames (pinned, row pitches padded by pitch_pad) of uneven sizes, kernel sizes
    and degrees, with their device call results."""
    items, expect = [], []
    for k, (W, H, L, d, N) in enumerate(specs):
        R, I, B, c = _inputs(W, H, L, d, N, seed=seed + 5 * k)
        ct = torch.from_numpy(c).cuda()
        Dh = torch.full((H, W + pitch_pad), float("nan"), dtype=torch.float32).pin_memory()
        items.append(dict(R=_host(R, pitch=W + pitch_pad), I=_host(I, pitch=W + 2 * pitch_pad), D=Dh[:, :W], basis=B,
                          coeffs=ct, degree=d))
        expect.append((R, I, B, ct, d, Dh))
    return items, expect


BATCH_SPECS = [(300, 173, 19, 2, 49), (129, 37, 25, 3, 49), (200, 61, 15, 0, 49), (64, 200, 19, 1, 30),
               (300, 173, 19, 2, 49)]


@pytest.mark.parametrize("method,prec", METHODS)
@pytest.mark.parametrize("n_bands", [1, 3])
def test_host_batch_equals_device_calls(method, prec, n_bands):
    # five frames through two staging sets (every set reused), uneven sizes, per-buffer
    # pitches: each frame equals its device call bit for bit; pitch padding stays untouched
    items, expect = _batch_items(BATCH_SPECS, pitch_pad=8 if n_bands == 3 else 0, seed=3)
    svk.svk_difference_host_batch(items, method=method, precision=prec, n_bands=n_bands)
    torch.cuda.synchronize()
    for it, (R, I, B, ct, d, Dh) in zip(items, expect):
        dev = svk.svk_difference(torch.from_numpy(R).cuda(), torch.from_numpy(I).cuda(), B, ct, d, method=method,
                                 precision=prec)
        assert torch.equal(it["D"], dev.cpu())
        W = R.shape[1]
        assert torch.isnan(Dh[:, W:]).all()


def test_host_batch_matches_oracle_with_workspace():
    specs = [(257, 61, 11, 1, 49), (130, 40, 15, 2, 49), (257, 61, 11, 1, 49)]
    items, expect = _batch_items(specs, seed=7)
    ws = torch.empty(svk.svk_host_batch_workspace_size(items), dtype=torch.uint8, device="cuda")
    svk.svk_difference_host_batch(items, n_bands=4, workspace=ws)
    torch.cuda.synchronize()
    for it, (R, I, B, ct, d, Dh) in zip(items, expect):
        ref = oracle_conv(R, B.cpu().numpy(), ct.cpu().numpy(), d)
        assert rel_err(it["D"].numpy() + I, ref) <= TOL_FP32


def test_host_batch_rejects_bad_frames():
    items, _ = _batch_items([(64, 32, 7, 1, 20), (64, 32, 7, 1, 20)])
    items[1]["degree"] = 5  # out of range in the second frame: nothing is queued
    with pytest.raises(svk.SvkError):
        svk.svk_difference_host_batch(items)
    items, _ = _batch_items([(64, 32, 7, 1, 20)])
    with pytest.raises(svk.SvkError):
        svk.svk_difference_host_batch(items, n_bands=0)
