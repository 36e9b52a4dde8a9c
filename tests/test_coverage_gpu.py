"""Every output pixel written exactly where it belongs: outputs are poisoned with NaN before
each call (with pitch padding that must stay NaN), on ragged frames whose width is not a
multiple of the 128-pixel tile and whose height is not a multiple of any block height."""
import numpy as np
import pytest
import torch

import paper_1209_5823_gb300 as svk
from _helpers import coeffs, star_pair

pytestmark = pytest.mark.gpu

PAD = 24


def _poisoned(H, W, device="cuda", pinned=False):
    if device == "cuda":
        big = torch.full((H, W + PAD), float("nan"), dtype=torch.float32, device="cuda")
    else:
        big = torch.full((H, W + PAD), float("nan"), dtype=torch.float32).pin_memory() if pinned else \
            torch.full((H, W + PAD), float("nan"), dtype=torch.float32)
    return big, big[:, :W]


def _check(big, W):
    assert not torch.isnan(big[:, :W]).any(), "unwritten output pixels"
    assert torch.isnan(big[:, W:]).all(), "writes past the row end"


def _inputs(W, H, L, N, d, seed):
    R, I = star_pair(W, H, max(3, W * H // 300), 1300 + seed)
    B = svk.svk_build_basis(svk.SVK_BASIS_GAUSS, L)[:N].contiguous()
    c = torch.from_numpy(coeffs(N, d, 30 + seed)).cuda()
    return R, I, B, c


@pytest.mark.parametrize("method,prec", [
    (svk.SVK_METHOD_DIRECT, svk.SVK_PREC_FP32),
    (svk.SVK_METHOD_BASIS, svk.SVK_PREC_BF16X3),
    (svk.SVK_METHOD_BASIS, svk.SVK_PREC_FP16X3),
    (svk.SVK_METHOD_BASIS, svk.SVK_PREC_BF16),
    (svk.SVK_METHOD_TFORM, svk.SVK_PREC_BF16X3),
    (svk.SVK_METHOD_TFORM, svk.SVK_PREC_FP32),
])
@pytest.mark.parametrize("W,H,L", [(300, 173, 19), (129, 37, 25), (7, 5, 11), (1000, 3, 31)])
def test_device_call_writes_every_pixel(method, prec, W, H, L):
    R, I, B, c = _inputs(W, H, L, 49, 2, W + H)
    big, out = _poisoned(H, W)
    svk.svk_difference(torch.from_numpy(R).cuda(), torch.from_numpy(I).cuda(), B, c, 2, method=method,
                       precision=prec, out=out)
    torch.cuda.synchronize()
    _check(big, W)


def test_host_call_writes_every_pixel():
    W, H, L = 300, 173, 19
    R, I, B, c = _inputs(W, H, L, 49, 2, 7)
    big, out = _poisoned(H, W, device="cpu", pinned=True)
    Rh = torch.zeros((H, W + PAD), dtype=torch.float32).pin_memory()
    Ih = torch.zeros((H, W + PAD), dtype=torch.float32).pin_memory()
    Rh[:, :W] = torch.from_numpy(R)
    Ih[:, :W] = torch.from_numpy(I)
    svk.svk_difference_host(Rh[:, :W], Ih[:, :W], B, c, 2, out=out, n_bands=5)
    torch.cuda.synchronize()
    _check(big, W)


def test_batch_writes_every_pixel():
    items, bigs = [], []
    for k, (W, H, L, d) in enumerate([(300, 173, 19, 2), (129, 37, 25, 3), (200, 61, 15, 0)]):
        R, I, B, c = _inputs(W, H, L, 49, d, 40 + k)
        big, out = _poisoned(H, W)
        bigs.append((big, W))
        items.append(dict(R=torch.from_numpy(R).cuda(), I=torch.from_numpy(I).cuda(), D=out, basis=B, coeffs=c,
                          degree=d))
    svk.svk_difference_batch(items, precision=svk.SVK_PREC_BF16X3)
    torch.cuda.synchronize()
    for big, W in bigs:
        _check(big, W)
