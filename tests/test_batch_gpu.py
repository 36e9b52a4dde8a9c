"""Batched frames (grouped persistent launches) and autotuned plans: every frame of a
batch must equal the single-frame result, also when the batch is replayed from a CUDA
graph, and the tuned plans must keep parity with the oracle."""
import numpy as np
import pytest
import torch

import paper_1209_5823_gb300 as svk
import starfield
from _helpers import TOL_FP32, coeffs, oracle_conv, rel_err, star_pair

pytestmark = pytest.mark.gpu


def _dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def _items(specs, seed0=300):
    items, bases = [], {}
    for k, (W, H, L, d) in enumerate(specs):
        R, I = star_pair(W, H, max(3, W * H // 400), seed0 + k)
        if L not in bases:
            bases[L] = svk.svk_build_basis(svk.SVK_BASIS_GAUSS, L)
        B = bases[L]
        items.append(dict(R=_dev(R), I=_dev(I), D=torch.full((H, W), float("nan"), device="cuda"), basis=B,
                          coeffs=_dev(coeffs(B.shape[0], d, seed0 + k)), degree=d, Rn=R, In=I))
    return items


SPECS = [(300, 77, 19, 2), (128, 300, 15, 0), (257, 64, 19, 3), (400, 50, 31, 1), (96, 96, 15, 1), (5, 200, 19, 2)]


@pytest.mark.parametrize("prec", [svk.SVK_PREC_BF16X3, svk.SVK_PREC_BF16])
def test_batch_equals_single_frame_calls(prec):
    items = _items(SPECS)
    svk.svk_difference_batch(items, precision=prec)
    torch.cuda.synchronize()
    for it in items:
        ref = svk.svk_difference(it["R"], it["I"], it["basis"], it["coeffs"], it["degree"],
                                 method=svk.SVK_METHOD_BASIS, precision=prec)
        assert torch.equal(it["D"], ref)


def test_batch_matches_oracle_and_graph_replay():
    items = _items(SPECS[:4], seed0=400)
    ws = torch.empty(svk.svk_batch_workspace_size(items), dtype=torch.uint8, device="cuda")
    s = torch.cuda.Stream()
    with torch.cuda.stream(s):
        svk.svk_difference_batch(items, workspace=ws)  # warm-up outside the capture
    torch.cuda.synchronize()
    g = torch.cuda.CUDAGraph()
    for it in items:
        it["D"].fill_(float("nan"))
    with torch.cuda.graph(g, stream=s):
        svk.svk_difference_batch(items, workspace=ws, stream=s)
    g.replay()
    torch.cuda.synchronize()
    for it in items:
        ref = oracle_conv(it["Rn"], it["basis"].cpu().numpy(), it["coeffs"].cpu().numpy(), it["degree"])
        got = it["D"].cpu().numpy().astype(np.float64) + it["In"]
        assert rel_err(got, ref) <= TOL_FP32


def test_autotune_keeps_parity():
    G, stages = svk.svk_autotune(49, 19, 2, svk.SVK_PREC_BF16X3, W=1024, H=256)
    assert 1 <= G <= 5 and stages in (4, 8, 16)
    R, I = star_pair(300, 77, 70, 7)
    B = svk.svk_build_basis(svk.SVK_BASIS_GAUSS, 19)
    c = coeffs(49, 2, 7)
    ref = oracle_conv(R, B.cpu().numpy(), c, 2)
    out = svk.svk_convolve(_dev(R), B, _dev(c), 2, method=svk.SVK_METHOD_BASIS, precision=svk.SVK_PREC_BF16X3)
    assert rel_err(out.cpu().numpy(), ref) <= TOL_FP32


def test_batch_rejects_a_bad_frame():
    items = _items(SPECS[:2], seed0=500)
    items[1]["degree"] = 5
    with pytest.raises(svk.SvkError) as e:
        svk.svk_difference_batch(items)
    assert e.value.status == svk.SVK_ERR_ARG and "frame 1" in str(e.value)
