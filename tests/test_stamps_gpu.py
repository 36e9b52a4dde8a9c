"""Stamp selection on the device (svk_select_stamps) against the oracle: the stamp list is
index work, so the comparison is exact (same centres, same order, same peak count)."""
import numpy as np
import pytest
import torch

import paper_1209_5823_gb300 as svk
import starfield
from oracle import stamps as ostamps

pytestmark = pytest.mark.gpu

SKY = 1000.0


def _field(W, H, n_stars, seed):
    g = starfield.rng(seed)
    cat = starfield.star_catalog(W, H, n_stars, g)
    return starfield.add_noise(starfield.render(cat, W, H, sky=SKY), 30.0, g).astype(np.float32)


def _run(R, sky, thr, sat, margin, rad, frac, max_stamps):
    Rt = torch.from_numpy(np.ascontiguousarray(R)).cuda()
    xy, counts = svk.svk_select_stamps(Rt, sky, thr, sat, margin, rad, frac, max_stamps)
    torch.cuda.synchronize()
    n, n_peaks = counts.tolist()
    return xy[:n].cpu().numpy(), n_peaks


def _check(R, *args):
    got, gp = _run(R, *args)
    want, wp = ostamps.select_stamps(R, *args)
    assert gp == wp
    assert got.tolist() == want.tolist()
    return want


@pytest.mark.parametrize("W,H,n_stars,seed", [(333, 517, 600, 1), (1000, 77, 300, 2), (64, 64, 10, 3)])
def test_parity_random_fields(W, H, n_stars, seed):
    R = _field(W, H, n_stars, seed)
    want = _check(R, SKY, 150.0, 15000.0, 20, 10, 0.1, 100000)
    if W >= 333:
        assert len(want) > 10
    _check(R, SKY, 150.0, 15000.0, 20, 10, 0.1, 7)       # truncated list
    _check(R, SKY, 150.0, 1e30, 0, 0, 0.0, 100000)         # no margin, no isolation test
    _check(R, SKY, 90.0, 5000.0, 3, 25, 0.5, 100000)       # low threshold, wide isolation


def test_parity_full_size_frame():
    # 4096 x 4096 at the survey density: 500 stamps of 41 x 41, 30 px from the edges,
    # isolated within their stamp
    spec = starfield.WORKLOADS["ccd_4096x4096_L25_d3"]
    R = _field(spec.W, spec.H, spec.n_stars, spec.seed)
    want = _check(R, SKY, 150.0, 20000.0, 30, 20, 0.05, 500)
    assert len(want) == 500


@pytest.mark.parametrize("max_stamps", [1500, 2048, 2049])
def test_top_k_and_full_sort_over_many_candidates(max_stamps):
    # thousands of isolated peaks: up to 2048 stamps come from the top-k merge rounds over
    # chunks of 2048 keys, more from the full sort; both must give the oracle's list
    R = _field(1536, 1024, 9000, 11)
    want = _check(R, SKY, 150.0, 1e9, 4, 2, 0.5, max_stamps)
    assert len(want) == max_stamps


def test_constructed_frame_on_device():
    cat = starfield.Catalog(x=np.array([20.0, 60.0, 40.0, 46.0, 80.0, 86.0, 100.0, 106.0, 3.0]),
                            y=np.array([20.0, 30.0, 60.0, 60.0, 70.0, 70.0, 20.0, 20.0, 50.0]),
                            sigma=np.full(9, 1.2),
                            flux=np.array([5e4, 2e4, 3e4, 2.5e4, 4e4, 1e3, 2e5, 1.5e4, 3e4]))
    R = starfield.render(cat, 128, 96, sky=SKY).astype(np.float32)
    got, n_peaks = _run(R, SKY, 50.0, 20000.0, 8, 10, 0.1, 10)
    assert n_peaks == 9
    assert got.tolist() == [[20, 20], [80, 70], [60, 30]]


def test_edge_cases():
    flat = np.full((40, 50), SKY, dtype=np.float32)
    got, n = _run(flat, SKY, 10.0, 1e9, 0, 3, 0.1, 10)
    assert n == 0 and got.shape == (0, 2)
    one = np.array([[5000.0]], dtype=np.float32)  # a 1 x 1 frame: its pixel has no neighbours
    got, n = _run(one, SKY, 10.0, 1e9, 0, 3, 0.1, 10)
    assert n == 1 and got.tolist() == [[0, 0]]
    col = _field(1, 300, 30, 9)  # a single column
    _check(col, SKY, 150.0, 1e9, 0, 5, 0.1, 100)
    R = _field(200, 150, 100, 4)
    got, _ = _run(R, SKY, 150.0, 15000.0, 10, 5, 0.1, 0)
    assert got.shape == (0, 2)
    # equal peaks: row-major order
    eq = np.full((40, 50), SKY, dtype=np.float32)
    for (x, y) in [(30, 10), (12, 25), (40, 10), (20, 30)]:
        eq[y, x] = 2000.0
    got, _ = _run(eq, SKY, 100.0, 1e9, 2, 3, 0.5, 10)
    assert got.tolist() == [[30, 10], [40, 10], [12, 25], [20, 30]]


def test_pitched_input_and_workspace():
    R = _field(300, 200, 150, 5)
    big = torch.zeros((200, 320), dtype=torch.float32, device="cuda")
    big[:, :300] = torch.from_numpy(R).cuda()
    view = big[:, :300]
    ws = torch.empty(svk.svk_select_workspace_size(300, 200), dtype=torch.uint8, device="cuda")
    xy, counts = svk.svk_select_stamps(view, SKY, 150.0, 15000.0, 10, 8, 0.1, 1000, workspace=ws)
    n = int(counts[0])
    want, _ = ostamps.select_stamps(R, SKY, 150.0, 15000.0, 10, 8, 0.1, 1000)
    assert xy[:n].cpu().numpy().tolist() == want.tolist()


def test_rejects_bad_arguments():
    R = torch.zeros((10, 10), dtype=torch.float32, device="cuda")
    with pytest.raises(svk.SvkError):
        svk.svk_select_stamps(R, SKY, float("nan"), 1e9, 0, 3, 0.1, 10)
    with pytest.raises(svk.SvkError):
        svk.svk_select_stamps(R, SKY, 10.0, 1e9, -1, 3, 0.1, 10)
    with pytest.raises(svk.SvkError):
        svk.svk_select_stamps(R, SKY, 10.0, 1e9, 0, 3, -0.5, 10)
