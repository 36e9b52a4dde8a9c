"""Host logic of one frame split over several GPUs, on CPU (gloo ranks, no GPU).

The partition (row bands aligned to the kernel's row block, the rows each band reads,
the stamps each rank owns) and the fit's one exchange step: every rank accumulates the
normal equations of its own stamps, reading only the rows it would hold, and the sum over
the ranks (shard.reduce_moments, an all-reduce) equals the normal equations of all stamps
on one rank (Sec. 2 fit; Sec. 4 split of an image between GPUs).  The normal equations
here are the oracle's, so the check is independent of the CUDA library.
"""
import os
import socket
import sys

import numpy as np
import pytest
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

from paper_1209_5823_gb300 import shard  # noqa: E402


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


@pytest.mark.parametrize("H,gran,world", [(2048, 5, 2), (2048, 5, 8), (4096, 12, 3), (100, 40, 4), (7, 16, 3),
                                          (4868, 16, 8)])
def test_row_bands_partition(H, gran, world):
    bands = shard.row_bands(H, gran, world)
    assert [b.rank for b in bands] == list(range(world))
    assert bands[0].y0 == 0 and bands[-1].y1 == H
    for a, b in zip(bands, bands[1:]):
        assert a.y1 == b.y0  # contiguous, in rank order
    for b in bands:
        assert b.y0 <= b.y1
        assert b.y0 % gran == 0 and (b.y1 % gran == 0 or b.y1 == H)
    # as even as the granule allows: no two non-empty bands differ by more than one block
    sizes = [(b.y1 - b.y0 + gran - 1) // gran for b in bands]
    assert max(sizes) - min(sizes) <= 1


def test_held_rows_cover_the_kernel_reach():
    H, L = 2048, 19
    h = L // 2
    for b in shard.row_bands(H, 5, 4):
        r0, r1 = shard.held_rows(b, h, H)
        assert r0 == max(0, b.y0 - h) and r1 == min(H, b.y1 + h)


def test_stamps_owned_by_exactly_one_rank():
    g = np.random.default_rng(5)
    xy = np.stack([g.integers(0, 512, 300), g.integers(0, 1000, 300)], 1)
    bands = shard.row_bands(1000, 1, 3)
    owned = np.concatenate([shard.stamps_of(xy, b) for b in bands])
    assert np.array_equal(np.sort(owned), np.arange(len(xy)))


def _fit_worker(rank, world, port, out_dir):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    sys.path.insert(0, ROOT)
    import torch
    import torch.distributed as dist

    import oracle
    from paper_1209_5823_gb300 import shard as sh
    import starfield
    dist.init_process_group("gloo", rank=rank, world_size=world)
    W, H, L, S, d, bd = 160, 150, 7, 11, 2, 1
    g = starfield.rng(77)
    cat = starfield.star_catalog(W, H, 120, g)
    R = starfield.add_noise(starfield.render(cat, W, H), 30.0, g)
    I = starfield.add_noise(starfield.render(cat, W, H), 30.0, g)
    B = oracle.gauss_basis(L, sigma=(0.9, 1.8), deg=(1, 0))
    xy = np.stack([g.integers(S, W - S, 40), g.integers(0, H, 40)], 1).astype(np.int32)  # some straddle the edges
    band = sh.row_bands(H, 1, world)[rank]
    own = sh.stamps_of(xy, band)
    r0, r1 = sh.held_rows(band, sh.fit_halo(S, L), H)
    # the rows a rank does not hold are poison: reading one would turn its sums into NaN
    Rr, Ir = np.full_like(R, np.nan), np.full_like(I, np.nan)
    Rr[r0:r1], Ir[r0:r1] = R[r0:r1], I[r0:r1]
    M = B.shape[0] * oracle.n_terms(d) + oracle.n_terms(bd)
    if len(own):
        A, b = oracle.normal_equations(Rr, Ir, xy[own], S, B, d, bg_degree=bd)
    else:
        A, b = np.zeros((M, M)), np.zeros(M)
    mom = torch.from_numpy(np.concatenate([A.ravel(), b]))
    sh.reduce_moments(mom)
    np.save(os.path.join(out_dir, f"rank{rank}.npy"), mom.numpy())
    if rank == 0:
        A1, b1 = oracle.normal_equations(R, I, xy, S, B, d, bg_degree=bd)
        np.save(os.path.join(out_dir, "single.npy"), np.concatenate([A1.ravel(), b1]))
        np.save(os.path.join(out_dir, "owned.npy"), np.array([len(xy)]))
    dist.barrier()
    dist.destroy_process_group()


@pytest.mark.parametrize("world", [2, 3])
def test_split_moments_sum_to_single_rank_normal_equations(tmp_path, world):
    mp.start_processes(_fit_worker, args=(world, _free_port(), str(tmp_path)), nprocs=world, start_method="spawn")
    single = np.load(tmp_path / "single.npy")
    for r in range(world):
        got = np.load(tmp_path / f"rank{r}.npy")
        assert np.all(np.isfinite(got))
        # the same sums, added in another order: equal to FP64 rounding
        np.testing.assert_allclose(got, single, rtol=1e-12, atol=1e-9 * np.abs(single).max())
    # every rank ends with the same array
    assert all(np.array_equal(np.load(tmp_path / "rank0.npy"), np.load(tmp_path / f"rank{r}.npy"))
               for r in range(world))
