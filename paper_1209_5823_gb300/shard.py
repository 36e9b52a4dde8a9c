"""One frame split over several GPUs, one process per GPU (torch.distributed ranks).

The paper splits an image between two GPUs (Sec. 4) and names more GPUs as the way on
(Sec. 6).  The difference image needs no exchange at all: each rank computes a band of
output rows from the band of R it reads (its rows plus an h-row halo on each side, h =
L // 2) and the same rows of I, copied from host memory; no rank reads another's memory.
The least-squares fit has one exchange step: each rank accumulates the FP64 moments of
the stamps whose centres lie in its band, the moment arrays are summed over the ranks
(one all-reduce), and every rank solves the same normal equations.

Everything here is host logic (partitions, copies, the all-reduce); every step of the
method runs in the library's kernels through the C ABI (svk_difference_rows,
svk_fit_moments, svk_fit_solve).
"""
from __future__ import annotations

from dataclasses import dataclass


@dataclass(frozen=True)
class Band:
    """Rank `rank`'s share of an H-row frame: output rows [y0, y1)."""
    rank: int
    y0: int
    y1: int


def row_bands(H: int, granule: int, world: int) -> list[Band]:
    """Contiguous bands of output rows, one per rank, covering [0, H) in rank order.

    Boundaries are multiples of `granule` (the kernel's block of output rows, so a block
    never straddles two ranks and every row equals the single-GPU result bit for bit) and
    as even as the granule allows; a rank may get an empty band when H is small."""
    if H < 1 or granule < 1 or world < 1:
        raise ValueError("H, granule and world must be positive")
    blocks = (H + granule - 1) // granule
    bounds = [min(H, (blocks * r // world) * granule) for r in range(world)] + [H]
    return [Band(r, bounds[r], bounds[r + 1]) for r in range(world)]


def held_rows(band: Band, halo: int, H: int) -> tuple[int, int]:
    """Rows [r0, r1) of the frame a rank holds for a band that reads `halo` rows beyond it."""
    return max(0, band.y0 - halo), min(H, band.y1 + halo)


def fit_halo(stamp_size: int, L: int) -> int:
    """Rows beyond a stamp's centre that its fit reads: the stamp's half size plus the
    kernel's half size (C_k = R (x) B_k at every stamp pixel)."""
    return (stamp_size - 1) // 2 + (L - 1) // 2


def stamps_of(stamp_xy, band: Band):
    """Indices of the stamps (rows of an [n][2] (x, y) array) whose centre row lies in the
    band: every stamp belongs to exactly one rank."""
    import numpy as np
    xy = np.asarray(stamp_xy).reshape(-1, 2)
    return np.nonzero((xy[:, 1] >= band.y0) & (xy[:, 1] < band.y1))[0]


def reduce_moments(moments, group=None):
    """Sum a moment array over the ranks in place (the fit's one exchange step): NCCL
    between GPUs, gloo for host tensors.  A single process returns it unchanged."""
    import torch.distributed as dist
    if dist.is_available() and dist.is_initialized() and dist.get_world_size(group) > 1:
        dist.all_reduce(moments, op=dist.ReduceOp.SUM, group=group)
    return moments


def _rank_world(group):
    import torch.distributed as dist
    if dist.is_available() and dist.is_initialized():
        return dist.get_rank(group), dist.get_world_size(group)
    return 0, 1


def difference_band(R_host, I_host, basis, coeffs, degree: int, method: int, precision: int, rank: int | None = None,
                    world: int | None = None, group=None, workspace=None, stream=None):
    """This rank's band of D = (R (x) K) - I for a frame held in (pinned) host memory.

    Copies the band's rows of I and the rows of R it reads to the current device, computes
    them with svk_difference_rows and returns (D_band on the device, Band)."""
    import torch

    import paper_1209_5823_gb300 as svk
    if rank is None or world is None:
        rank, world = _rank_world(group)
    H, W = R_host.shape
    N, L = basis.shape[0], basis.shape[1]
    gran = svk.svk_band_rows(method, precision, N, L, degree)
    if gran < 1:
        raise ValueError("no kernel plan for this method and basis")
    band = row_bands(H, gran, world)[rank]
    if band.y1 <= band.y0:
        return torch.empty((0, W), dtype=torch.float32, device="cuda"), band
    r0, r1 = held_rows(band, (L - 1) // 2, H)
    dev = torch.device("cuda", torch.cuda.current_device())
    Rb = R_host[r0:r1].to(dev, non_blocking=True)
    Ib = I_host[band.y0:band.y1].to(dev, non_blocking=True)
    D = svk.svk_difference_rows(Rb, Ib, basis, coeffs, degree, W, H, band.y0, band.y1, r0, method=method,
                                precision=precision, workspace=workspace, stream=stream)
    return D, band


def fit_coeffs(R_host, I_host, stamp_xy, stamp_size: int, basis, degree: int, bg_degree: int = -1, weight_host=None,
               rank: int | None = None, world: int | None = None, group=None, sync: bool = False):
    """The OIS fit of one frame over the ranks: moments of this rank's stamps (centres in
    its band of rows), summed over the ranks, solved on every rank.

    R_host, I_host (and weight_host): the frame in host memory; stamp_xy: all stamps of the
    frame (host [n][2] int array), the same on every rank.  Returns (coeffs, chi2, info)
    device tensors, identical on every rank."""
    import numpy as np
    import torch

    import paper_1209_5823_gb300 as svk
    if rank is None or world is None:
        rank, world = _rank_world(group)
    H, W = R_host.shape
    N, L = basis.shape[0], basis.shape[1]
    band = row_bands(H, 1, world)[rank]
    own = stamps_of(stamp_xy, band)
    dev = torch.device("cuda", torch.cuda.current_device())
    moments = torch.zeros(svk.svk_fit_moments_count(N, degree, bg_degree), dtype=torch.float64, device=dev)
    if len(own) > 0:
        r0, r1 = held_rows(band, fit_halo(stamp_size, L), H)
        Rb = R_host[r0:r1].to(dev, non_blocking=True)
        Ib = I_host[r0:r1].to(dev, non_blocking=True)
        wb = weight_host[r0:r1].to(dev, non_blocking=True) if weight_host is not None else None
        st = torch.from_numpy(np.ascontiguousarray(np.asarray(stamp_xy).reshape(-1, 2)[own], dtype=np.int32)).to(dev)
        svk.svk_fit_moments(Rb, Ib, st, stamp_size, basis, degree, bg_degree, W=W, H=H, row_begin=r0, weight=wb,
                            moments=moments)
    reduce_moments(moments, group)
    return svk.svk_fit_solve(moments, N, degree, bg_degree, sync=sync)
