"""Oracle of the stamp selection that feeds the least-squares fit (test infrastructure).

Only ``tests/``, ``__graft_entry__.smoke()`` and ``bench.py``'s CPU legs may import this
module; the CUDA library shares no code with it.

Sec. 2 fits the kernel coefficients over stamps around isolated stars and leaves the
selection rule open.  The rule followed here (and by the library):

* a *peak* is a pixel p with R(p) - sky >= threshold that is strictly greater than each
  of its in-frame 8-neighbours (a flat top has no peak);
* a peak is *selectable* when margin <= x <= W-1-margin, margin <= y <= H-1-margin,
  R(p) < saturation, and it is isolated: no other peak q with max(|dx|, |dy|) <=
  iso_radius has R(q) - sky >= iso_frac * (R(p) - sky);
* selectable peaks are ordered by R(p) descending, equal values by the row-major index
  y*W + x ascending, and the first max_stamps are returned as (x, y).

Every comparison and difference is taken in float32, the precision of the image, so the
GPU and this oracle decide each pixel identically.
"""
from __future__ import annotations

import numpy as np


def peaks(R, sky, threshold):
    """Boolean map of the peaks of R (strict local maxima over the 8 in-frame neighbours)."""
    R = np.asarray(R, dtype=np.float32)
    H, W = R.shape
    pad = np.full((H + 2, W + 2), -np.inf, dtype=np.float32)
    pad[1:-1, 1:-1] = R
    pk = (R - np.float32(sky)) >= np.float32(threshold)
    for dy in (-1, 0, 1):
        for dx in (-1, 0, 1):
            if dy or dx:
                pk &= R > pad[1 + dy:1 + dy + H, 1 + dx:1 + dx + W]
    return pk


def select_stamps(R, sky, threshold, saturation, margin, iso_radius, iso_frac, max_stamps):
    """(xy [n][2] int32, n_peaks): the stamp centres chosen by the rule above."""
    R = np.asarray(R, dtype=np.float32)
    H, W = R.shape
    sky32, sat32, frac32 = np.float32(sky), np.float32(saturation), np.float32(iso_frac)
    pk = peaks(R, sky, threshold)
    ys, xs = np.nonzero(pk)
    chosen = []
    for y, x in zip(ys.tolist(), xs.tolist()):
        if not (margin <= x <= W - 1 - margin and margin <= y <= H - 1 - margin):
            continue
        if not R[y, x] < sat32:
            continue
        bar = np.float32(frac32 * np.float32(R[y, x] - sky32))
        y0, y1 = max(0, y - iso_radius), min(H, y + iso_radius + 1)
        x0, x1 = max(0, x - iso_radius), min(W, x + iso_radius + 1)
        qy, qx = np.nonzero(pk[y0:y1, x0:x1])
        isolated = True
        for a, b in zip((qy + y0).tolist(), (qx + x0).tolist()):
            if (a, b) != (y, x) and np.float32(R[a, b] - sky32) >= bar:
                isolated = False
                break
        if isolated:
            chosen.append((-float(R[y, x]), y * W + x, x, y))
    chosen.sort()
    xy = np.array([[c[2], c[3]] for c in chosen[:max_stamps]], dtype=np.int32).reshape(-1, 2)
    return xy, int(pk.sum())
