"""Pins of the stamp-selection oracle (Sec. 2: the fit runs over isolated stars).

The expected selections are fixed by how the frames are built (positions, fluxes,
saturation, edges), not by running the oracle; a loop-by-loop restatement checks the
rule's invariants on noisy frames.
"""
import numpy as np

import starfield
from oracle import stamps as ostamps

SKY = 1000.0


def _field(stars, W=128, H=96, sigma=1.2):
    """Noise-free frame with Gaussian stars centred on pixel centres (x, y, flux)."""
    # render() samples each Gaussian at integer pixel positions: integer centres peak there
    x = np.array([s[0] for s in stars], dtype=np.float64)
    y = np.array([s[1] for s in stars], dtype=np.float64)
    cat = starfield.Catalog(x=x, y=y, sigma=np.full(len(stars), sigma), flux=np.array([s[2] for s in stars]))
    return starfield.render(cat, W, H, sky=SKY).astype(np.float32)


A, B, C, D, E, F = (20, 20, 5e4), (60, 30, 2e4), (40, 60, 3e4), (46, 60, 2.5e4), (80, 70, 4e4), (86, 70, 1e3)
G, Hs, Ie = (100, 20, 2e5), (106, 20, 1.5e4), (3, 50, 3e4)


def _select(R, max_stamps=10, saturation=20000.0):
    return ostamps.select_stamps(R, SKY, 50.0, saturation, margin=8, iso_radius=10, iso_frac=0.1,
                                 max_stamps=max_stamps)


def test_constructed_frame():
    # A, B isolated; C/D a close pair of similar flux (both rejected); E with a faint
    # companion F (E kept, F rejected); G saturated (rejected) and it rejects its
    # neighbour H; I too close to the edge.  Equal widths: order = order of flux.
    R = _field([A, B, C, D, E, F, G, Hs, Ie])
    xy, n_peaks = _select(R)
    assert n_peaks == 9
    assert xy.tolist() == [[A[0], A[1]], [E[0], E[1]], [B[0], B[1]]]


def test_max_stamps_truncates_the_order():
    R = _field([A, B, C, D, E, F, G, Hs, Ie])
    xy, _ = _select(R, max_stamps=2)
    assert xy.tolist() == [[A[0], A[1]], [E[0], E[1]]]
    xy, _ = _select(R, max_stamps=0)
    assert xy.shape == (0, 2)


def test_saturation_and_isolation_switches():
    R = _field([A, B, C, D, E, F, G, Hs, Ie])
    # no saturation limit: G is selected first; H stays rejected by G
    xy, _ = _select(R, saturation=1e9)
    assert xy.tolist()[0] == [G[0], G[1]]
    assert [Hs[0], Hs[1]] not in xy.tolist()
    # iso_radius 0: only the margin and saturation rules remain
    xy, _ = ostamps.select_stamps(R, SKY, 50.0, 20000.0, margin=8, iso_radius=0, iso_frac=0.1, max_stamps=20)
    assert sorted(map(tuple, xy.tolist())) == sorted([(s[0], s[1]) for s in (A, B, C, D, E, F, Hs)])


def test_equal_peaks_order_by_row_major_index():
    R = np.full((40, 50), SKY, dtype=np.float32)
    for (x, y) in [(30, 10), (12, 25), (40, 10), (20, 30)]:
        R[y, x] = 2000.0  # four equal isolated single-pixel peaks
    xy, n = ostamps.select_stamps(R, SKY, 100.0, 1e9, margin=2, iso_radius=3, iso_frac=0.5, max_stamps=10)
    assert n == 4
    assert xy.tolist() == [[30, 10], [40, 10], [12, 25], [20, 30]]


def test_flat_top_is_not_a_peak():
    R = np.full((20, 20), SKY, dtype=np.float32)
    R[10, 10] = R[10, 11] = 5000.0
    xy, n = ostamps.select_stamps(R, SKY, 10.0, 1e9, margin=0, iso_radius=0, iso_frac=0.1, max_stamps=10)
    assert n == 0 and xy.shape == (0, 2)


def _loop_rule(R, sky, thr, sat, margin, rad, frac):
    """The selection rule restated pixel by pixel with plain loops (no numpy masks)."""
    H, W = R.shape
    f32 = np.float32

    def is_peak(y, x):
        if not f32(R[y, x] - f32(sky)) >= f32(thr):
            return False
        for dy in (-1, 0, 1):
            for dx in (-1, 0, 1):
                if (dy or dx) and 0 <= y + dy < H and 0 <= x + dx < W and not R[y, x] > R[y + dy, x + dx]:
                    return False
        return True

    pk = [[is_peak(y, x) for x in range(W)] for y in range(H)]
    out = []
    for y in range(margin, H - margin):
        for x in range(margin, W - margin):
            if not pk[y][x] or not R[y, x] < f32(sat):
                continue
            bar = f32(f32(frac) * f32(R[y, x] - f32(sky)))
            ok = True
            for yy in range(max(0, y - rad), min(H, y + rad + 1)):
                for xx in range(max(0, x - rad), min(W, x + rad + 1)):
                    if (yy, xx) != (y, x) and pk[yy][xx] and f32(R[yy, xx] - f32(sky)) >= bar:
                        ok = False
            if ok:
                out.append((x, y))
    out.sort(key=lambda p: (-float(R[p[1], p[0]]), p[1] * W + p[0]))
    return out, sum(map(sum, pk))


def test_matches_loop_restatement_on_noisy_fields():
    for seed in range(3):
        g = starfield.rng(500 + seed)
        W, H = 72, 56
        cat = starfield.star_catalog(W, H, 40, g)
        R = starfield.add_noise(starfield.render(cat, W, H), 30.0, g).astype(np.float32)
        args = (SKY, 120.0, 15000.0, 5, 6, 0.2)
        want, n_want = _loop_rule(R, *args)
        xy, n = ostamps.select_stamps(R, *args, max_stamps=1000)
        assert n == n_want
        assert [tuple(p) for p in xy.tolist()] == want
        assert len(want) > 3
