"""The debug build (compiled with -DSVK_DEBUG): the kernels check their shared-memory,
tensor-memory and MMA-descriptor indices and report a failed check through the library's
status word (svk_device_status returns SVK_ERR_INDEX) instead of trapping.

The same cases -- every method and precision on ragged frames, row bands from band
buffers, a mixed batch -- run in a child process against the debug build and here
against the release build: no check may fire, and the results must be the same bit for
bit (the checks only guard accesses)."""
import os
import subprocess
import sys

import numpy as np
import pytest
import torch

pytestmark = pytest.mark.gpu

HERE = os.path.dirname(os.path.abspath(__file__))


def run_cases():
    """Outputs of the cases, as numpy arrays keyed by case name (any library build)."""
    import paper_1209_5823_gb300 as svk
    from _helpers import coeffs, star_pair
    out = {}
    methods = [(svk.SVK_METHOD_DIRECT, svk.SVK_PREC_FP32), (svk.SVK_METHOD_BASIS, svk.SVK_PREC_BF16X3),
               (svk.SVK_METHOD_BASIS, svk.SVK_PREC_FP16X3), (svk.SVK_METHOD_BASIS, svk.SVK_PREC_BF16),
               (svk.SVK_METHOD_TFORM, svk.SVK_PREC_BF16X3), (svk.SVK_METHOD_TFORM, svk.SVK_PREC_FP32)]
    for W, H, L, d in ((300, 173, 19, 2), (129, 37, 25, 3), (7, 5, 11, 1), (1000, 3, 31, 0), (520, 260, 7, 2)):
        R, I = star_pair(W, H, max(3, W * H // 300), 4000 + W + H)
        Rt, It = torch.from_numpy(R).cuda(), torch.from_numpy(I).cuda()
        B = svk.svk_build_basis(svk.SVK_BASIS_GAUSS, L)
        c = torch.from_numpy(coeffs(49, d, W + L)).cuda()
        for m, p in methods:
            D = svk.svk_difference(Rt, It, B, c, d, method=m, precision=p)
            out[f"frame_{W}x{H}_L{L}_m{m}_p{p}"] = D.cpu().numpy()
            # two bands from buffers holding only the rows they read
            gran = svk.svk_band_rows(m, p, 49, L, d)
            y1 = min(H, gran * max(1, (H // 2) // gran))
            for y0, ye in ((0, y1), (y1, H)):
                if ye <= y0:
                    continue
                r0, r1 = max(0, y0 - L // 2), min(H, ye + L // 2)
                Db = svk.svk_difference_rows(Rt[r0:r1].contiguous(), It[y0:ye].contiguous(), B, c, d, W, H, y0, ye, r0,
                                             method=m, precision=p)
                out[f"band_{W}x{H}_L{L}_m{m}_p{p}_{y0}"] = Db.cpu().numpy()
    # a mixed batch (frames of several sizes and kernel sizes in grouped launches)
    items = []
    for k, (W, H, L, d) in enumerate(((300, 100, 15, 1), (129, 64, 19, 2), (260, 33, 15, 3), (64, 200, 23, 0))):
        R, I = star_pair(W, H, max(3, W * H // 300), 5000 + k)
        items.append(dict(R=torch.from_numpy(R).cuda(), I=torch.from_numpy(I).cuda(),
                          D=torch.empty((H, W), device="cuda"), basis=svk.svk_build_basis(svk.SVK_BASIS_GAUSS, L),
                          coeffs=torch.from_numpy(coeffs(49, d, 60 + k)).cuda(), degree=d))
    svk.svk_difference_batch(items)
    for k, it in enumerate(items):
        out[f"batch_{k}"] = it["D"].cpu().numpy()
    torch.cuda.synchronize()
    return out


def child(path):
    """Entry of the child process: run the cases against the library SVK_LIBRARY names,
    save the outputs, and fail if any device index check fired."""
    import paper_1209_5823_gb300 as svk
    res = run_cases()
    np.savez(path, **res)
    st = svk.load_library().svk_device_status(1, None)
    if st != svk.SVK_OK:
        print("device status", st, svk.load_library().svk_last_error().decode())
        sys.exit(3)


def test_debug_build_checks_stay_silent_and_change_nothing(tmp_path):
    from paper_1209_5823_gb300 import build
    dbg = build.build(debug=True)
    path = str(tmp_path / "debug_out.npz")
    env = dict(os.environ, SVK_LIBRARY=dbg)
    code = f"import sys; sys.path[:0] = [{HERE!r}, {os.path.dirname(HERE)!r}]; import test_debug_gpu as t; t.child({path!r})"
    p = subprocess.run([sys.executable, "-c", code], env=env, capture_output=True, text=True, timeout=900)
    assert p.returncode == 0, p.stdout[-2000:] + p.stderr[-3000:]
    got = np.load(path)
    want = run_cases()
    assert set(got.files) == set(want)
    for k, v in want.items():
        assert np.array_equal(got[k], v, equal_nan=True), k
