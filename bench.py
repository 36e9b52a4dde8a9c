"""Throughput of the spatially-varying convolution + difference image on one GB300.

One step = one pass of the hot path over one synthetic CCD frame (2048 rows x 4096
columns, ~20k stars, kernel 19 x 19, 49-stamp Gaussian basis, quadratic spatial
variation): basis tabulation on the device, then D = (R (x) K_{x,y}) - I by the
tensor-core basis form (BF16 hi+lo split, FP32 accumulation) through the C ABI.

Printed JSON line (rank 0): value = Mpixel/s of D with inputs resident in HBM; e2e =
the same from pinned host buffers through the C ABI (svk_difference_host_batch: every
frame's R and I copied in and D copied out, the copies overlapped with the computation of
the neighbouring frames, all timed; the single-frame svk_difference_host beside it);
roofline of the dominant kernel (algorithmic FLOP / CUDA-event launch time vs the measured bf16 peak);
the direct form's throughput beside it; the FP64 oracle timed on the host cores on a
band of rows (cpu_baseline), whose output also gives the measured max relative error
of both GPU forms on that band.

`--impl reference` times the FP64 oracle alone (the reference arm).
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "Mpixel/s spatially-varying conv, TC basis form vs direct, at stated max rel err"
UNIT = "Mpixel/s"
WORKLOAD = "ccd_2048x4096_L19_d2"
L2_BYTES = 129 * 2 ** 20
NROT = 4  # rotating input frames: 4 x (R, I, D) = 384 MB > L2
E2E_BANDS = 2  # row bands per frame of the pipelined host-buffer call
E2E_SINGLE_BANDS = 8  # row bands of the single-frame host-buffer call (reported beside it)
NROT_HOST = 3  # distinct pinned host frames the end-to-end steps rotate through


def _peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            d = json.load(f)
        return d.get("bf16_tflops", 1900.0), d.get("hbm_gbs", 6800.0), "measured"
    return 1900.0, 6800.0, "fallback"


def _plan_str(svk, N, L, prec=None):
    G, st, sm = svk.svk_tc_plan(N, L, svk.SVK_PREC_BF16X3 if prec is None else prec)
    rpg = st // 4 if sm else st // 2
    return (f"G={G} output rows per block, {st} stages ({rpg}-row handshakes), "
            + ("basis slices streamed through a ring" if sm else "basis tables resident"))


def _algo_flops_per_px(N, L, degree):
    T = (degree + 1) * (degree + 2) // 2
    # basis contraction 2 N L^2, coefficient polynomials 2 N T, combination 2 N, subtraction 1
    return 2 * N * L * L + 2 * N * T + 2 * N + 1


def _direct_flops_per_px(N, L, degree):
    """Direct form per pixel: a_k (2NT), K = sum_k a_k B_k (2NL^2), sum K R (2L^2), - I."""
    T = (degree + 1) * (degree + 2) // 2
    return 2 * N * T + 2 * N * L * L + 2 * L * L + 1


def _raw_mma_flops(W, H, L, G, nmma, n_prod):
    """MMA FLOP one tensor-core launch issues: per block of G output rows the reference
    rows are taken in pairs; a pair costs 2 * (nG // 2) + (nG % 2) K steps of 16 taps, an
    odd last row (nG + nG % 2) / 2, with nG = ceil(L / 8) groups of 8 taps per row."""
    h = L // 2
    nG = (L + 7) // 8
    k_steps = 0
    for y0 in range(0, H, G):
        n = min(H - 1, y0 + G - 1 + h) - max(0, y0 - h) + 1
        k_steps += (n // 2) * (2 * (nG // 2) + (nG % 2)) + (n % 2) * ((nG + (nG % 2)) // 2)
    return k_steps * ((W + 127) // 128) * n_prod * 2 * 128 * nmma * 16


def _traffic(precision):
    """DRAM bytes per launch of the tensor-core kernel from the committed ncu summary, or
    None when that summary was taken on another workload or an older kernel source."""
    import hashlib
    p = os.path.join(ROOT, "profiles", "tc_basis_kernel_traffic.txt")
    if not os.path.exists(p):
        return None
    kv = {}
    with open(p) as f:
        for line in f:
            if ":" in line and not line.startswith("#"):
                k, v = line.split(":", 1)
                kv[k.strip()] = v.strip()
    h = hashlib.sha256()
    for name in ("svk_tc.cu", "svk_umma.cuh"):  # the kernel and its tcgen05 wrappers
        with open(os.path.join(ROOT, "paper_1209_5823_gb300", "csrc", name), "rb") as f:
            h.update(f.read())
    sha = h.hexdigest()
    if kv.get("workload") != WORKLOAD or kv.get("precision") != precision or kv.get("source_sha256") != sha:
        return None
    return int(kv["dram_bytes_per_launch"])


def _dist():
    """(dist module or None, rank, world size, local rank) from the torchrun environment.

    NCCL between GPUs; gloo when CUDA is absent (the host logic's CPU tests)."""
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    if ws > 1:
        import torch
        import torch.distributed as dist
        backend = "nccl" if torch.cuda.is_available() else "gloo"
        dist.init_process_group(backend=backend)
        return dist, dist.get_rank(), ws, int(os.environ.get("LOCAL_RANK", "0"))
    return None, 0, 1, 0


def _max_over_ranks(dist, values, device):
    """Element-wise maximum of a list of floats over all ranks (the job's slowest rank)."""
    import torch
    t = torch.tensor(values, dtype=torch.float64, device=device)
    if dist:
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return t.tolist()


def _job_rate(world, px_per_rank_step, steps, ms):
    """Whole-job Mpixel/s: every rank's pixels over the slowest rank's time."""
    return world * px_per_rank_step * steps / (ms / 1e3) / 1e6


class ClockSampler:
    """nvidia-smi clock / throttle sampling during the timed region."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,clocks_event_reasons.hw_slowdown,"
         "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
         "clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.gpu = gpu_index
        self.p = None

    def start(self):
        try:
            self.p = subprocess.Popen(["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.Q}",
                                       "--format=csv,noheader,nounits", "-lms", "100"],
                                      stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except OSError:
            self.p = None

    def stop(self):
        if self.p is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"], "samples": 0}
        self.p.terminate()
        try:
            out, _ = self.p.communicate(timeout=5)
        except subprocess.TimeoutExpired:
            self.p.kill()
            out, _ = self.p.communicate()
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in out.strip().splitlines():
            f = [x.strip() for x in line.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                mx.append(float(f[2]))
            except ValueError:
                continue
            for n, v in zip(names, f[5:9]):
                if v.lower() == "active":
                    reasons.add(n)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": sorted(reasons), "samples": len(sm)}


def _config(W, H, L, N, d):
    """The workload both arms run (the same dict on the svk and the reference line)."""
    return {"workload": WORKLOAD, "W": W, "H": H, "L": L, "N": N, "degree": d,
            "basis": "gauss 0.7/1.5/2.5 deg 6/4/2",
            "l2": f"inputs larger than L2: {NROT} rotating frames of R, I, D ({NROT * 3 * W * H * 4 / 2**20:.0f} MB)"}


def _frame_spec(rank=0):
    """Rank r of a multi-GPU run times its own frame: same shape, seed offset by r."""
    import dataclasses
    import starfield
    spec = starfield.WORKLOADS[WORKLOAD]
    return spec if rank == 0 else dataclasses.replace(spec, seed=spec.seed + 1000 * rank)


def _frame(rank=0):
    import numpy as np
    import starfield
    spec = _frame_spec(rank)
    R, I, _ = starfield.frame_pair(spec)
    c = starfield.planted_coeffs(49, spec.degree, starfield.rng(spec.seed + 7))
    return spec, R.astype(np.float32), I.astype(np.float32), c.astype(np.float32)


def _oracle_band(R, I, basis32, c32, degree, budget_s=12.0):
    """Time the FP64 oracle on a band of rows sized to ~budget_s of host CPU time."""
    import numpy as np
    import oracle
    H, W = R.shape
    R64, B64, C64 = R.astype(np.float64), basis32.astype(np.float64), c32.astype(np.float64)
    y0 = H // 2
    t = time.perf_counter()
    oracle.convolve(R64, B64, C64, degree, rows=(y0, y0 + 1))
    per_row = max(time.perf_counter() - t, 1e-4)
    nrows = int(max(1, min(H - y0, budget_s / per_row)))
    t = time.perf_counter()
    ref = oracle.convolve(R64, B64, C64, degree, rows=(y0, y0 + nrows))
    dt = time.perf_counter() - t
    return ref, (y0, y0 + nrows), dt, oracle.get_threads()


def _oracle_one_core(R, basis32, c32, degree, cores, rows=4):
    """The same oracle on one host thread, a few rows of the frame's middle."""
    import numpy as np
    import oracle
    H, W = R.shape
    y0 = H // 2
    oracle.set_threads(1)
    try:
        t = time.perf_counter()
        oracle.convolve(R.astype(np.float64), basis32.astype(np.float64), c32.astype(np.float64), degree,
                        rows=(y0, y0 + rows))
        dt = time.perf_counter() - t
    finally:
        oracle.set_threads(cores)
    return {"value": rows * W / dt / 1e6, "unit": UNIT, "cores": 1, "sample": f"rows {y0}..{y0 + rows - 1}"}


def _night_batch(svk, torch, dev, stream, reps=3):
    """The night batch: 60 frames (20 x 2048^2, 20 x 2048x4096, 20 x 4096^2, seeded order),
    L in {15..31}, degree 0..3.  One CUDA graph replaying svk_difference_batch against 60
    per-frame svk_difference calls; plans autotuned per L first."""
    import numpy as np
    import starfield
    specs = starfield.batch_specs()
    base = {}
    host = {}
    for sp in specs:  # one rendered field per size; frames are scaled copies (distinct buffers)
        if (sp.W, sp.H) not in base:
            R, I, _ = starfield.frame_pair(starfield.FrameSpec("b", sp.W, sp.H, sp.n_stars, sp.L, sp.degree, sp.seed))
            base[(sp.W, sp.H)] = (torch.from_numpy(R.astype(np.float32)).to(dev),
                                  torch.from_numpy(I.astype(np.float32)).to(dev))
            # pinned host copies for the night streamed from host memory (R, I read, D written)
            host[(sp.W, sp.H)] = (torch.from_numpy(R.astype(np.float32)).pin_memory(),
                                  torch.from_numpy(I.astype(np.float32)).pin_memory(),
                                  torch.empty((sp.H, sp.W), dtype=torch.float32).pin_memory())
    bases, items = {}, []
    for k, sp in enumerate(specs):
        if sp.L not in bases:
            bases[sp.L] = svk.svk_build_basis(svk.SVK_BASIS_GAUSS, sp.L)
        R0, I0 = base[(sp.W, sp.H)]
        c = starfield.planted_coeffs(49, sp.degree, starfield.rng(sp.seed))
        items.append(dict(R=R0 * (1.0 + 1e-3 * k), I=I0 * (1.0 + 1e-3 * k), D=torch.empty_like(R0),
                          basis=bases[sp.L], coeffs=torch.from_numpy(c.astype(np.float32)).to(dev), degree=sp.degree))
    del base
    tuned = {}
    for L in sorted(bases):
        tuned[L] = svk.svk_autotune(49, L, 2, svk.SVK_PREC_BF16X3, W=2048, H=512)
    px = sum(it["R"].numel() for it in items)
    ws = torch.empty(svk.svk_batch_workspace_size(items), dtype=torch.uint8, device=dev)
    wsf = torch.empty(max(svk.svk_workspace_size(1, svk.SVK_PREC_BF16X3, 0, 0, 49, L, 0) for L in bases),
                      dtype=torch.uint8, device=dev)

    def per_frame():
        for it in items:
            svk.svk_difference(it["R"], it["I"], it["basis"], it["coeffs"], it["degree"], method=svk.SVK_METHOD_BASIS,
                               precision=svk.SVK_PREC_BF16X3, out=it["D"], workspace=wsf)

    s = torch.cuda.Stream()
    with torch.cuda.stream(s):
        svk.svk_difference_batch(items, workspace=ws, stream=s)
    torch.cuda.synchronize()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g, stream=s):
        svk.svk_difference_batch(items, workspace=ws, stream=s)
    # the same night streamed from pinned host memory: every frame's R and I copied in and
    # D copied out, overlapped with the neighbouring frames' computation
    hitems = [dict(R=host[(it["R"].shape[1], it["R"].shape[0])][0], I=host[(it["R"].shape[1], it["R"].shape[0])][1],
                   D=host[(it["R"].shape[1], it["R"].shape[0])][2], basis=it["basis"], coeffs=it["coeffs"],
                   degree=it["degree"]) for it in items]
    wsh = torch.empty(svk.svk_host_batch_workspace_size(hitems), dtype=torch.uint8, device=dev)

    def host_stream():
        svk.svk_difference_host_batch(hitems, n_bands=2, workspace=wsh)

    out = {}
    for name, fn in (("graph_batch", g.replay), ("per_frame_launches", per_frame), ("host_stream", host_stream)):
        fn()
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        for _ in range(reps):
            fn()
        e1.record()
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1) / reps
        out[name] = {"ms_per_night": ms, "value": px / (ms / 1e3) / 1e6, "unit": UNIT}
    out["host_stream"]["call"] = ("svk_difference_host_batch from pinned host memory, 2 row bands per frame "
                                  f"({3 * px * 4 / 2**30:.1f} GiB copied per night)")
    out["frames"] = len(items)
    out["mpixels"] = px / 1e6
    out["tuned_plans"] = {str(L): {"G": v[0], "stages": v[1], "streamed": svk.svk_tc_plan(49, L)[2]}
                          for L, v in tuned.items()}
    out["workload"] = "night_60_frames_2048sq_2048x4096_4096sq_L15-31_d0-3"
    # roofline of the graph-captured night: the algorithmic FLOP of every frame (basis
    # contraction, coefficient polynomials, combination, subtraction) over the night's time
    flop = sum(_algo_flops_per_px(49, it["basis"].shape[1], it["degree"]) * it["R"].numel() for it in items)
    peak_bf16 = _peaks()[0]
    ach = flop / (out["graph_batch"]["ms_per_night"] / 1e3) / 1e12
    out["roofline"] = {"bound": "tensor", "achieved": ach, "peak": peak_bf16, "unit": "TFLOP/s",
                       "frac": ach / peak_bf16, "algorithmic_tflop_per_night": flop / 1e12,
                       "peak_source": "measured bf16 burst (MEASURED_PEAKS.json)"}
    # where the night's time goes: one 2048^2 frame per kernel size with its tuned plan
    per_L = {}
    R0 = torch.empty((2048, 2048), device=dev).uniform_(900.0, 1500.0)
    D0 = torch.empty_like(R0)
    for L in sorted(bases):
        c = torch.from_numpy(starfield.planted_coeffs(49, 2, starfield.rng(L)).astype(np.float32)).to(dev)
        wsl = torch.empty(svk.svk_workspace_size(1, svk.SVK_PREC_BF16X3, 0, 0, 49, L, 2), dtype=torch.uint8, device=dev)
        ms = _time(torch, lambda: svk.svk_difference(R0, R0, bases[L], c, 2, method=svk.SVK_METHOD_BASIS,
                                                     precision=svk.SVK_PREC_BF16X3, out=D0, workspace=wsl), reps=10)
        f = _algo_flops_per_px(49, L, 2) * R0.numel()
        per_L[str(L)] = {"ms_2048sq": ms, "tflops": f / (ms / 1e3) / 1e12, "frac": f / (ms / 1e3) / 1e12 / peak_bf16}
    out["per_kernel_size"] = per_L
    return out


def _fit_timing(svk, torch, dev, R, I, fp64_peak, reps=3):
    """Stamp selection and the device OIS fit at 500 stamps of 41 x 41, L = 25, 49 stamps,
    cubic coefficients and a constant background (on the 2048 x 4096 frame)."""
    H, W = R.shape
    Rt, It = torch.from_numpy(R).to(dev), torch.from_numpy(I).to(dev)
    # the 500 brightest isolated, unsaturated peaks at least 30 px from the edges with no
    # other peak above 5 % of their height within their stamp
    sel = dict(sky=1000.0, threshold=150.0, saturation=20000.0, margin=30, iso_radius=20, iso_frac=0.05,
               max_stamps=500)
    wsel = torch.empty(svk.svk_select_workspace_size(W, H), dtype=torch.uint8, device=dev)
    xy, counts = svk.svk_select_stamps(Rt, workspace=wsel, **sel)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(reps):
        xy, counts = svk.svk_select_stamps(Rt, workspace=wsel, **sel)
    e1.record()
    torch.cuda.synchronize()
    sel_ms = e0.elapsed_time(e1) / reps
    n_sel, n_peaks = counts.tolist()
    if n_sel < 1:
        raise RuntimeError("no stamp selected on the bench frame")
    st = xy[:n_sel].contiguous()
    B = svk.svk_build_basis(svk.SVK_BASIS_GAUSS, 25)
    ws = torch.empty(svk.svk_fit_workspace_size(n_sel, 41, 49, 25, 3, 0), dtype=torch.uint8, device=dev)
    svk.svk_fit_coeffs(Rt, It, st, 41, B, 3, bg_degree=0, workspace=ws)
    torch.cuda.synchronize()
    e0.record()
    for _ in range(reps):
        co, chi2, info = svk.svk_fit_coeffs(Rt, It, st, 41, B, 3, bg_degree=0, workspace=ws)
    e1.record()
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / reps
    # The moments as defined: per stamp pixel and column pair ((N+2)(N+3)/2 pairs, N = 49)
    # one product and 28 multiply-adds (monomials of degree <= 6), 57 FP64-equivalent FLOP.
    # The kernel forms them with row sums in double-float on the FP32 pipe and FP64 folds
    # once per row, so it is bound by neither pipe's peak (latency-bound, ncu); the line
    # reports the definition's FLOP rate and its ratio to the measured FP64 peak (the rate
    # the direct FP64 form could at best reach).
    px = n_sel * 41 * 41
    pairs = 51 * 52 // 2
    flop_def = px * pairs * (1 + 2 * 28)
    return {"ms": ms, "unknowns": 49 * 10 + 1, "stamp_pixels": px, "info": int(info.item()),
            "workload": "fit_500x41x41_L25_N49_d3_bg0",
            "stamps": {"selected": n_sel, "peaks": n_peaks, "select_ms": sel_ms, "rule": sel},
            "roofline": {"bound": "latency", "achieved": flop_def / (ms / 1e3) / 1e12,
                         "unit": "TFLOP/s (moments as defined, FP64-equivalent)",
                         "fp64_peak": fp64_peak / 1e12, "vs_fp64_peak": flop_def / (ms / 1e3) / fp64_peak,
                         "note": "whole fit time (selection excluded); moments by double-float row sums and "
                                 "row folds on the FP32 pipe (FP64 for the sums across CTAs), chi-square pass "
                                 "in double-float"}}


def _precision_table(svk, torch, dev):
    """4096 x 4096 frame, L = 25, 49 stamps, cubic coefficients: every arithmetic of the
    contraction against the FP64 oracle on 2000 random pixels plus the 200 brightest
    star centres (so the scale max|R (x) K| includes the star peaks), and its time."""
    import numpy as np
    import oracle
    import starfield
    spec = starfield.WORKLOADS["ccd_4096x4096_L25_d3"]
    g = starfield.rng(spec.seed)
    cat = starfield.star_catalog(spec.W, spec.H, spec.n_stars, g)
    R = starfield.add_noise(starfield.render(cat, spec.W, spec.H), 30.0, g).astype(np.float32)
    c = starfield.planted_coeffs(49, spec.degree, starfield.rng(spec.seed + 7)).astype(np.float32)
    Rt = torch.from_numpy(R).to(dev)
    ct = torch.from_numpy(c).to(dev)
    B = svk.svk_build_basis(svk.SVK_BASIS_GAUSS, spec.L)
    gs = starfield.rng(spec.seed + 9)
    top = np.argsort(cat.flux)[::-1][:200]
    px = np.concatenate([gs.integers(0, spec.W, 2000), np.clip(np.round(cat.x[top]), 0, spec.W - 1)]).astype(np.int32)
    py = np.concatenate([gs.integers(0, spec.H, 2000), np.clip(np.round(cat.y[top]), 0, spec.H - 1)]).astype(np.int32)
    ref = oracle.convolve_points(R.astype(np.float64), B.cpu().numpy().astype(np.float64), c.astype(np.float64),
                                 spec.degree, px, py)
    scale = np.abs(ref).max()
    # the same basis rounded so that 1024 B is FP16-exact, for SVK_PREC_FP16X2 (its errors
    # against the oracle on that rounded basis)
    Br = svk.svk_round_basis_fp16(B.clone())
    ref_r = oracle.convolve_points(R.astype(np.float64), Br.cpu().numpy().astype(np.float64), c.astype(np.float64),
                                   spec.degree, px, py)
    out = {"workload": spec.name, "sample": "2000 random pixels + 200 brightest star centres", "paths": {}}
    for name, method, prec, Bx, refx in (("basis_bf16x3", svk.SVK_METHOD_BASIS, svk.SVK_PREC_BF16X3, B, ref),
                                         ("basis_fp16x3", svk.SVK_METHOD_BASIS, svk.SVK_PREC_FP16X3, B, ref),
                                         ("basis_bf16", svk.SVK_METHOD_BASIS, svk.SVK_PREC_BF16, B, ref),
                                         ("basis_fp16x2_fp16_exact_basis", svk.SVK_METHOD_BASIS,
                                          svk.SVK_PREC_FP16X2, Br, ref_r),
                                         ("direct_fp32", svk.SVK_METHOD_DIRECT, svk.SVK_PREC_FP32, B, ref)):
        B_, ref_ = Bx, refx
        o = svk.svk_convolve(Rt, B_, ct, spec.degree, method=method, precision=prec)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        reps = 3
        e0.record()
        for _ in range(reps):
            svk.svk_convolve(Rt, B_, ct, spec.degree, method=method, precision=prec, out=o)
        e1.record()
        torch.cuda.synchronize()
        got = o[torch.from_numpy(py).to(dev).long(), torch.from_numpy(px).to(dev).long()].double().cpu().numpy()
        ms = e0.elapsed_time(e1) / reps
        out["paths"][name] = {"max_rel_err": float(np.abs(got - ref_).max() / scale),
                              "rms_rel_err": float(np.sqrt(((got - ref_) ** 2).mean()) / scale),
                              "ms": ms, "mpixel_s": spec.W * spec.H / (ms / 1e3) / 1e6}
    return out


def _learned(svk, torch, dev, R, I_unused, n_pairs=100000, steps=10000):
    """Coefficient network trained on n_pairs (R, I) stamp pairs the plain method makes,
    then applied to the 2048 x 4096 frame against the FP64 fit."""
    import time as _t
    import numpy as np
    import starfield
    from paper_1209_5823_gb300 import learned
    N, L = 49, 19
    basis = svk.svk_build_basis(svk.SVK_BASIS_GAUSS, L)
    prior = learned.CoeffPrior(N)
    gen = torch.Generator(device=dev).manual_seed(starfield.BASE_SEED + 4)
    H, W = R.shape
    Rt = torch.from_numpy(R).to(dev)
    g = starfield.rng(starfield.BASE_SEED + 4)
    cat = starfield.star_catalog(W, H, 20000, starfield.rng(starfield.WORKLOADS["ccd_2048x4096_L19_d2"].seed))
    bright = np.nonzero(cat.flux > 3000)[0]
    pick = g.choice(bright, n_pairs)
    cx = torch.from_numpy(np.clip(np.round(cat.x[pick]), 48, W - 49).astype(np.int64)).to(dev)
    cy = torch.from_numpy(np.clip(np.round(cat.y[pick]), 48, H - 49).astype(np.int64)).to(dev)
    a = prior.mean(dev) + prior.std(dev) * torch.randn((n_pairs, N), device=dev, generator=gen)
    t0 = _t.perf_counter()
    x, _, _ = learned.make_pairs(Rt, cx, cy, a, basis, 30.0, gen)
    torch.cuda.synchronize()
    t_pairs = _t.perf_counter() - t0
    n_hold = 2000
    net = learned.CoefficientNetwork(torch.from_numpy(starfield.cnn_init_params(N, starfield.BASE_SEED)).to(dev), prior,
                                     seed=starfield.BASE_SEED + 4)
    t0 = _t.perf_counter()
    losses = net.train(x[:-n_hold], a[:-n_hold], steps, lr=3e-3)
    torch.cuda.synchronize()
    t_train = _t.perf_counter() - t0
    # held-out error in standardised units (the prior mean scores 1), on the host
    pred = net.predict(x[-n_hold:]).cpu().numpy().astype(np.float64)
    a_h = a[-n_hold:].cpu().numpy().astype(np.float64)
    err = (((pred - a_h) / prior.std(dev).cpu().numpy()) ** 2).mean(axis=0)
    # device time of one gradient call (batch 256) and of a 4096-stamp forward pass
    xb = x[:net.batch].contiguous()
    zb = svk.svk_cnn_standardise(a[:net.batch], prior.mean(dev), prior.std(dev))
    gbuf, lbuf = torch.empty_like(net.params), torch.empty(1, device=dev)
    grad_ms = _time(torch, lambda: svk.svk_cnn_gradient(net.params, xb, zb, grad=gbuf, loss=lbuf, workspace=net.ws),
                    reps=50)
    # the same call at batch 1024 (the network's kernels are latency-bound at 256)
    xb4 = x[:1024].contiguous()
    zb4 = svk.svk_cnn_standardise(a[:1024], prior.mean(dev), prior.std(dev))
    ws4 = torch.empty(svk.svk_cnn_workspace_size(1024, N), dtype=torch.uint8, device=dev)
    grad1024_ms = _time(torch, lambda: svk.svk_cnn_gradient(net.params, xb4, zb4, grad=gbuf, loss=lbuf, workspace=ws4),
                        reps=20)
    xf = x[:4096].contiguous()
    fout = torch.empty((4096, N), device=dev)
    fws = torch.empty(svk.svk_cnn_workspace_size(4096, N), dtype=torch.uint8, device=dev)
    fwd_ms = _time(torch, lambda: svk.svk_cnn_forward(net.params, xf, N, out=fout, workspace=fws), reps=20)
    # algorithmic FLOP per stamp: forward convolutions (2 x MACs), the same again for the
    # weight gradients, and the data gradients of the three 32-channel layers
    conv = [32 * 32 * 32 * 18, 16 * 16 * 32 * 288, 8 * 8 * 32 * 288, 8 * 8 * 32 * 288]
    f_fwd = 2 * sum(conv)
    f_train = 2 * f_fwd + 2 * sum(conv[1:])
    # frames with a spatially varying kernel: network + field fit against the FP64 fit, at
    # quadratic (49 x 6) and cubic (49 x 10) coefficient fields, fitted from the 20 or the
    # 500 brightest stars; both judged by the D residual over 200 further stars neither
    # fitted (held out) and over their own fit stamps, and timed to coefficients
    order = np.argsort(cat.flux)[::-1]
    xy_all = np.stack([np.clip(np.round(cat.x[order]), 30, W - 31), np.clip(np.round(cat.y[order]), 30, H - 31)],
                      1).astype(np.int32)
    held = torch.from_numpy(xy_all[500:700]).to(dev)

    def frame_eval(d, n_fit, seed):
        T = (d + 1) * (d + 2) // 2
        c_true = torch.from_numpy(starfield.planted_coeffs(N, d, starfield.rng(starfield.BASE_SEED + 5 + 10 * seed))
                                  .astype(np.float32)).to(dev)
        fg = torch.Generator(device=dev).manual_seed(starfield.BASE_SEED + 50 + seed)
        I = svk.svk_convolve(Rt, basis, c_true, d, method=svk.SVK_METHOD_BASIS, precision=svk.SVK_PREC_BF16X3)
        I = I + 30.0 * torch.randn(I.shape, device=dev, generator=fg)
        st = torch.from_numpy(xy_all[:n_fit]).to(dev)
        learned.apply_to_frame(net, Rt, I, st, basis, d, 30.0, fallback_ratio=1e9, reference_noise_sigma=0.0)
        svk.svk_fit_coeffs(Rt, I, st, 41, basis, d, bg_degree=0)
        torch.cuda.synchronize()
        t0 = _t.perf_counter()
        res = learned.apply_to_frame(net, Rt, I, st, basis, d, 30.0, fallback_ratio=1e9, reference_noise_sigma=0.0)
        torch.cuda.synchronize()
        t_net = _t.perf_counter() - t0
        t0 = _t.perf_counter()
        co_fit, _, finfo = svk.svk_fit_coeffs(Rt, I, st, 41, basis, d, bg_degree=0)
        torch.cuda.synchronize()
        t_fit = _t.perf_counter() - t0
        cf = co_fit[:N * T].reshape(N, T).float().contiguous()
        out = {"degree": d, "field": f"{N}x{T}", "stamps": n_fit, "network_s": t_net, "fp64_fit_s": t_fit,
               "fit_info": int(finfo.item()), "noise_floor": res["floor"]}
        for name, co in (("network", res["coeffs"]), ("fit", cf)):
            D = svk.svk_difference(Rt, I, basis, co, d, method=svk.SVK_METHOD_BASIS, precision=svk.SVK_PREC_BF16X3)
            own, _ = svk.svk_stamp_residual(D, st, 41, basis[0], 30.0, 0.0, 2.0)
            ho, _ = svk.svk_stamp_residual(D, held, 41, basis[0], 30.0, 0.0, 2.0)
            out[f"{name}_chi2_per_px_fit_stamps"] = float(own[0].item())
            out[f"{name}_chi2_per_px_held_out"] = float(ho[0].item())
        out["network_to_floor"] = res["chi2_per_px"] / res["floor"]
        out["default_rule_source"] = "fit" if res["chi2_per_px"] > 2.0 * res["floor"] else "network"
        return out

    frames = [frame_eval(d, n_fit, 0) for d in (2, 3) for n_fit in (20, 500)]
    # the default rule (residual > 2 x floor hands the frame to the fit) over further frames
    rule = [frame_eval(d, 500, sd) for d in (2, 3) for sd in range(1, 5)]
    ratios = [f["network_to_floor"] for f in frames if f["stamps"] == 500] + [f["network_to_floor"] for f in rule]
    fallback_rule = {"ratio_bar": 2.0, "frames": len(ratios), "network_to_floor": ratios,
                     "fallbacks": sum(r > 2.0 for r in ratios)}
    return {"workload": "cnn_4conv32_64x64_pairs_to_49_local_coeffs",
            "pairs": n_pairs, "steps": steps, "batch": net.batch, "pairs_s": t_pairs, "train_s": t_train,
            "train_step_ms": 1e3 * t_train / steps, "gradient_ms": grad_ms,
            "train_stamps_per_s": net.batch / (1e-3 * grad_ms), "forward_4096_ms": fwd_ms,
            "forward_stamps_per_s": 4096 / (1e-3 * fwd_ms), "flop_per_stamp_forward": f_fwd,
            "flop_per_stamp_train": f_train, "gradient_tflops": f_train * net.batch / (1e-3 * grad_ms) / 1e12,
            "forward_tflops": f_fwd * 4096 / (1e-3 * fwd_ms) / 1e12,
            "gradient_1024_ms": grad1024_ms,
            "gradient_1024_tflops": f_train * 1024 / (1e-3 * grad1024_ms) / 1e12,
            "loss_first100": float(losses[:100].mean()), "loss_last100": float(losses[-100:].mean()),
            "heldout_mse_std_units": float(err.mean()), "heldout_mse_a0": float(err[0]), "prior_mse_std_units": 1.0,
            "frames": frames, "fallback_rule": fallback_rule}


def n_terms_d(d):
    return (d + 1) * (d + 2) // 2


def _time(torch, fn, reps=5):
    fn()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(reps):
        fn()
    e1.record()
    torch.cuda.synchronize()
    return e0.elapsed_time(e1) / reps


def _paper_sweep(svk, torch, dev):
    """The paper's measured workload (Sec. 3, Fig. 1): delta basis, L = 7 (49 stamps),
    second-order coefficients, images from 256^2 to one 4846 x 4868 camera tile; every
    form's Mpixel/s and the rate in the paper's cost model (20 L^2 + 1 FLOP per pixel)."""
    import numpy as np
    import starfield
    L, d = 7, 2
    B = svk.svk_build_basis(svk.SVK_BASIS_DELTA, L)
    c = torch.from_numpy(starfield.planted_coeffs(49, d, starfield.rng(starfield.BASE_SEED + 6), const_sd=0.01,
                                                  spatial_sd=0.005).astype(np.float32)).to(dev)
    rows = []
    for (W, H) in ((256, 256), (512, 512), (1024, 1024), (2048, 2048), (4096, 4096), (4846, 4868)):
        g = torch.Generator(device=dev).manual_seed(W)
        R = 1000.0 + 30.0 * torch.randn((H, W), device=dev, generator=g)
        I = 1000.0 + 30.0 * torch.randn((H, W), device=dev, generator=g)
        D = torch.empty_like(R)
        row = {"W": W, "H": H}
        for name, method, prec in (("direct_fp32", svk.SVK_METHOD_DIRECT, svk.SVK_PREC_FP32),
                                   ("basis_bf16x3", svk.SVK_METHOD_BASIS, svk.SVK_PREC_BF16X3),
                                   ("tform_bf16x3", svk.SVK_METHOD_TFORM, svk.SVK_PREC_BF16X3),
                                   ("tform_fp32", svk.SVK_METHOD_TFORM, svk.SVK_PREC_FP32)):
            ws = torch.empty(max(1, svk.svk_workspace_size(method, prec, W, H, 49, L, d)), dtype=torch.uint8, device=dev)
            ms = _time(torch, lambda: svk.svk_difference(R, I, B, c, d, method=method, precision=prec, out=D,
                                                         workspace=ws if method else None))
            row[name] = {"ms": ms, "mpixel_s": W * H / (ms / 1e3) / 1e6,
                         "paper_model_tflops": (20 * L * L + 1) * W * H / (ms / 1e3) / 1e12}
        rows.append(row)
    return {"workload": "paper_dfb_L7_d2_sizes_256sq_to_4846x4868", "rows": rows,
            "paper_model": "20 L^2 + 1 FLOP per pixel (Sec. 3)"}


def _sharded_frame(svk, torch, dist, rank, world, reps=5):
    """One frame split over the ranks (strong scaling of a single frame): each rank copies
    its band of rows (plus the kernel's halo) from pinned host memory, computes its rows of
    D, and the OIS fit sums the ranks' FP64 moments with one all-reduce before every rank
    solves.  Runs only with more than one rank."""
    from paper_1209_5823_gb300 import shard
    spec, R, I, c = _frame(0)  # every rank takes part in the same frame
    H, W = R.shape
    Rh, Ih = torch.from_numpy(R).pin_memory(), torch.from_numpy(I).pin_memory()
    B = svk.svk_build_basis(svk.SVK_BASIS_GAUSS, spec.L)
    ct = torch.from_numpy(c).cuda()
    sel = dict(sky=1000.0, threshold=150.0, saturation=20000.0, margin=30, iso_radius=20, iso_frac=0.05,
               max_stamps=500)
    xy, counts = svk.svk_select_stamps(torch.from_numpy(R).cuda(), **sel)
    xy = xy[:int(counts[0].item())].cpu().numpy()
    B25 = svk.svk_build_basis(svk.SVK_BASIS_GAUSS, 25)

    def band():
        return shard.difference_band(Rh, Ih, B, ct, spec.degree, svk.SVK_METHOD_BASIS, svk.SVK_PREC_BF16X3,
                                     rank=rank, world=world)

    def fit():
        return shard.fit_coeffs(Rh, Ih, xy, 41, B25, 3, 0, rank=rank, world=world)

    out = {}
    for name, fn in (("difference_rows", band), ("fit", fit)):
        fn()
        torch.cuda.synchronize()
        dist.barrier()
        t = time.perf_counter()
        for _ in range(reps):
            fn()
        torch.cuda.synchronize()
        ms = (time.perf_counter() - t) / reps * 1e3
        ms = _max_over_ranks(dist, [ms], torch.device("cuda", torch.cuda.current_device()))[0]
        out[name] = {"ms": ms}
    out["difference_rows"]["value"] = W * H / (out["difference_rows"]["ms"] / 1e3) / 1e6
    out["difference_rows"]["unit"] = UNIT
    out["scaling"] = "strong"
    out["workload"] = f"{WORKLOAD} split into {world} row bands; fit of {len(xy)} stamps, moments all-reduced"
    return out


def run_reference(args, rank):
    """Reference arm: the FP64 oracle on the host cores, same metric and workload."""
    if rank != 0:
        return
    import numpy as np
    import oracle
    import starfield
    spec, R, I, c = _frame()
    B = oracle.gauss_basis(spec.L).astype(np.float32)  # the same basis stamps, tabulated by the oracle
    H, W = R.shape
    # size each step so that (warmup + steps) steps take about two minutes in total
    y0 = H // 2
    R64, B64, C64 = R.astype(np.float64), B.astype(np.float64), c.astype(np.float64)
    t = time.perf_counter()
    oracle.convolve(R64, B64, C64, spec.degree, rows=(y0, y0 + 1))
    per_row = max(time.perf_counter() - t, 1e-4)
    rows = int(max(1, min(64, 120.0 / (args.steps + args.warmup) / per_row)))
    for _ in range(args.warmup):
        oracle.convolve(R64, B64, C64, spec.degree, rows=(y0, y0 + rows))
    t = time.perf_counter()
    for _ in range(args.steps):
        out = oracle.convolve(R64, B64, C64, spec.degree, rows=(y0, y0 + rows))
        _ = out - I[y0:y0 + rows]
    dt = time.perf_counter() - t
    px = args.steps * rows * W
    v = px / dt / 1e6
    cores = oracle.get_threads()
    line = {"metric": METRIC, "value": v, "unit": UNIT, "impl": "reference", "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": dt / args.steps * 1e3,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": _config(W, H, spec.L, 49, spec.degree),
            "path": {"method": "FP64 C oracle on the host cores"},
            "cpu_baseline": {"value": v, "unit": UNIT, "cores": cores, "kind": "oracle",
                             "sample": f"{rows} rows x {W} px of the frame per step (rows {y0}..{y0 + rows - 1})"},
            "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def main():
    global WORKLOAD
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=1000)
    ap.add_argument("--warmup", type=int, default=20)
    ap.add_argument("--impl", default="svk", choices=["svk", "reference"])
    ap.add_argument("--precision", default="bf16x3", choices=["bf16x3", "fp16x3", "bf16"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-extras", action="store_true", help="skip the night-batch and fit measurements")
    ap.add_argument("--workload", default="ccd_2048x4096_L19_d2", choices=["ccd_2048x4096_L19_d2", "ccd_4096x4096_L25_d3"],
                    help="the frame the step times (the default is the metric's; the other one profiles a "
                         "25-tap kernel)")
    ap.add_argument("--fit-only", action="store_true",
                    help="only the stamp selection and OIS fit measurement (one JSON object)")
    ap.add_argument("--learned-only", action="store_true",
                    help="only the coefficient-network measurement (its own JSON line; for profiling)")
    ap.add_argument("--learned-steps", type=int, default=10000, help="training steps of that measurement")
    args = ap.parse_args()
    args.warmup = max(3, args.warmup)
    WORKLOAD = args.workload

    if args.impl == "reference":
        # rank 0 alone runs the oracle; the other ranks of a torchrun launch exit at once
        run_reference(args, int(os.environ.get("RANK", "0")))
        return
    dist, rank, world, local_rank = _dist()

    import numpy as np
    import torch
    import paper_1209_5823_gb300 as svk
    from paper_1209_5823_gb300 import build as svk_build

    if rank == 0:
        svk_build.build()
    if dist:
        dist.barrier()
    torch.cuda.set_device(local_rank)
    dev = torch.device("cuda", local_rank)
    prec = {"bf16x3": svk.SVK_PREC_BF16X3, "fp16x3": svk.SVK_PREC_FP16X3, "bf16": svk.SVK_PREC_BF16}[args.precision]
    spec, R, I, c = _frame(rank)
    if args.fit_only:
        res = _fit_timing(svk, torch, dev, R, I, svk.svk_measure_fma_peak(svk.SVK_FMA_FP64))
        if rank == 0:
            print(json.dumps({"fit": res}), flush=True)
        return
    if args.learned_only:
        res = _learned(svk, torch, dev, R, I, steps=args.learned_steps)
        if rank == 0:
            print(json.dumps({"learned": res}), flush=True)
        return
    H, W, L, d = spec.H, spec.W, spec.L, spec.degree
    N = 49
    stream = torch.cuda.current_stream()

    Rs = [torch.from_numpy(R).to(dev) for _ in range(NROT)]
    Is = [torch.from_numpy(I).to(dev) for _ in range(NROT)]
    Ds = [torch.empty((H, W), dtype=torch.float32, device=dev) for _ in range(NROT)]
    ct = torch.from_numpy(c).to(dev)
    basis = torch.empty((N, L, L), dtype=torch.float32, device=dev)
    ws = torch.empty(svk.svk_workspace_size(svk.SVK_METHOD_BASIS, prec, W, H, N, L, d), dtype=torch.uint8, device=dev)

    def step(i, ev=None):
        svk.svk_build_basis(svk.SVK_BASIS_GAUSS, L, out=basis)
        if ev is not None:
            ev[0].record(stream)
        svk.svk_difference(Rs[i % NROT], Is[i % NROT], basis, ct, d, method=svk.SVK_METHOD_BASIS, precision=prec,
                           out=Ds[i % NROT], workspace=ws)
        if ev is not None:
            ev[1].record(stream)

    launches_per_step = 3  # basis tabulation, table preparation, tensor-core kernel
    for i in range(args.warmup):
        step(i)
    torch.cuda.synchronize()
    evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    clk = ClockSampler(local_rank if os.environ.get("CUDA_VISIBLE_DEVICES") is None else 0)
    clk.start()
    time.sleep(0.3)
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    t0 = torch.cuda.Event(enable_timing=True)
    t1 = torch.cuda.Event(enable_timing=True)
    t0.record(stream)
    for i in range(args.steps):
        step(i, evs[i])
    t1.record(stream)
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    ms_total = t0.elapsed_time(t1)
    kern_ms = statistics.mean(a.elapsed_time(b) for a, b in evs)

    # e2e through the C ABI with host buffers: every step is one frame whose R and I are
    # copied in from pinned host memory and whose D is copied out, its basis built and its
    # tables prepared; svk_difference_host_batch pipelines the timed steps' frames (frame
    # k + 1's copies in and frame k - 1's copies out overlap frame k's computation).
    Rh = [torch.from_numpy(R).clone().pin_memory() for _ in range(NROT_HOST)]
    Ih = [torch.from_numpy(I).clone().pin_memory() for _ in range(NROT_HOST)]
    Dh = [torch.empty((H, W), dtype=torch.float32).pin_memory() for _ in range(NROT_HOST)]
    n_e2e = max(10, args.steps // 4)
    bases = [torch.empty((N, L, L), dtype=torch.float32, device=dev) for _ in range(n_e2e)]
    items = [dict(R=Rh[k % NROT_HOST], I=Ih[k % NROT_HOST], D=Dh[k % NROT_HOST], basis=bases[k], coeffs=ct, degree=d)
             for k in range(n_e2e)]
    wsh = torch.empty(svk.svk_host_batch_workspace_size(items, svk.SVK_METHOD_BASIS, prec), dtype=torch.uint8,
                      device=dev)

    def e2e_run():
        for b in bases:
            svk.svk_build_basis(svk.SVK_BASIS_GAUSS, L, out=b)
        svk.svk_difference_host_batch(items, method=svk.SVK_METHOD_BASIS, precision=prec, n_bands=E2E_BANDS,
                                      workspace=wsh)

    e2e_run()
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    e2e_run()
    e1.record(stream)
    torch.cuda.synchronize()
    e2e_ms = e0.elapsed_time(e1)

    # the same frames one svk_difference_host call at a time (no overlap across frames)
    ws1 = torch.empty(svk.svk_host_workspace_size(svk.SVK_METHOD_BASIS, prec, W, H, N, L, d), dtype=torch.uint8,
                      device=dev)

    def e2e_single(k):
        svk.svk_build_basis(svk.SVK_BASIS_GAUSS, L, out=bases[k])
        svk.svk_difference_host(Rh[k % NROT_HOST], Ih[k % NROT_HOST], bases[k], ct, d, method=svk.SVK_METHOD_BASIS,
                                precision=prec, out=Dh[k % NROT_HOST], n_bands=E2E_SINGLE_BANDS, workspace=ws1)

    for k in range(3):
        e2e_single(k)
    torch.cuda.synchronize()
    e0.record(stream)
    for k in range(n_e2e):
        e2e_single(k)
    e1.record(stream)
    torch.cuda.synchronize()
    e2e1_ms = e0.elapsed_time(e1)
    clocks = clk.stop()

    # the direct form on the same frame, for the "vs direct" half of the metric
    n_dir = max(5, min(50, args.steps // 20))
    Dd = torch.empty((H, W), dtype=torch.float32, device=dev)
    for _ in range(2):
        svk.svk_difference(Rs[0], Is[0], basis, ct, d, method=svk.SVK_METHOD_DIRECT, out=Dd)
    torch.cuda.synchronize()
    d0, d1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    d0.record(stream)
    for i in range(n_dir):
        svk.svk_difference(Rs[i % NROT], Is[i % NROT], basis, ct, d, method=svk.SVK_METHOD_DIRECT, out=Dd)
    d1.record(stream)
    torch.cuda.synchronize()
    dir_ms = d0.elapsed_time(d1) / n_dir

    # the T-factored form on the same frame (a different form of the same result)
    Dt = torch.empty((H, W), dtype=torch.float32, device=dev)
    wst = torch.empty(svk.svk_workspace_size(svk.SVK_METHOD_TFORM, prec, W, H, N, L, d), dtype=torch.uint8, device=dev)
    tf_ms = _time(torch, lambda: svk.svk_difference(Rs[0], Is[0], basis, ct, d, method=svk.SVK_METHOD_TFORM,
                                                    precision=prec, out=Dt, workspace=wst), reps=20)
    # the T-form on the CUDA cores (FP32 FFMA: the T convolutions R (x) K_t accumulated per pixel)
    Dtf32 = torch.empty((H, W), dtype=torch.float32, device=dev)
    wst32 = torch.empty(max(1, svk.svk_workspace_size(svk.SVK_METHOD_TFORM, svk.SVK_PREC_FP32, W, H, N, L, d)),
                        dtype=torch.uint8, device=dev)
    tf32_ms = _time(torch, lambda: svk.svk_difference(Rs[0], Is[0], basis, ct, d, method=svk.SVK_METHOD_TFORM,
                                                      precision=svk.SVK_PREC_FP32, out=Dtf32, workspace=wst32),
                    reps=20)

    # max over ranks
    ms_total, e2e_ms, e2e1_ms, kern_ms, dir_ms = _max_over_ranks(dist, [ms_total, e2e_ms, e2e1_ms, kern_ms, dir_ms],
                                                                 dev)
    px = W * H
    value = _job_rate(world, px, args.steps, ms_total)
    e2e_value = _job_rate(world, px, n_e2e, e2e_ms)
    e2e1_value = _job_rate(world, px, n_e2e, e2e1_ms)
    # one frame split over the ranks (every rank takes part in its all-reduce)
    sharded = _sharded_frame(svk, torch, dist, rank, world) if dist and not args.no_extras else None
    if rank != 0:
        return

    peak_bf16, hbm, peak_src = _peaks()
    # the FP32 ALU peak is the larger of scalar FFMA and packed f32x2 FMA throughput (the
    # packed form reaches the 128 lanes per SM with fewer issue slots)
    fp32_ffma = svk.svk_measure_fma_peak(svk.SVK_FMA_FP32)
    fp32_x2 = svk.svk_measure_fma_peak(svk.SVK_FMA_FP32X2)
    fp32_peak = max(fp32_ffma, fp32_x2)
    fp64_peak = svk.svk_measure_fma_peak(svk.SVK_FMA_FP64)
    dir_flop = _direct_flops_per_px(N, L, d) * px
    tf32_flop = 2 * n_terms_d(d) * L * L + 2 * n_terms_d(d) + 1  # T convolutions, monomial sum, difference
    algo = _algo_flops_per_px(N, L, d) * px
    achieved = algo / (kern_ms / 1e3) / 1e12
    # raw MMA work of the launch (split products, padded taps, window rows), for context:
    # the default plan for N = 49, L = 19 stacks G = 5 output rows per block (MMA N = 256)
    Gp = svk.svk_tc_plan(N, L, prec)[0]
    raw_flops = _raw_mma_flops(W, H, L, G=Gp, nmma=(Gp * N + 15) // 16 * 16,
                               n_prod={"bf16x3": 3, "fp16x3": 3, "bf16": 1}[args.precision])
    traffic = _traffic(args.precision)

    out = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms_total / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": f"{args.precision}-f32acc", "data": "synthetic",
        "config": _config(W, H, L, N, d),
        "path": {"method": "basis (tcgen05)", "precision": args.precision},
        "gpu_launches": launches_per_step * args.steps,
        "e2e": {"value": e2e_value, "unit": UNIT, "h2d_bytes_per_step": 2 * px * 4, "d2h_bytes_per_step": px * 4,
                "call": f"svk_difference_host_batch over the {n_e2e} timed frames (pinned host buffers rotating over "
                        f"{NROT_HOST} frames, {E2E_BANDS} row bands each, basis built per frame)",
                "single_frame_calls": {"value": e2e1_value, "unit": UNIT,
                                       "call": f"svk_difference_host per frame, {E2E_SINGLE_BANDS} row bands"}},
        "roofline": {"bound": "tensor", "achieved": achieved, "peak": peak_bf16, "unit": "TFLOP/s",
                     "frac": achieved / peak_bf16, "traffic": traffic,
                     "peak_source": f"{peak_src} bf16 burst (MEASURED_PEAKS.json)",
                     "kernel": "tc_basis_kernel (+ table prep) per CUDA-event bracket",
                     "algorithmic_flop_per_px": _algo_flops_per_px(N, L, d),
                     "plan": _plan_str(svk, N, L, prec),
                     "raw_mma_tflops": raw_flops / (kern_ms / 1e3) / 1e12,
                     "raw_mma_frac": raw_flops / (kern_ms / 1e3) / 1e12 / peak_bf16},
        "direct": {"value": world * px / (dir_ms / 1e3) / 1e6, "unit": UNIT, "ms_per_frame": dir_ms,
                   "dtype": "f32",
                   "roofline": {"bound": "alu", "achieved": dir_flop / (dir_ms / 1e3) / 1e12,
                                "peak": fp32_peak / 1e12, "unit": "TFLOP/s",
                                "frac": dir_flop / (dir_ms / 1e3) / fp32_peak,
                                "algorithmic_flop_per_px": _direct_flops_per_px(N, L, d),
                                "peak_source": "measured FP32 FMA throughput, max of scalar FFMA and packed "
                                               "f32x2 (svk_measure_fma_peak)"}},
        "measured_fma": {"fp32_tflops": fp32_ffma / 1e12, "fp32x2_tflops": fp32_x2 / 1e12,
                         "fp32_peak_tflops": fp32_peak / 1e12, "fp64_tflops": fp64_peak / 1e12},
        "clocks": clocks,
        "tform": {"value": world * px / (tf_ms / 1e3) / 1e6, "unit": UNIT, "ms_per_frame": tf_ms,
                  "form": "sum_t m_t (R (x) K_t) - I, K_t = sum_k c[k][t] B_k (same result, T = 6 convolutions)",
                  "fp32_ffma": {"value": world * px / (tf32_ms / 1e3) / 1e6, "unit": UNIT, "ms_per_frame": tf32_ms,
                                "tflops": tf32_flop * px / (tf32_ms / 1e3) / 1e12,
                                "frac": tf32_flop * px / (tf32_ms / 1e3) / fp32_peak,
                                "flop_per_px": tf32_flop,
                                "kernel": "tform_fp32_kernel: T convolutions R (x) K_t per pixel, "
                                          "sum_t m_t C_t - I in the epilogue"}},
    }
    if sharded is not None:
        out["sharded_frame"] = sharded
    if not args.no_extras:
        out["night_batch"] = _night_batch(svk, torch, dev, stream)
        out["fit"] = _fit_timing(svk, torch, dev, R, I, fp64_peak)
        out["precision"] = _precision_table(svk, torch, dev)
        out["paper_sweep"] = _paper_sweep(svk, torch, dev)
        out["learned"] = _learned(svk, torch, dev, R, I, steps=args.learned_steps)
    if not args.no_cpu_baseline:
        ref, rows, dt, cores = _oracle_band(R, I, basis.cpu().numpy(), c, d)
        y0, y1 = rows
        Dtc = Ds[(args.steps - 1) % NROT][y0:y1].cpu().numpy().astype(np.float64) + I[y0:y1]
        Ddir = Dd[y0:y1].cpu().numpy().astype(np.float64) + I[y0:y1]
        scale = np.abs(ref).max()
        out["cpu_baseline"] = {"value": (y1 - y0) * W / dt / 1e6, "unit": UNIT, "cores": cores, "kind": "oracle",
                               "sample": f"rows {y0}..{y1 - 1} ({(y1 - y0) * W} px) of the frame, FP64 C oracle"}
        out["cpu_baseline"]["single_core"] = _oracle_one_core(R, basis.cpu().numpy(), c, d, cores)
        Dtf = Dt[y0:y1].cpu().numpy().astype(np.float64) + I[y0:y1]
        out["tform"]["max_rel_err"] = float(np.abs(Dtf - ref).max() / scale)
        Dtf32h = Dtf32[y0:y1].cpu().numpy().astype(np.float64) + I[y0:y1]
        out["tform"]["fp32_ffma"]["max_rel_err"] = float(np.abs(Dtf32h - ref).max() / scale)
        out["max_rel_err"] = {"basis": float(np.abs(Dtc - ref).max() / scale),
                              "direct": float(np.abs(Ddir - ref).max() / scale),
                              "measure": "max|D_gpu - D_oracle| / max|R (x) K| over the cpu_baseline band"}
    print(json.dumps(out), flush=True)
    if dist:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
