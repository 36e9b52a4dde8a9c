"""Python binding of the SVK C ABI (include/svk.h): argument marshalling only.

Every function here has the name of the C entry point it calls and takes torch tensors
on the current CUDA device; all arithmetic runs in the CUDA kernels of ``libsvk.so``.
There is no fallback: if the library is missing, importing the functions raises.
"""
from __future__ import annotations

import ctypes
import os

PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(PKG, "libsvk.so")

SVK_OK = 0
SVK_ERR_ARG = 1
SVK_ERR_CUDA = 2
SVK_ERR_NOT_SPD = 3
SVK_ERR_TIMEOUT = 4
SVK_ERR_UNSUPPORTED = 5
SVK_ERR_WORKSPACE = 6
SVK_ERR_INDEX = 7

SVK_BASIS_GAUSS = 0
SVK_BASIS_DELTA = 1
SVK_NORM_NONE = 0
SVK_NORM_ALARD = 1
SVK_METHOD_DIRECT = 0
SVK_METHOD_BASIS = 1
SVK_METHOD_TFORM = 2
SVK_PREC_FP32 = 0
SVK_PREC_BF16X3 = 1
SVK_PREC_FP16X3 = 2
SVK_PREC_BF16 = 3
SVK_PREC_FP16X2 = 4
SVK_FMA_FP32 = 0
SVK_FMA_FP64 = 1
SVK_FMA_FP32X2 = 2
SVK_EDGE_ZERO = 0

# every symbol include/svk.h declares (checked by the tests)
EXPORTS = (
    "svk_last_error", "svk_version", "svk_gauss_basis_count", "svk_build_basis", "svk_workspace_size",
    "svk_convolve", "svk_difference", "svk_fit_workspace_size", "svk_fit_coeffs", "svk_difference_noalloc",
    "svk_batch_workspace_size", "svk_difference_batch", "svk_autotune", "svk_cnn_param_count",
    "svk_cnn_workspace_size", "svk_cnn_forward", "svk_cnn_gradient", "svk_cnn_adam", "svk_cnn_adam_device_step",
    "svk_cnn_field_fit",
    "svk_select_workspace_size", "svk_select_stamps", "svk_measure_fma_peak", "svk_host_workspace_size",
    "svk_difference_host", "svk_host_batch_workspace_size", "svk_difference_host_batch", "svk_selftest_bounded_wait",
    "svk_device_status", "svk_fit_moments_count", "svk_fit_moments_workspace_size", "svk_fit_moments",
    "svk_fit_solve_workspace_size", "svk_fit_solve", "svk_band_rows", "svk_difference_rows", "svk_cut_stamps",
    "svk_stamp_residual_workspace_size", "svk_stamp_residual", "svk_cnn_standardise", "svk_cnn_draw_batch",
    "svk_gather_rows", "svk_cnn_step_end", "svk_tc_plan", "svk_set_plan", "svk_round_basis_fp16",
)


class svk_frame(ctypes.Structure):
    """struct svk_frame of include/svk.h (device pointers, pitches in elements)."""
    _fields_ = [("R", ctypes.c_void_p), ("pitch_R", ctypes.c_int), ("I", ctypes.c_void_p), ("pitch_I", ctypes.c_int),
                ("D", ctypes.c_void_p), ("pitch_D", ctypes.c_int), ("W", ctypes.c_int), ("H", ctypes.c_int),
                ("basis", ctypes.c_void_p), ("N", ctypes.c_int), ("L", ctypes.c_int), ("coeffs", ctypes.c_void_p),
                ("degree", ctypes.c_int)]


class SvkError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"svk status {status}: {msg}")
        self.status = status


_lib = None


def load_library(path: str | None = None):
    """Load libsvk.so (built by paper_1209_5823_gb300.build); raises if it is missing."""
    global _lib
    if _lib is not None and path is None:
        return _lib
    # SVK_LIBRARY selects another build of the same ABI (e.g. the debug build, libsvk_debug.so)
    p = path or os.environ.get("SVK_LIBRARY") or LIB_PATH
    if not os.path.exists(p):
        raise RuntimeError(f"CUDA library {p} is not built; run `python -c 'import __graft_entry__ as g; g.build()'`")
    lib = ctypes.CDLL(p)
    vp, i, sz, f = ctypes.c_void_p, ctypes.c_int, ctypes.c_size_t, ctypes.c_float
    sig = {
        "svk_last_error": (ctypes.c_char_p, []),
        "svk_version": (i, []),
        "svk_gauss_basis_count": (i, [i, vp]),
        "svk_build_basis": (i, [i, i, i, vp, vp, i, vp, vp, vp]),
        "svk_workspace_size": (sz, [i, i, i, i, i, i, i]),
        "svk_convolve": (i, [vp, i, i, i, vp, i, i, vp, i, i, i, i, vp, i, vp, sz, vp]),
        "svk_difference": (i, [vp, i, vp, i, i, i, vp, i, i, vp, i, i, i, i, vp, i, vp, sz, vp]),
        "svk_fit_workspace_size": (sz, [i, i, i, i, i, i]),
        "svk_fit_coeffs": (i, [vp, vp, i, i, i, vp, i, i, vp, i, i, i, i, vp, vp, vp, vp, vp, sz, i, vp]),
        "svk_difference_noalloc": (i, [vp, i, vp, i, i, i, vp, i, i, vp, i, i, i, vp, i, vp]),
        "svk_batch_workspace_size": (sz, [vp, i, i]),
        "svk_difference_batch": (i, [vp, i, i, vp, sz, vp]),
        "svk_autotune": (i, [i, i, i, i, i, i, vp, vp, vp]),
        "svk_tc_plan": (i, [i, i, i, vp, vp, vp]),
        "svk_set_plan": (i, [i, i, i, i, i, i]),
        "svk_round_basis_fp16": (i, [vp, ctypes.c_longlong, vp]),
        "svk_cnn_param_count": (i, [i]),
        "svk_cnn_workspace_size": (sz, [i, i]),
        "svk_cnn_forward": (i, [vp, vp, i, i, vp, vp, sz, vp]),
        "svk_cnn_gradient": (i, [vp, vp, vp, i, i, vp, vp, vp, sz, vp]),
        "svk_cnn_adam": (i, [vp, vp, vp, vp, i, i, ctypes.c_float, ctypes.c_float, ctypes.c_float, ctypes.c_float,
                             vp]),
        "svk_cnn_adam_device_step": (i, [vp, vp, vp, vp, i, vp, ctypes.c_float, ctypes.c_float, ctypes.c_float,
                                         ctypes.c_float, vp]),
        "svk_cnn_field_fit": (i, [vp, vp, vp, i, i, i, i, i, vp, vp, vp]),
        "svk_measure_fma_peak": (i, [i, vp, vp]),
        "svk_selftest_bounded_wait": (i, [ctypes.c_ulonglong, vp, vp]),
        "svk_device_status": (i, [i, vp]),
        "svk_host_workspace_size": (sz, [i, i, i, i, i, i, i]),
        "svk_difference_host": (i, [vp, vp, vp, i, i, i, vp, i, i, vp, i, i, i, i, vp, sz, vp]),
        "svk_host_batch_workspace_size": (sz, [vp, i, i, i]),
        "svk_difference_host_batch": (i, [vp, i, i, i, i, vp, sz, vp]),
        "svk_select_workspace_size": (sz, [i, i]),
        "svk_select_stamps": (i, [vp, i, i, i, f, f, f, i, i, f, i, vp, vp, vp, sz, vp]),
        "svk_fit_moments_count": (sz, [i, i, i]),
        "svk_fit_moments_workspace_size": (sz, [i, i, i]),
        "svk_fit_moments": (i, [vp, vp, vp, i, i, i, i, i, vp, i, i, vp, i, i, i, i, vp, i, vp, sz, vp]),
        "svk_fit_solve_workspace_size": (sz, [i, i, i]),
        "svk_fit_solve": (i, [vp, i, i, i, vp, vp, vp, vp, sz, i, vp]),
        "svk_band_rows": (i, [i, i, i, i, i]),
        "svk_difference_rows": (i, [vp, i, i, i, vp, i, vp, i, i, i, i, i, vp, i, i, vp, i, i, i, i, vp, sz, vp]),
        "svk_cut_stamps": (i, [vp, i, i, i, vp, i, i, f, f, vp, ctypes.c_longlong, vp]),
        "svk_stamp_residual_workspace_size": (sz, [i]),
        "svk_stamp_residual": (i, [vp, i, i, i, vp, i, i, vp, i, ctypes.c_double, ctypes.c_double, ctypes.c_double,
                                   vp, vp, vp, vp, sz, vp]),
        "svk_cnn_standardise": (i, [vp, ctypes.c_longlong, i, vp, vp, i, vp, vp]),
        "svk_cnn_draw_batch": (i, [ctypes.c_ulonglong, vp, i, i, vp, vp]),
        "svk_gather_rows": (i, [vp, ctypes.c_longlong, vp, i, vp, vp]),
        "svk_cnn_step_end": (i, [vp, vp, vp, i, vp]),
    }
    for name, (res, args) in sig.items():
        f = getattr(lib, name)
        f.restype = res
        f.argtypes = args
    if path is None:
        _lib = lib
    return lib


def _check(status: int):
    if status != SVK_OK:
        raise SvkError(status, load_library().svk_last_error().decode())


def _stream(stream):
    import torch
    if stream is None:
        stream = torch.cuda.current_stream()
    return ctypes.c_void_p(stream.cuda_stream)


def _ptr(t):
    return ctypes.c_void_p(t.data_ptr()) if t is not None else ctypes.c_void_p(0)


def _img(t, name, host=False):
    import torch
    where = "host" if host else "CUDA"
    if t.dtype != torch.float32 or t.is_cuda == host or t.dim() != 2 or t.stride(1) != 1:
        raise ValueError(f"{name} must be a {where} float32 [H][pitch] tensor with unit column stride")
    return t.shape[0], t.shape[1], t.stride(0)


def n_terms(degree: int) -> int:
    return 0 if degree < 0 else (degree + 1) * (degree + 2) // 2


def svk_version() -> int:
    return int(load_library().svk_version())


def svk_gauss_basis_count(deg) -> int:
    arr = (ctypes.c_int * len(deg))(*deg)
    return int(load_library().svk_gauss_basis_count(len(deg), arr))


def svk_build_basis(kind: int, L: int, sigma=(0.7, 1.5, 2.5), deg=(6, 4, 2), normalize: int = SVK_NORM_ALARD,
                    out=None, stream=None):
    """Tabulate the basis stamps on the device; returns a float32 [N][L][L] tensor."""
    import torch
    lib = load_library()
    sg = (ctypes.c_double * len(sigma))(*sigma)
    dg = (ctypes.c_int * len(deg))(*deg)
    if kind == SVK_BASIS_GAUSS:
        N = int(lib.svk_gauss_basis_count(len(deg), dg))
        if N < 0:
            raise ValueError("bad degree list")
    else:
        N = L * L
    if out is None:
        out = torch.empty((N, L, L), dtype=torch.float32, device="cuda")
    nb = ctypes.c_int(0)
    _check(lib.svk_build_basis(int(kind), int(L), len(sigma), sg, dg, int(normalize), _ptr(out),
                               ctypes.byref(nb), _stream(stream)))
    return out


def svk_round_basis_fp16(basis, stream=None):
    """Round a device float32 basis in place so that 1024 b is FP16-exact (SVK_PREC_FP16X2)."""
    _check(load_library().svk_round_basis_fp16(_ptr(basis), int(basis.numel()), _stream(stream)))
    return basis


def svk_workspace_size(method: int, precision: int, W: int, H: int, N: int, L: int, degree: int) -> int:
    return int(load_library().svk_workspace_size(method, precision, W, H, N, L, degree))


def svk_convolve(R, basis, coeffs, degree: int, method: int = SVK_METHOD_DIRECT, precision: int = SVK_PREC_FP32,
                 out=None, workspace=None, stream=None, edge: int = SVK_EDGE_ZERO):
    """out = R (x) K_{x,y} (Eq. 1-3); all tensors on the CUDA device."""
    import torch
    H, W, pR = _img(R, "R")
    N, L = basis.shape[0], basis.shape[1]
    if out is None:
        out = torch.empty((H, W), dtype=torch.float32, device=R.device)
    _, _, pO = _img(out, "out")
    ws_bytes = 0 if workspace is None else workspace.numel() * workspace.element_size()
    _check(load_library().svk_convolve(_ptr(R), W, H, pR, _ptr(basis), N, L, _ptr(coeffs), int(degree), int(method),
                                       int(precision), int(edge), _ptr(out), pO, _ptr(workspace), ws_bytes,
                                       _stream(stream)))
    return out


def svk_difference(R, I, basis, coeffs, degree: int, method: int = SVK_METHOD_DIRECT,
                   precision: int = SVK_PREC_FP32, out=None, workspace=None, stream=None, edge: int = SVK_EDGE_ZERO):
    """D = (R (x) K_{x,y}) - I (Eq. 1); all tensors on the CUDA device."""
    import torch
    H, W, pR = _img(R, "R")
    H2, W2, pI = _img(I, "I")
    if (H2, W2) != (H, W):
        raise ValueError("R and I differ in size")
    N, L = basis.shape[0], basis.shape[1]
    if out is None:
        out = torch.empty((H, W), dtype=torch.float32, device=R.device)
    _, _, pD = _img(out, "D")
    ws_bytes = 0 if workspace is None else workspace.numel() * workspace.element_size()
    _check(load_library().svk_difference(_ptr(R), pR, _ptr(I), pI, W, H, _ptr(basis), N, L, _ptr(coeffs),
                                         int(degree), int(method), int(precision), int(edge), _ptr(out), pD,
                                         _ptr(workspace), ws_bytes, _stream(stream)))
    return out


def svk_difference_noalloc(R, I, basis, coeffs, degree: int, precision: int = SVK_PREC_BF16X3, out=None,
                           stream=None, edge: int = SVK_EDGE_ZERO):
    """D = (R (x) K_{x,y}) - I by the tensor-core basis form without any device allocation.

    For callers that cannot allocate device memory while they run (their heap is owned by
    a host application, or allocation is not allowed after start-up): the library uses
    one built-in 512 KiB scratch array instead of a workspace.  Calls share that array,
    so overlapping calls on the GPU must be serialised by the caller.
    """
    import torch
    H, W, pR = _img(R, "R")
    H2, W2, pI = _img(I, "I")
    if (H2, W2) != (H, W):
        raise ValueError("R and I differ in size")
    N, L = basis.shape[0], basis.shape[1]
    if out is None:
        out = torch.empty((H, W), dtype=torch.float32, device=R.device)
    _, _, pD = _img(out, "D")
    _check(load_library().svk_difference_noalloc(_ptr(R), pR, _ptr(I), pI, W, H, _ptr(basis), N, L, _ptr(coeffs),
                                                 int(degree), int(precision), int(edge), _ptr(out), pD,
                                                 _stream(stream)))
    return out


def _frames(items, host=False):
    """items: sequence of dicts with R, I (or None), D, basis, coeffs, degree (torch tensors;
    R, I, D in host memory when `host`)."""
    arr = (svk_frame * len(items))()
    for k, it in enumerate(items):
        H, W, pR = _img(it["R"], "R", host)
        _, _, pD = _img(it["D"], "D", host)
        pI = _img(it["I"], "I", host)[2] if it.get("I") is not None else W
        b = it["basis"]
        arr[k] = svk_frame(it["R"].data_ptr(), pR, it["I"].data_ptr() if it.get("I") is not None else None, pI,
                           it["D"].data_ptr(), pD, W, H, b.data_ptr(), b.shape[0], b.shape[1],
                           it["coeffs"].data_ptr(), int(it["degree"]))
    return arr


def svk_batch_workspace_size(items, precision: int = SVK_PREC_BF16X3) -> int:
    arr = _frames(items)
    return int(load_library().svk_batch_workspace_size(ctypes.cast(arr, ctypes.c_void_p), len(items), int(precision)))


def svk_difference_batch(items, precision: int = SVK_PREC_BF16X3, workspace=None, stream=None):
    """D = (R (x) K) - I for every frame of `items` (dicts of CUDA tensors) in grouped
    persistent launches; each item's "D" tensor receives its result."""
    arr = _frames(items)
    ws_bytes = 0 if workspace is None else workspace.numel() * workspace.element_size()
    _check(load_library().svk_difference_batch(ctypes.cast(arr, ctypes.c_void_p), len(items), int(precision),
                                               _ptr(workspace), ws_bytes, _stream(stream)))


def svk_autotune(N: int, L: int, degree: int, precision: int = SVK_PREC_BF16X3, W: int = 2048, H: int = 1024,
                 stream=None):
    """Time the tensor-core plans for (N, L, degree, precision); returns (G, stages) chosen."""
    g, st = ctypes.c_int(0), ctypes.c_int(0)
    _check(load_library().svk_autotune(int(N), int(L), int(degree), int(precision), int(W), int(H),
                                       ctypes.byref(g), ctypes.byref(st), _stream(stream)))
    return g.value, st.value


def svk_tc_plan(N: int, L: int, precision: int = SVK_PREC_BF16X3):
    """The tensor-core plan calls with (N, L, precision) use: (G, stages, streamed)."""
    g, st, sm = ctypes.c_int(0), ctypes.c_int(0), ctypes.c_int(0)
    _check(load_library().svk_tc_plan(int(N), int(L), int(precision), ctypes.byref(g), ctypes.byref(st),
                                       ctypes.byref(sm)))
    return g.value, st.value, sm.value


def svk_set_plan(N: int, L: int, precision: int, G: int, stages: int = 16, streamed: int = 0):
    """Pin the tensor-core plan for (N, L, precision); G = 0 restores the default."""
    _check(load_library().svk_set_plan(int(N), int(L), int(precision), int(G), int(stages), int(streamed)))


def svk_fit_workspace_size(n_stamps: int, stamp_size: int, N: int, L: int, degree: int, bg_degree: int) -> int:
    return int(load_library().svk_fit_workspace_size(n_stamps, stamp_size, N, L, degree, bg_degree))


def svk_fit_coeffs(R, I, stamp_xy, stamp_size: int, basis, degree: int, bg_degree: int = -1, weight=None,
                   workspace=None, sync: bool = False, stream=None):
    """OIS least-squares fit on the device; returns (coeffs[M] f64, chi2[1] f64, info[1] i32) tensors."""
    import torch
    H, W, p = _img(R, "R")
    _, _, pI = _img(I, "I")
    if pI != p or (weight is not None and weight.stride(0) != p):
        raise ValueError("R, I and weight must share one pitch")
    N, L = basis.shape[0], basis.shape[1]
    M = N * n_terms(degree) + n_terms(bg_degree)
    coeffs = torch.zeros(M, dtype=torch.float64, device=R.device)
    chi2 = torch.zeros(1, dtype=torch.float64, device=R.device)
    info = torch.zeros(1, dtype=torch.int32, device=R.device)
    ws_bytes = 0 if workspace is None else workspace.numel() * workspace.element_size()
    st = stamp_xy.to(torch.int32).contiguous()
    _check(load_library().svk_fit_coeffs(_ptr(R), _ptr(I), W, H, p, _ptr(st), st.shape[0], int(stamp_size),
                                         _ptr(basis), N, L, int(degree), int(bg_degree), _ptr(weight), _ptr(coeffs),
                                         _ptr(chi2), _ptr(info), _ptr(workspace), ws_bytes, int(bool(sync)),
                                         _stream(stream)))
    return coeffs, chi2, info


def svk_fit_moments_count(N: int, degree: int, bg_degree: int) -> int:
    return int(load_library().svk_fit_moments_count(int(N), int(degree), int(bg_degree)))


def svk_fit_moments_workspace_size(n_stamps: int, stamp_size: int, N: int) -> int:
    return int(load_library().svk_fit_moments_workspace_size(int(n_stamps), int(stamp_size), int(N)))


def svk_fit_moments(R, I, stamp_xy, stamp_size: int, basis, degree: int, bg_degree: int = -1, W: int | None = None,
                    H: int | None = None, row_begin: int = 0, weight=None, moments=None, accumulate: bool = False,
                    workspace=None, stream=None):
    """FP64 moments of the stamps' pixels (the summable part of the fit).

    R, I (and weight) hold the frame rows [row_begin, row_begin + rows) of a W x H frame
    (W, H default to R's own shape: a whole frame).  Returns the moments tensor (float64,
    svk_fit_moments_count entries), new or the given one (added to when `accumulate`)."""
    import torch
    rows, Wb, p = _img(R, "R")
    _, _, pI = _img(I, "I")
    if pI != p or (weight is not None and weight.stride(0) != p):
        raise ValueError("R, I and weight must share one pitch")
    W = Wb if W is None else int(W)
    H = rows if H is None else int(H)
    N, L = basis.shape[0], basis.shape[1]
    if moments is None:
        moments = torch.zeros(svk_fit_moments_count(N, degree, bg_degree), dtype=torch.float64, device=R.device)
    st = stamp_xy.to(torch.int32).contiguous() if stamp_xy is not None else None
    n = 0 if st is None else st.shape[0]
    ws_bytes = 0 if workspace is None else workspace.numel() * workspace.element_size()
    _check(load_library().svk_fit_moments(_ptr(R), _ptr(I), _ptr(weight), W, H, p, int(row_begin),
                                          int(row_begin) + rows, _ptr(st) if n else _ptr(None), n, int(stamp_size),
                                          _ptr(basis), N, L, int(degree), int(bg_degree), _ptr(moments),
                                          int(bool(accumulate)), _ptr(workspace), ws_bytes, _stream(stream)))
    return moments


def svk_fit_solve_workspace_size(N: int, degree: int, bg_degree: int) -> int:
    return int(load_library().svk_fit_solve_workspace_size(int(N), int(degree), int(bg_degree)))


def svk_fit_solve(moments, N: int, degree: int, bg_degree: int = -1, workspace=None, sync: bool = False, stream=None):
    """Coefficients from (summed) moments; returns (coeffs[M] f64, chi2[1] f64, info[1] i32) tensors."""
    import torch
    M = N * n_terms(degree) + n_terms(bg_degree)
    coeffs = torch.zeros(M, dtype=torch.float64, device=moments.device)
    chi2 = torch.zeros(1, dtype=torch.float64, device=moments.device)
    info = torch.zeros(1, dtype=torch.int32, device=moments.device)
    ws_bytes = 0 if workspace is None else workspace.numel() * workspace.element_size()
    _check(load_library().svk_fit_solve(_ptr(moments), int(N), int(degree), int(bg_degree), _ptr(coeffs), _ptr(chi2),
                                        _ptr(info), _ptr(workspace), ws_bytes, int(bool(sync)), _stream(stream)))
    return coeffs, chi2, info


def svk_band_rows(method: int, precision: int, N: int, L: int, degree: int) -> int:
    return int(load_library().svk_band_rows(int(method), int(precision), int(N), int(L), int(degree)))


def svk_difference_rows(R, I, basis, coeffs, degree: int, W: int, H: int, y_begin: int, y_end: int, r_begin: int,
                        method: int = SVK_METHOD_BASIS, precision: int = SVK_PREC_BF16X3, out=None, workspace=None,
                        stream=None, edge: int = SVK_EDGE_ZERO):
    """Rows [y_begin, y_end) of D = (R (x) K) - I for a W x H frame from band buffers:
    R holds frame rows [r_begin, r_begin + R.shape[0]), I and out rows [y_begin, y_end)
    (I may be None: out = R (x) K)."""
    import torch
    rows, Wb, pR = _img(R, "R")
    if Wb != W:
        raise ValueError("R's width differs from W")
    pI = 0
    if I is not None:
        Hi, Wi, pI = _img(I, "I")
        if (Hi, Wi) != (y_end - y_begin, W):
            raise ValueError("I must hold the band's rows")
    if out is None:
        out = torch.empty((y_end - y_begin, W), dtype=torch.float32, device=R.device)
    _, _, pD = _img(out, "D")
    N, L = basis.shape[0], basis.shape[1]
    ws_bytes = 0 if workspace is None else workspace.numel() * workspace.element_size()
    _check(load_library().svk_difference_rows(_ptr(R), pR, int(r_begin), int(r_begin) + rows, _ptr(I), pI, _ptr(out),
                                              pD, int(W), int(H), int(y_begin), int(y_end), _ptr(basis), N, L,
                                              _ptr(coeffs), int(degree), int(method), int(precision), int(edge),
                                              _ptr(workspace), ws_bytes, _stream(stream)))
    return out


def svk_host_workspace_size(method: int, precision: int, W: int, H: int, N: int, L: int, degree: int) -> int:
    return int(load_library().svk_host_workspace_size(method, precision, W, H, N, L, degree))


def svk_difference_host(R, I, basis, coeffs, degree: int, method: int = SVK_METHOD_BASIS,
                        precision: int = SVK_PREC_BF16X3, out=None, n_bands: int = 8, workspace=None, stream=None):
    """D = (R (x) K_{x,y}) - I with R, I and D in host memory (CPU float32 [H][pitch]
    tensors; pin them for copy/compute overlap).  Asynchronous on the stream: D is valid
    after the stream is synchronised."""
    import torch
    for name, t in (("R", R), ("I", I)):
        if t.dtype != torch.float32 or t.is_cuda or t.dim() != 2 or t.stride(1) != 1:
            raise ValueError(f"{name} must be a host float32 [H][pitch] tensor with unit column stride")
    if R.shape != I.shape or R.stride(0) != I.stride(0):
        raise ValueError("R and I must have one shape and pitch")
    H, W = R.shape
    if out is None:
        out = torch.empty_strided((H, W), (R.stride(0), 1), dtype=torch.float32, pin_memory=R.is_pinned())
    if out.shape != R.shape or out.stride(0) != R.stride(0) or out.is_cuda:
        raise ValueError("out must be a host tensor with the shape and pitch of R")
    N, L = basis.shape[0], basis.shape[1]
    ws_bytes = 0 if workspace is None else workspace.numel() * workspace.element_size()
    _check(load_library().svk_difference_host(_ptr(R), _ptr(I), _ptr(out), W, H, R.stride(0), _ptr(basis), N, L,
                                              _ptr(coeffs), int(degree), int(method), int(precision), int(n_bands),
                                              _ptr(workspace), ws_bytes, _stream(stream)))
    return out


def svk_host_batch_workspace_size(items, method: int = SVK_METHOD_BASIS, precision: int = SVK_PREC_BF16X3) -> int:
    arr = _frames(items, host=True)
    return int(load_library().svk_host_batch_workspace_size(ctypes.cast(arr, ctypes.c_void_p), len(items), int(method),
                                                            int(precision)))


def svk_difference_host_batch(items, method: int = SVK_METHOD_BASIS, precision: int = SVK_PREC_BF16X3,
                              n_bands: int = 2, workspace=None, stream=None):
    """D = (R (x) K) - I for a sequence of frames in host memory: each item a dict with host
    float32 [H][pitch] tensors R, I, D (pinned for overlap) and device basis, coeffs, degree.
    Frames are pipelined (the next frame's copies in and the previous frame's copies out
    overlap the current frame's computation).  Asynchronous on the stream."""
    arr = _frames(items, host=True)
    ws_bytes = 0 if workspace is None else workspace.numel() * workspace.element_size()
    _check(load_library().svk_difference_host_batch(ctypes.cast(arr, ctypes.c_void_p), len(items), int(method),
                                                    int(precision), int(n_bands), _ptr(workspace), ws_bytes,
                                                    _stream(stream)))


def svk_device_status(reset: bool = False, stream=None) -> int:
    """Synchronise the stream and return the library's sticky device status (SVK_OK, or
    SVK_ERR_TIMEOUT after a bounded device wait gave up); clears it when `reset`."""
    return int(load_library().svk_device_status(int(bool(reset)), _stream(stream)))


def svk_selftest_bounded_wait(limit_ns: int, stream=None):
    """Run the bounded-wait self-test; returns (status, waited_ns).  status is
    SVK_ERR_TIMEOUT when the wait gave up as designed."""
    w = ctypes.c_ulonglong(0)
    st = int(load_library().svk_selftest_bounded_wait(int(limit_ns), ctypes.byref(w), _stream(stream)))
    return st, int(w.value)


def svk_measure_fma_peak(kind: int = SVK_FMA_FP32, stream=None) -> float:
    """Measured multiply-add throughput of the current device, FLOP/s: SVK_FMA_FP32
    (scalar FFMA; also False), SVK_FMA_FP64 (DFMA; also True) or SVK_FMA_FP32X2 (packed)."""
    v = ctypes.c_double(0.0)
    _check(load_library().svk_measure_fma_peak(int(kind), ctypes.byref(v), _stream(stream)))
    return v.value


def svk_select_workspace_size(W: int, H: int) -> int:
    return int(load_library().svk_select_workspace_size(int(W), int(H)))


def svk_select_stamps(R, sky: float, threshold: float, saturation: float, margin: int, iso_radius: int,
                      iso_frac: float, max_stamps: int, workspace=None, stream=None):
    """Stamp centres of isolated, unsaturated peaks of R, brightest first.

    Returns (xy int32 [max_stamps][2], counts int32 [2] = {written, peaks}) on the device;
    rows of xy past counts[0] are zero."""
    import torch
    H, W, p = _img(R, "R")
    xy = torch.zeros((max(int(max_stamps), 0), 2), dtype=torch.int32, device=R.device)
    counts = torch.zeros(2, dtype=torch.int32, device=R.device)
    ws_bytes = 0 if workspace is None else workspace.numel() * workspace.element_size()
    _check(load_library().svk_select_stamps(_ptr(R), W, H, p, float(sky), float(threshold), float(saturation),
                                            int(margin), int(iso_radius), float(iso_frac), int(max_stamps),
                                            _ptr(xy) if max_stamps > 0 else _ptr(None), _ptr(counts),
                                            _ptr(workspace), ws_bytes, _stream(stream)))
    return xy, counts


def svk_cut_stamps(img, xy, size: int, offset: float = 0.0, divisor: float = 1.0, out=None, stamp_stride=None,
                   stream=None):
    """Stamps of img around the int32 [n][2] centres xy, (value - offset) / divisor, zero
    outside the image; returns out ([n][size][size] float32 unless given with its stride)."""
    import torch
    H, W, p = _img(img, "img")
    xy = xy.to(torch.int32).contiguous()
    n = xy.shape[0]
    if out is None:
        out = torch.empty((n, size, size), dtype=torch.float32, device=img.device)
        stamp_stride = size * size
    elif stamp_stride is None:
        stamp_stride = size * size
    _check(load_library().svk_cut_stamps(_ptr(img), W, H, p, _ptr(xy), n, int(size), float(offset), float(divisor),
                                         _ptr(out), int(stamp_stride), _stream(stream)))
    return out


def svk_stamp_residual(D, xy, size: int, basis0, noise_sigma: float, ref_noise_sigma: float, ratio: float,
                       field_info=None, workspace=None, stream=None):
    """(out [2] f64 = {chi2_per_px, floor}, fallback [1] i32) device tensors."""
    import torch
    H, W, p = _img(D, "D")
    xy = xy.to(torch.int32).contiguous()
    out = torch.zeros(2, dtype=torch.float64, device=D.device)
    fb = torch.zeros(1, dtype=torch.int32, device=D.device)
    ws_bytes = 0 if workspace is None else workspace.numel() * workspace.element_size()
    _check(load_library().svk_stamp_residual(_ptr(D), W, H, p, _ptr(xy), xy.shape[0], int(size), _ptr(basis0),
                                             basis0.shape[-1], float(noise_sigma), float(ref_noise_sigma), float(ratio),
                                             _ptr(field_info), _ptr(out), _ptr(fb), _ptr(workspace), ws_bytes,
                                             _stream(stream)))
    return out, fb


def svk_cnn_standardise(x, mean, sd, inverse: bool = False, out=None, stream=None):
    """(x - mean) / sd per column, or mean + sd * x (inverse); x float32 [rows][cols]."""
    import torch
    x = x.contiguous()
    if out is None:
        out = torch.empty_like(x)
    _check(load_library().svk_cnn_standardise(_ptr(x), x.shape[0], x.shape[1], _ptr(mean), _ptr(sd),
                                              int(bool(inverse)), _ptr(out), _stream(stream)))
    return out


def svk_cnn_draw_batch(seed: int, step, n: int, idx_out, stream=None):
    _check(load_library().svk_cnn_draw_batch(int(seed) & 0xFFFFFFFFFFFFFFFF, _ptr(step), int(n), idx_out.numel(),
                                             _ptr(idx_out), _stream(stream)))
    return idx_out


def svk_gather_rows(src, idx, out, stream=None):
    """out[i] = src[idx[i]] along the first dimension (contiguous tensors)."""
    row_bytes = src[0].numel() * src.element_size()
    _check(load_library().svk_gather_rows(_ptr(src), int(row_bytes), _ptr(idx), idx.numel(), _ptr(out),
                                          _stream(stream)))
    return out


def svk_cnn_step_end(loss, step, history, stream=None):
    _check(load_library().svk_cnn_step_end(_ptr(loss), _ptr(step), _ptr(history), history.numel(), _stream(stream)))


# ---------------------------------------------------------------- coefficient network
def svk_cnn_param_count(n_out: int) -> int:
    return int(load_library().svk_cnn_param_count(int(n_out)))


def svk_cnn_workspace_size(batch: int, n_out: int) -> int:
    return int(load_library().svk_cnn_workspace_size(int(batch), int(n_out)))


def svk_cnn_forward(params, x, n_out: int, out=None, workspace=None, stream=None):
    """Local coefficients [batch][n_out] from normalised stamp pairs x [batch][2][64][64]."""
    import torch
    B = x.shape[0]
    if out is None:
        out = torch.empty((B, n_out), dtype=torch.float32, device=x.device)
    ws_bytes = 0 if workspace is None else workspace.numel() * workspace.element_size()
    _check(load_library().svk_cnn_forward(_ptr(params), _ptr(x), B, int(n_out), _ptr(out), _ptr(workspace), ws_bytes,
                                          _stream(stream)))
    return out


def svk_cnn_gradient(params, x, target, grad=None, loss=None, workspace=None, stream=None):
    """(grad [param_count], loss [1]) of the mean squared error against target."""
    import torch
    B, n_out = target.shape
    if grad is None:
        grad = torch.empty_like(params)
    if loss is None:
        loss = torch.empty(1, dtype=torch.float32, device=x.device)
    ws_bytes = 0 if workspace is None else workspace.numel() * workspace.element_size()
    _check(load_library().svk_cnn_gradient(_ptr(params), _ptr(x), _ptr(target), B, int(n_out), _ptr(grad), _ptr(loss),
                                           _ptr(workspace), ws_bytes, _stream(stream)))
    return grad, loss


def svk_cnn_adam(params, m, v, grad, step: int, lr: float = 1e-3, beta1: float = 0.9, beta2: float = 0.999,
                 eps: float = 1e-8, stream=None):
    _check(load_library().svk_cnn_adam(_ptr(params), _ptr(m), _ptr(v), _ptr(grad), params.numel(), int(step), lr,
                                       beta1, beta2, eps, _stream(stream)))


def svk_cnn_adam_device_step(params, m, v, grad, step, lr: float = 1e-3, beta1: float = 0.9, beta2: float = 0.999,
                             eps: float = 1e-8, stream=None):
    """svk_cnn_adam with the step count read from `step` (device int32 tensor of one element)."""
    _check(load_library().svk_cnn_adam_device_step(_ptr(params), _ptr(m), _ptr(v), _ptr(grad), params.numel(),
                                                   _ptr(step), lr, beta1, beta2, eps, _stream(stream)))


def svk_cnn_field_fit(local, xy, W: int, H: int, degree: int, weights=None, stream=None):
    """FP64 polynomial field c[k][t] from local predictions local [S][N] at stamp centres xy [S][2]."""
    import torch
    S, N = local.shape
    T = n_terms(degree)
    coeffs = torch.zeros((N, T), dtype=torch.float64, device=local.device)
    info = torch.zeros(1, dtype=torch.int32, device=local.device)
    xy32 = xy.to(torch.int32).contiguous()
    _check(load_library().svk_cnn_field_fit(_ptr(local), _ptr(xy32), _ptr(weights), S, N, int(W), int(H), int(degree),
                                            _ptr(coeffs), _ptr(info), _stream(stream)))
    return coeffs, info
