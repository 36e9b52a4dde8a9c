"""FP64 CPU oracle for the spatially-varying kernel convolution (test infrastructure).

Only ``tests/``, ``__graft_entry__.smoke()`` and ``bench.py``'s CPU-baseline leg may
import this package.  The CUDA library never calls it, and it shares no code with it.

The arithmetic lives in ``svk_oracle.c`` (plain C, FP64), compiled on first use with
``gcc -O2 -fopenmp``; this module only marshals numpy arrays.  The readings of the paper
that the oracle adopts are listed in the C file's header.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "svk_oracle.c")
_LIB_PATH = os.path.join(_HERE, "libsvk_oracle.so")
_lock = threading.Lock()
_lib = None

NORM_NONE = 0
NORM_ALARD = 1
OK = 0
ERR_NOT_SPD = 3


def build(force: bool = False) -> str:
    """Compile the oracle shared library (gcc; OpenMP when available)."""
    if not force and os.path.exists(_LIB_PATH) and os.path.getmtime(_LIB_PATH) >= os.path.getmtime(_SRC):
        return _LIB_PATH
    tmp = _LIB_PATH + f".tmp{os.getpid()}"
    base = ["gcc", "-O2", "-fPIC", "-shared", "-o", tmp, _SRC, "-lm"]
    try:
        subprocess.run(base[:1] + ["-fopenmp"] + base[1:], check=True, capture_output=True)
    except subprocess.CalledProcessError:
        subprocess.run(base, check=True, capture_output=True)
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _load():
    global _lib
    with _lock:
        if _lib is None:
            lib = ctypes.CDLL(build())
            D = ctypes.POINTER(ctypes.c_double)
            I = ctypes.POINTER(ctypes.c_int)
            c_int, c_double = ctypes.c_int, ctypes.c_double
            sig = {
                "svko_set_threads": (None, [c_int]),
                "svko_get_threads": (c_int, []),
                "svko_n_terms": (c_int, [c_int]),
                "svko_norm_coord": (c_double, [c_int, c_int]),
                "svko_monomials": (None, [c_double, c_double, c_int, D]),
                "svko_gauss_basis_count": (c_int, [c_int, I]),
                "svko_gauss_basis": (c_int, [c_int, c_int, D, I, c_int, D]),
                "svko_delta_basis": (c_int, [c_int, c_int, D]),
                "svko_convolve_rows": (c_int, [D, c_int, c_int, D, c_int, c_int, D, c_int, c_int, c_int, D]),
                "svko_convolve": (c_int, [D, c_int, c_int, D, c_int, c_int, D, c_int, D]),
                "svko_convolve_points": (c_int, [D, c_int, c_int, D, c_int, c_int, D, c_int, I, I, c_int, D]),
                "svko_difference": (c_int, [D, D, c_int, c_int, D, c_int, c_int, D, c_int, D]),
                "svko_cholesky": (c_int, [D, c_int]),
                "svko_cholesky_solve": (None, [D, c_int, D, D]),
                "svko_normal_equations": (c_int, [D, D, c_int, c_int, I, c_int, c_int, D, c_int, c_int,
                                                  c_int, c_int, D, D, D]),
                "svko_chi2": (c_double, [D, D, c_int, c_int, I, c_int, c_int, D, c_int, c_int, c_int,
                                         c_int, D, D]),
                "svko_fit": (c_int, [D, D, c_int, c_int, I, c_int, c_int, D, c_int, c_int, c_int, c_int,
                                     D, D, D, D, D, I]),
                "svko_flops_dfb_per_pixel": (c_double, [c_int]),
                "svko_flops_gfb_per_pixel": (c_double, [c_int, c_int]),
            }
            for name, (res, args) in sig.items():
                f = getattr(lib, name)
                f.restype = res
                f.argtypes = args
            _lib = lib
    return _lib


def _d(a):
    a = np.ascontiguousarray(a, dtype=np.float64)
    return a, a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def _i(a):
    a = np.ascontiguousarray(a, dtype=np.int32)
    return a, a.ctypes.data_as(ctypes.POINTER(ctypes.c_int))


_NULLD = ctypes.POINTER(ctypes.c_double)()


def set_threads(n: int) -> None:
    _load().svko_set_threads(int(n))


def get_threads() -> int:
    return int(_load().svko_get_threads())


def n_terms(d: int) -> int:
    return int(_load().svko_n_terms(int(d)))


def norm_coord(x: int, W: int) -> float:
    return float(_load().svko_norm_coord(int(x), int(W)))


def monomials(xt: float, yt: float, d: int) -> np.ndarray:
    m = np.zeros(max(1, n_terms(d)), dtype=np.float64)
    _load().svko_monomials(float(xt), float(yt), int(d), m.ctypes.data_as(ctypes.POINTER(ctypes.c_double)))
    return m[: n_terms(d)]


def gauss_basis(L: int, sigma=(0.7, 1.5, 2.5), deg=(6, 4, 2), normalize: int = NORM_ALARD) -> np.ndarray:
    lib = _load()
    s, sp = _d(sigma)
    g, gp = _i(deg)
    N = lib.svko_gauss_basis_count(len(sigma), gp)
    out = np.zeros((N, L, L), dtype=np.float64)
    n = lib.svko_gauss_basis(int(L), len(sigma), sp, gp, int(normalize),
                             out.ctypes.data_as(ctypes.POINTER(ctypes.c_double)))
    if n != N:
        raise ValueError("bad basis arguments")
    return out


def delta_basis(L: int, normalize: int = NORM_NONE) -> np.ndarray:
    out = np.zeros((L * L, L, L), dtype=np.float64)
    n = _load().svko_delta_basis(int(L), int(normalize), out.ctypes.data_as(ctypes.POINTER(ctypes.c_double)))
    if n != L * L:
        raise ValueError("bad basis arguments")
    return out


def _check_conv_args(R, basis, coeffs, degree):
    R, Rp = _d(R)
    B, Bp = _d(basis)
    C, Cp = _d(coeffs)
    H, W = R.shape
    N, L, L2 = B.shape
    assert L == L2 and C.shape == (N, n_terms(degree)), (C.shape, N, degree)
    return R, Rp, B, Bp, C, Cp, H, W, N, L


def convolve(R, basis, coeffs, degree: int, rows=None) -> np.ndarray:
    """R (x) K_{x,y} (Eq. 1-3) over the whole frame, or over rows [y0, y1)."""
    R, Rp, B, Bp, C, Cp, H, W, N, L = _check_conv_args(R, basis, coeffs, degree)
    y0, y1 = (0, H) if rows is None else rows
    out = np.empty((y1 - y0, W), dtype=np.float64)
    st = _load().svko_convolve_rows(Rp, W, H, Bp, N, L, Cp, int(degree), int(y0), int(y1),
                                    out.ctypes.data_as(ctypes.POINTER(ctypes.c_double)))
    if st != OK:
        raise ValueError(f"oracle convolve: status {st}")
    return out


def convolve_points(R, basis, coeffs, degree: int, px, py) -> np.ndarray:
    R, Rp, B, Bp, C, Cp, H, W, N, L = _check_conv_args(R, basis, coeffs, degree)
    X, Xp = _i(px)
    Y, Yp = _i(py)
    out = np.empty(len(X), dtype=np.float64)
    st = _load().svko_convolve_points(Rp, W, H, Bp, N, L, Cp, int(degree), Xp, Yp, len(X),
                                      out.ctypes.data_as(ctypes.POINTER(ctypes.c_double)))
    if st != OK:
        raise ValueError(f"oracle convolve_points: status {st}")
    return out


def difference(R, I, basis, coeffs, degree: int) -> np.ndarray:
    """D = (R (x) K) - I, Eq. 1."""
    R, Rp, B, Bp, C, Cp, H, W, N, L = _check_conv_args(R, basis, coeffs, degree)
    Iv, Ip = _d(I)
    out = np.empty((H, W), dtype=np.float64)
    st = _load().svko_difference(Rp, Ip, W, H, Bp, N, L, Cp, int(degree),
                                 out.ctypes.data_as(ctypes.POINTER(ctypes.c_double)))
    if st != OK:
        raise ValueError(f"oracle difference: status {st}")
    return out


def cholesky(A) -> tuple[np.ndarray, int]:
    """Lower Cholesky factor (textbook); returns (G, pivot) with pivot -1 on success."""
    G = np.array(A, dtype=np.float64, copy=True, order="C")
    piv = _load().svko_cholesky(G.ctypes.data_as(ctypes.POINTER(ctypes.c_double)), G.shape[0])
    return np.tril(G), int(piv)


def cholesky_solve(G, b) -> np.ndarray:
    G, Gp = _d(G)
    b, bp = _d(b)
    x = np.empty_like(b)
    _load().svko_cholesky_solve(Gp, G.shape[0], bp, x.ctypes.data_as(ctypes.POINTER(ctypes.c_double)))
    return x


def _fit_common(R, I, stamps, S, basis, degree, bg_degree, weight):
    R, Rp = _d(R)
    Iv, Ip = _d(I)
    st, sp = _i(np.asarray(stamps).reshape(-1, 2))
    B, Bp = _d(basis)
    H, W = R.shape
    N, L, _ = B.shape
    if weight is None:
        wv, wp = None, _NULLD
    else:
        wv, wp = _d(weight)
    M = N * n_terms(degree) + n_terms(bg_degree)
    keep = (R, Iv, st, B, wv)
    return keep, Rp, Ip, sp, len(st), Bp, W, H, N, L, wp, M


def normal_equations(R, I, stamps, S, basis, degree, bg_degree=-1, weight=None):
    keep, Rp, Ip, sp, ns, Bp, W, H, N, L, wp, M = _fit_common(R, I, stamps, S, basis, degree, bg_degree, weight)
    A = np.empty((M, M), dtype=np.float64)
    b = np.empty(M, dtype=np.float64)
    st = _load().svko_normal_equations(Rp, Ip, W, H, sp, ns, int(S), Bp, N, L, int(degree), int(bg_degree), wp,
                                       A.ctypes.data_as(ctypes.POINTER(ctypes.c_double)),
                                       b.ctypes.data_as(ctypes.POINTER(ctypes.c_double)))
    if st != OK:
        raise ValueError(f"oracle normal_equations: status {st}")
    return A, b


def chi2(R, I, stamps, S, basis, degree, c, bg_degree=-1, weight=None) -> float:
    keep, Rp, Ip, sp, ns, Bp, W, H, N, L, wp, M = _fit_common(R, I, stamps, S, basis, degree, bg_degree, weight)
    cv, cp = _d(c)
    return float(_load().svko_chi2(Rp, Ip, W, H, sp, ns, int(S), Bp, N, L, int(degree), int(bg_degree), wp, cp))


def fit(R, I, stamps, S, basis, degree, bg_degree=-1, weight=None):
    """OIS least-squares fit; returns dict(coeffs, chi2, A, b, status, info)."""
    keep, Rp, Ip, sp, ns, Bp, W, H, N, L, wp, M = _fit_common(R, I, stamps, S, basis, degree, bg_degree, weight)
    c = np.zeros(M, dtype=np.float64)
    A = np.empty((M, M), dtype=np.float64)
    b = np.empty(M, dtype=np.float64)
    x2 = ctypes.c_double(0.0)
    info = ctypes.c_int(0)
    st = _load().svko_fit(Rp, Ip, W, H, sp, ns, int(S), Bp, N, L, int(degree), int(bg_degree), wp,
                          c.ctypes.data_as(ctypes.POINTER(ctypes.c_double)), ctypes.byref(x2),
                          A.ctypes.data_as(ctypes.POINTER(ctypes.c_double)),
                          b.ctypes.data_as(ctypes.POINTER(ctypes.c_double)), ctypes.byref(info))
    return dict(coeffs=c, chi2=float(x2.value), A=A, b=b, status=int(st), info=int(info.value))


def flops_dfb_per_pixel(L: int) -> float:
    return float(_load().svko_flops_dfb_per_pixel(int(L)))


def flops_gfb_per_pixel(N: int, L: int) -> float:
    return float(_load().svko_flops_gfb_per_pixel(int(N), int(L)))
