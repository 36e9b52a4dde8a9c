"""The C ABI library loads, exports every symbol include/svk.h declares, and rejects bad
arguments on the host (no CUDA call is made, so these run without a GPU)."""
import ctypes
import os
import re

import pytest

import paper_1209_5823_gb300 as svk
from paper_1209_5823_gb300 import build as svk_build

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    svk_build.build()
    return svk.load_library()


def declared_symbols():
    names = []
    for h in sorted(os.listdir(os.path.join(ROOT, "include"))):
        if h.endswith(".h"):
            txt = open(os.path.join(ROOT, "include", h)).read()
            names += re.findall(r"SVK_API\s+[\w\s\*]*?\b(svk_\w+)\s*\(", txt)
    return names


def test_header_declares_the_binding_exports():
    assert set(declared_symbols()) == set(svk.EXPORTS)


def test_library_exports_every_declared_symbol(lib):
    for name in declared_symbols():
        assert hasattr(lib, name), name
    assert lib.svk_version() == 1


def test_gauss_basis_count(lib):
    deg = (ctypes.c_int * 3)(6, 4, 2)
    assert lib.svk_gauss_basis_count(3, deg) == 49
    bad = (ctypes.c_int * 1)(-1)
    assert lib.svk_gauss_basis_count(1, bad) == -1


def _conv(lib, **kw):
    a = dict(R=1, W=64, H=64, pR=64, B=1, N=49, L=11, C=1, d=2, method=0, prec=0, edge=0, out=1, pO=64)
    a.update(kw)
    vp = ctypes.c_void_p
    return lib.svk_convolve(vp(a["R"]), a["W"], a["H"], a["pR"], vp(a["B"]), a["N"], a["L"], vp(a["C"]), a["d"],
                            a["method"], a["prec"], a["edge"], vp(a["out"]), a["pO"], vp(0), 0, vp(0))


@pytest.mark.parametrize("kw,status", [
    (dict(L=10), svk.SVK_ERR_ARG), (dict(L=33), svk.SVK_ERR_ARG), (dict(R=0), svk.SVK_ERR_ARG),
    (dict(pR=63), svk.SVK_ERR_ARG), (dict(W=0), svk.SVK_ERR_ARG), (dict(d=4), svk.SVK_ERR_ARG),
    (dict(N=0), svk.SVK_ERR_ARG), (dict(edge=1), svk.SVK_ERR_ARG), (dict(method=7), svk.SVK_ERR_ARG),
    (dict(method=0, prec=1), svk.SVK_ERR_UNSUPPORTED), (dict(method=1, prec=0), svk.SVK_ERR_UNSUPPORTED),
    (dict(method=1, prec=1, N=300), svk.SVK_ERR_UNSUPPORTED), (dict(method=2, prec=7), svk.SVK_ERR_UNSUPPORTED),
])
def test_host_argument_checks(lib, kw, status):
    assert _conv(lib, **kw) == status
    assert lib.svk_last_error().decode() != ""


def test_build_basis_argument_checks(lib):
    vp = ctypes.c_void_p
    sg = (ctypes.c_double * 1)(1.0)
    dg = (ctypes.c_int * 1)(2)
    assert lib.svk_build_basis(0, 4, 1, sg, dg, 1, vp(1), None, vp(0)) == svk.SVK_ERR_ARG
    assert lib.svk_build_basis(0, 5, 1, sg, dg, 1, vp(0), None, vp(0)) == svk.SVK_ERR_ARG
    assert lib.svk_build_basis(5, 5, 1, sg, dg, 1, vp(1), None, vp(0)) == svk.SVK_ERR_ARG
    neg = (ctypes.c_double * 1)(-1.0)
    assert lib.svk_build_basis(0, 5, 1, neg, dg, 1, vp(1), None, vp(0)) == svk.SVK_ERR_ARG


def test_fma_peak_argument_checks(lib):
    v = ctypes.c_double(0.0)
    assert lib.svk_measure_fma_peak(3, ctypes.byref(v), None) == svk.SVK_ERR_ARG
    assert lib.svk_measure_fma_peak(-1, ctypes.byref(v), None) == svk.SVK_ERR_ARG
    assert lib.svk_measure_fma_peak(svk.SVK_FMA_FP32X2, None, None) == svk.SVK_ERR_ARG


def test_fit_argument_checks(lib):
    vp = ctypes.c_void_p
    f = lambda **k: lib.svk_fit_coeffs(vp(1), vp(1), k.get("W", 64), 64, 64, vp(1), k.get("ns", 4),
                                       k.get("S", 9), vp(1), k.get("N", 49), 11, k.get("d", 2), k.get("bd", -1),
                                       vp(0), vp(1), vp(0), vp(1), vp(0), 0, 0, vp(0))
    assert f(S=8) == svk.SVK_ERR_ARG
    assert f(ns=0) == svk.SVK_ERR_ARG
    assert f(d=5) == svk.SVK_ERR_ARG
    assert f(N=200, d=3) == svk.SVK_ERR_ARG  # M = 2000 > 1024
