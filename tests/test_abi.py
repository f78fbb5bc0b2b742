"""The C ABI library loads, exports every entry point of include/sal.h, and rejects bad
arguments on the host before launching anything (no GPU needed)."""
import ctypes
import os
import re

import pytest

from paper_1901_11095_gb300 import _native as N
from paper_1901_11095_gb300 import build as B

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    B.build()
    return N.lib()


def header_symbols():
    txt = open(os.path.join(ROOT, "include", "sal.h")).read()
    return sorted(set(re.findall(r"SAL_API\s+[\w\s\*]*?\b(sal_\w+)\s*\(", txt)))


def test_exports_every_declared_symbol(lib):
    names = header_symbols()
    assert len(names) >= 11
    for n in names:
        assert hasattr(lib, n), n
    assert sorted(N.exported_symbols()) == sorted(names)


def test_params_default(lib):
    p = N.SalParams()
    assert lib.sal_params_default(ctypes.byref(p)) == N.SAL_OK
    assert (p.L, p.precision, p.boundary, p.stencil) == (7, 0, 0, 0)
    assert p.sigma == 1.0 and abs(p.a - 1 / 3) < 1e-15 and p.eps == 1e-6


def _p(lib, **kw):
    p = N.SalParams()
    lib.sal_params_default(ctypes.byref(p))
    for k, v in kw.items():
        setattr(p, k, v)
    return p


def test_workspace_size_grows_with_volume(lib):
    p = _p(lib)
    a, b = ctypes.c_size_t(), ctypes.c_size_t()
    assert lib.sal_workspace_size(N.SalDims(64, 64, 64), ctypes.byref(p), ctypes.byref(a)) == 0
    assert lib.sal_workspace_size(N.SalDims(128, 64, 64), ctypes.byref(p), ctypes.byref(b)) == 0
    assert b.value > a.value >= 24 * 64 ** 3
    assert a.value % 256 == 0


@pytest.mark.parametrize("field,val,status", [
    ("L", 6, N.SAL_ERR_UNSUPPORTED), ("L", 1, N.SAL_ERR_INVALID_ARG), ("L", 17, N.SAL_ERR_INVALID_ARG),
    ("precision", 7, N.SAL_ERR_INVALID_ARG), ("boundary", 2, N.SAL_ERR_INVALID_ARG),
    ("stencil", 5, N.SAL_ERR_INVALID_ARG), ("sigma", 0.0, N.SAL_ERR_INVALID_ARG),
    ("sigma", float("nan"), N.SAL_ERR_INVALID_ARG), ("eps", -1.0, N.SAL_ERR_INVALID_ARG),
    ("stride", 4, N.SAL_ERR_INVALID_ARG), ("stride", -1, N.SAL_ERR_INVALID_ARG)])
def test_bad_params_rejected(lib, field, val, status):
    p = _p(lib, **{field: val})
    n = ctypes.c_size_t()
    assert lib.sal_workspace_size(N.SalDims(8, 8, 8), ctypes.byref(p), ctypes.byref(n)) == status
    assert lib.sal_last_error().decode()


def test_bad_dims_and_pointers_rejected(lib):
    p = _p(lib)
    n = ctypes.c_size_t()
    assert lib.sal_workspace_size(N.SalDims(0, 8, 8), ctypes.byref(p), ctypes.byref(n)) == N.SAL_ERR_INVALID_ARG
    d = N.SalDims(8, 8, 8)
    assert lib.sal_saliency(None, d, ctypes.byref(p), None, None, None, 0, None) == N.SAL_ERR_INVALID_ARG
    assert lib.sal_spectral_energy(16, d, ctypes.byref(p), None, None) == N.SAL_ERR_INVALID_ARG
    # misaligned device pointers are refused before any launch
    assert lib.sal_spectral_energy(20, d, ctypes.byref(p), 64, None) == N.SAL_ERR_INVALID_ARG
    # a workspace below the queried size is refused
    assert lib.sal_saliency(256, d, ctypes.byref(p), 512, None, 1024, 16, None) == N.SAL_ERR_WORKSPACE
    lo = (ctypes.c_int64 * 3)(0, 0, 0)
    ext = (ctypes.c_int64 * 3)(9, 1, 1)
    assert lib.sal_local_spectra(256, d, ctypes.byref(p), lo, ext, 512, None) == N.SAL_ERR_INVALID_ARG
    assert lib.sal_project(256, 4, 8, 512, None) == N.SAL_ERR_UNSUPPORTED


def test_status_strings(lib):
    for s in range(7):
        assert lib.sal_status_string(s).decode().startswith("SAL_")


def test_host_entry_argument_checks(lib):
    p = _p(lib)
    d = N.SalDims(8, 8, 8)
    n = ctypes.c_size_t()
    assert lib.sal_host_workspace_size(d, ctypes.byref(p), ctypes.byref(n)) == 0
    # two V, E, S_m and two S buffers (10 N floats) plus the reduction records
    assert n.value >= 40 * 8 ** 3 and n.value % 256 == 0
    assert lib.sal_saliency_host(None, d, ctypes.byref(p), None, None, None, 0, None, None) == N.SAL_ERR_INVALID_ARG
    buf = (ctypes.c_float * 512)()
    # a workspace below the queried size is refused before any copy or launch
    assert lib.sal_saliency_host(buf, d, ctypes.byref(p), buf, None, 256, 16, None, None) == N.SAL_ERR_WORKSPACE
    assert lib.sal_host_release(None) == N.SAL_ERR_INVALID_ARG
    assert lib.sal_host_release(256) == N.SAL_OK          # never used: nothing to release
