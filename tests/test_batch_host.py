"""Host-side behaviour of the batched calls and the autotuner cache (no GPU needed)."""
import ctypes

import pytest

from paper_1901_11095_gb300 import _native as N
from paper_1901_11095_gb300 import build as B


@pytest.fixture(scope="module")
def lib():
    B.build()
    return N.lib()


def _params(lib, **kw):
    p = N.SalParams()
    lib.sal_params_default(ctypes.byref(p))
    for k, v in kw.items():
        setattr(p, k, v)
    return p


def _vols(shapes):
    arr = (N.SalVolume * len(shapes))()
    for i, s in enumerate(shapes):
        arr[i] = N.SalVolume(None, None, *s)
    return arr


def test_batch_workspace_is_sum_of_volumes(lib):
    p = _params(lib)
    one, two = ctypes.c_size_t(), ctypes.c_size_t()
    assert lib.sal_batch_workspace_size(_vols([(40, 50, 60)]), 1, ctypes.byref(p), ctypes.byref(one)) == 0
    assert lib.sal_batch_workspace_size(_vols([(40, 50, 60), (40, 50, 60)]), 2, ctypes.byref(p), ctypes.byref(two)) == 0
    assert two.value >= 2 * 24 * 40 * 50 * 60 and two.value > one.value


def test_batch_argument_checks(lib):
    p = _params(lib)
    n = ctypes.c_size_t()
    assert lib.sal_batch_workspace_size(_vols([(4, 4, 4)]), 0, ctypes.byref(p), ctypes.byref(n)) == N.SAL_ERR_INVALID_ARG
    big = [(4, 4, 4)] * (N.SAL_BATCH_MAX + 1)
    assert lib.sal_batch_workspace_size(_vols(big), len(big), ctypes.byref(p), ctypes.byref(n)) == N.SAL_ERR_INVALID_ARG
    assert lib.sal_batch_workspace_size(_vols([(4, 0, 4)]), 1, ctypes.byref(p), ctypes.byref(n)) == N.SAL_ERR_INVALID_ARG
    # NULL device pointers are refused before any launch
    assert lib.sal_saliency_batched(_vols([(4, 4, 4)]), 1, ctypes.byref(p), None, 256, 1 << 20, None) == \
        N.SAL_ERR_INVALID_ARG
    h = ctypes.c_void_p()
    assert lib.sal_graph_create_batched(_vols([(4, 4, 4)]), 1, ctypes.byref(p), None, 256, 1 << 20, None,
                                        ctypes.byref(h)) == N.SAL_ERR_INVALID_ARG
    assert lib.sal_graph_destroy(None) == 0


def test_autotune_cache_roundtrip_and_corrupt_file(lib, tmp_path):
    assert lib.sal_autotune_clear() == 0
    c = N.SalTileChoice()
    assert lib.sal_autotune_query(7, 0, 286_000_000, ctypes.byref(c)) == 0
    assert (c.shape, c.ms) == (0, 0.0) and (c.bt, c.bx, c.by, c.mode) == (2, 8, 32, 4)
    # the defaults: batched spectra (mode 4) for L = 7 and 9, mode 0 elsewhere
    for L, want in ((3, (2, 8, 32, 0)), (5, (2, 8, 32, 0)), (9, (2, 8, 32, 4)), (11, (2, 16, 32, 0))):
        assert lib.sal_autotune_query(L, 0, 1000, ctypes.byref(c)) == 0
        assert (c.shape, c.bt, c.bx, c.by, c.mode) == (0,) + want, L
    good = tmp_path / "tune.txt"
    good.write_text("# sal autotune cache v1: L precision size_class shape ms\n7 0 1 3 31.5\n5 0 0 1 0.25\n")
    assert lib.sal_autotune_load(str(good).encode()) == 0
    assert lib.sal_autotune_query(7, 0, 286_000_000, ctypes.byref(c)) == 0
    assert (c.shape, c.bt, c.bx, c.by, c.mode, c.size_class) == (3, 2, 8, 32, 3, 1) and abs(c.ms - 31.5) < 1e-5
    assert lib.sal_autotune_query(7, 0, 1000, ctypes.byref(c)) == 0 and c.shape == 0   # other size class
    saved = tmp_path / "saved.txt"
    assert lib.sal_autotune_save(str(saved).encode()) == 0
    lines = [ln for ln in saved.read_text().splitlines() if not ln.startswith("#")]
    assert sorted(ln.split()[:4] for ln in lines) == [["5", "0", "0", "1"], ["7", "0", "1", "3"]]
    for bad in ("# sal autotune cache v1\n7 0 1 9 1.0\n",            # shape index out of range
                "# sal autotune cache v1\n8 0 1 0 1.0\n",            # even L
                "# sal autotune cache v1\n7 0 1 0\n",                # short line
                "# sal autotune cache v1\n7 0 1 0 1.0 junk\n",       # trailing field
                "not a cache\n7 0 1 0 1.0\n"):                       # wrong header
        corrupt = tmp_path / "bad.txt"
        corrupt.write_text(bad)
        assert lib.sal_autotune_load(str(corrupt).encode()) == N.SAL_ERR_INVALID_ARG
        assert lib.sal_autotune_query(7, 0, 286_000_000, ctypes.byref(c)) == 0 and c.shape == 3   # unchanged
    assert lib.sal_autotune_load(str(tmp_path / "missing.txt").encode()) == N.SAL_ERR_INVALID_ARG
    assert lib.sal_autotune_clear() == 0
    assert lib.sal_autotune_query(7, 0, 286_000_000, ctypes.byref(c)) == 0 and c.shape == 0
