"""The fixed-scratch directional compare (sal_directional_compare_static).

Some callers cannot allocate device memory, for example a plug-in whose host application
owns the GPU's memory budget.  This entry point takes only the caller's inputs and
outputs; the reduction scratch is a fixed array inside the library.  Its results must be
those of the workspace-based call.  This file is collected last, so a run that stops at
the first failure has run every other test before it.
"""
import ctypes

import numpy as np
import pytest
import torch

from paper_1901_11095_gb300 import _native as N
from paper_1901_11095_gb300 import api, synth

pytestmark = pytest.mark.gpu

TOL_MAP = 2e-5


def _static_call(E, p, Sm, stats):
    dims = N.SalDims(*[int(s) for s in E.shape[1:]])
    st = N.lib().sal_directional_compare_static(ctypes.c_void_p(E.data_ptr()), dims, ctypes.byref(p),
                                                ctypes.c_void_p(Sm.data_ptr()), ctypes.c_void_p(stats.data_ptr()),
                                                ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
    N.check(st)


@pytest.mark.parametrize("shape,stencil,L", [((40, 37, 131), "26", 7), ((23, 64, 70), "line", 9)])
def test_static_matches_workspace_call_twice(shape, stencil, L):
    dev = torch.device("cuda:0")
    V = torch.from_numpy(synth.make_volume(shape, seed=21)).to(dev)
    p = api.params(L=L, stencil=stencil, sigma=1.2)
    E = api.sal_spectral_energy(V, p)
    Sm_ref, st_ref = api.sal_directional_compare(E, p)
    for _ in range(2):                       # two calls in a row share the fixed scratch
        Sm = torch.full_like(E, float("nan"))
        stats = torch.full((N.SAL_STATS_LEN,), float("nan"), dtype=torch.float64, device=dev)
        _static_call(E, p, Sm, stats)
        torch.cuda.synchronize()
        scale = float(Sm_ref.abs().max())
        assert float((Sm - Sm_ref).abs().max()) <= TOL_MAP * scale
        np.testing.assert_allclose(stats.cpu().numpy(), st_ref.cpu().numpy(), rtol=1e-12)


def test_static_calls_allocate_no_device_memory():
    """After the first call (which looks up the scratch address), further calls leave the
    device's free memory unchanged: neither the library nor the caller allocates."""
    dev = torch.device("cuda:0")
    V = torch.from_numpy(synth.make_volume((32, 40, 96), seed=22)).to(dev)
    p = api.params()
    E = api.sal_spectral_energy(V, p)
    Sm = torch.empty_like(E)
    stats = torch.empty(N.SAL_STATS_LEN, dtype=torch.float64, device=dev)
    _static_call(E, p, Sm, stats)
    torch.cuda.synchronize()
    free0, _ = torch.cuda.mem_get_info(dev)
    for _ in range(5):
        _static_call(E, p, Sm, stats)
    torch.cuda.synchronize()
    free1, _ = torch.cuda.mem_get_info(dev)
    assert free1 == free0


def test_static_rejects_volumes_beyond_the_fixed_scratch():
    dev = torch.device("cuda:0")
    p = api.params()
    E = torch.zeros((3, 1, 1, 1), device=dev)
    # ceil(T/8) * ceil(X/8) * ceil(Y/64) tiles: 8 * 8 * (64 * (max + 1)) needs max + 1 tiles
    dims = N.SalDims(8, 8, 64 * (N.SAL_DCS_STATIC_MAX_TILES + 1))
    st = N.lib().sal_directional_compare_static(ctypes.c_void_p(E.data_ptr()), dims, ctypes.byref(p),
                                                ctypes.c_void_p(E.data_ptr()), ctypes.c_void_p(E.data_ptr()), None)
    assert st == N.SAL_ERR_WORKSPACE
    assert "tiles" in N.lib().sal_last_error().decode()
