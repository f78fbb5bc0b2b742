"""Slabs along t through the C ABI on one GPU: every slab run in turn with its halo of V,
the statistics of all slabs merged by the library, each slab combined; the stitched S must
equal the whole-volume call bit for bit (each value is computed from the same samples in the
same order) and the FP64 oracle within the FP32 tolerance."""
import numpy as np
import pytest
import torch

import oracle as O
from paper_1901_11095_gb300 import api, shard, synth

pytestmark = pytest.mark.gpu

DEV = "cuda:0"
TOL_S = 1e-4


def _stitched(V, p, parts):
    dims = api.SalDims(*V.shape)
    H = api.sal_slab_halo(p)
    slabs = shard.slab_partition(V.shape[0], parts, H)
    Sms, sts = [], []
    for sl in slabs:
        Sm, st = api.sal_slab_maps(V[sl.ext_lo:sl.ext_hi].clone(), dims, sl.ext_lo, sl.ext_hi, sl.own_lo,
                                   sl.own_hi, p)
        Sms.append(Sm)
        sts.append(st)
    merged = api.sal_stats_merge(torch.stack(sts))
    S = torch.cat([api.sal_combine(Sm, merged, p) for Sm in Sms])
    Sm_all = torch.cat(Sms, dim=1)
    return S, Sm_all, merged


@pytest.mark.parametrize("shape,L,stc,parts", [((64, 40, 70), 7, "26", 3), ((50, 21, 64), 5, "line", 4),
                                               ((45, 19, 33), 9, "diag_tx", 2), ((130, 12, 64), 7, "26", 2),
                                               ((31, 17, 36), 3, "26", 8),
                                               # slabs of several chunks of 128 planes for the streamed stencils
                                               ((300, 10, 40), 7, "line", 2), ((270, 9, 35), 5, "diag_tx", 3)])
def test_slabs_equal_the_whole_volume(shape, L, stc, parts):
    V = torch.from_numpy(synth.make_volume(shape, seed=13)).to(DEV)
    p = api.params(L=L, stencil=stc)
    S, Sm, merged = _stitched(V, p, parts)
    st_ref = torch.empty(9, dtype=torch.float64, device=DEV)
    S_ref, _ = api.sal_saliency(V, p, stats=st_ref)
    E = api.sal_spectral_energy(V, p)
    Sm_ref, _ = api.sal_directional_compare(E, p)
    assert torch.equal(Sm, Sm_ref)
    assert torch.equal(S, S_ref)
    m, r = merged.cpu().numpy().reshape(3, 3), st_ref.cpu().numpy().reshape(3, 3)
    np.testing.assert_array_equal(m[:, :2], r[:, :2])
    np.testing.assert_allclose(m[:, 2], r[:, 2], rtol=1e-6)     # FP32 partial sums per warp, grouped by tile


def test_slabs_match_the_oracle():
    Vn = synth.make_volume((40, 24, 40), seed=14)
    p = api.params(L=7)
    S, _, _ = _stitched(torch.from_numpy(Vn).to(DEV), p, 3)
    S_ref = O.saliency(Vn, L=7)
    assert float(np.abs(S.cpu().numpy() - S_ref).max() / np.abs(S_ref).max()) < TOL_S


def test_slab_argument_checks():
    V = torch.zeros((20, 8, 8), device=DEV)
    dims = api.SalDims(20, 8, 8)
    p = api.params(L=5)
    H = api.sal_slab_halo(p)
    assert H == 3
    with pytest.raises(api.N.SalError) as ei:     # halo one plane short
        api.sal_slab_maps(V[3:13].clone(), dims, 3, 13, 5, 10, p)
    assert ei.value.status == api.N.SAL_ERR_INVALID_ARG
    with pytest.raises(api.N.SalError) as ei:     # a periodic volume cannot be cut along t
        api.sal_slab_maps(V[2:13].clone(), dims, 2, 13, 5, 10, api.params(L=5, boundary="periodic"))
    assert ei.value.status == api.N.SAL_ERR_UNSUPPORTED
