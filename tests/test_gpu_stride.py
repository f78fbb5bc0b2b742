"""Parity of the coarse-stride cubes (Sec. 2, first step: cubes sliding with more than 50 %
overlap) with the FP64 oracle, through the C ABI: the lattice energies, the interpolation back
to every voxel, and the whole method with a stride."""
import numpy as np
import pytest
import torch

import oracle as O
from paper_1901_11095_gb300 import api, synth

pytestmark = pytest.mark.gpu

DEV = "cuda:0"
TOL_MAP = 2e-5
TOL_S = 1e-4
BND = {"reflect": O.REFLECT, "periodic": O.PERIODIC}


def nerr(got, ref):
    got = np.asarray(got, dtype=np.float64)
    ref = np.asarray(ref, dtype=np.float64)
    scale = np.abs(ref).max()
    return float(np.abs(got - ref).max() / (scale if scale > 0 else 1.0))


def to_dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).to(DEV)


CASES = [
    # shape, L, stride, boundary, seed
    ((40, 37, 70), 7, 3, "reflect", 0),
    ((33, 45, 64), 7, 2, "periodic", 1),
    ((29, 31, 130), 5, 2, "reflect", 2),      # several lattice blocks along y, ragged
    ((17, 23, 41), 9, 4, "reflect", 3),
    ((20, 26, 27), 11, 5, "periodic", 4),
    ((16, 18, 20), 15, 7, "reflect", 5),      # the largest cube and stride: smaller lattice blocks
    ((1, 9, 12), 5, 2, "reflect", 6),         # one plane: a one-point lattice along t
    ((1, 1, 1), 7, 3, "reflect", 7),          # a single voxel
    ((12, 13, 260), 7, 3, "reflect", 8),      # rows longer than a CTA (y walked in two passes)
]


@pytest.mark.parametrize("shape,L,s,bnd,seed", CASES)
def test_lattice_energy_matches_oracle(shape, L, s, bnd, seed):
    V = synth.make_volume(shape, seed=seed)
    p = api.params(L=L, boundary=bnd, stride=s)
    Ec = api.sal_lattice_energy(to_dev(V), p).cpu().numpy()
    Ec_ref = O.energy_lattice(V, L, s, bnd=BND[bnd])
    assert Ec.shape == Ec_ref.shape
    for m in range(3):
        assert nerr(Ec[m], Ec_ref[m]) < TOL_MAP, (m, nerr(Ec[m], Ec_ref[m]))


@pytest.mark.parametrize("shape,s", [((40, 37, 70), 3), ((9, 300, 11), 2), ((1, 1, 1), 2), ((5, 1, 33), 4),
                                     ((2, 2, 2), 7), ((31, 2, 700), 5)])
def test_interpolation_matches_oracle(shape, s):
    rng = np.random.default_rng(s)
    lat = O.lattice_shape(shape, s)
    Ec = rng.uniform(0.0, 2.0, size=(3,) + lat).astype(np.float32)
    E = api.sal_interpolate_lattice(to_dev(Ec), shape, api.params(L=15, stride=s)).cpu().numpy()
    E_ref = O.interp_lattice(Ec.astype(np.float64), shape, s)
    assert np.abs(E - E_ref).max() <= 4e-7 * np.abs(E_ref).max()


@pytest.mark.parametrize("shape,L,s,bnd,seed", CASES)
def test_strided_saliency_matches_oracle(shape, L, s, bnd, seed):
    V = synth.make_volume(shape, seed=seed)
    p = api.params(L=L, boundary=bnd, stride=s)
    stats = torch.empty(9, dtype=torch.float64, device=DEV)
    S, _ = api.sal_saliency(to_dev(V), p, stats=stats)
    S_ref, E_ref, Sm_ref, st_ref = O.saliency_strided(V, L=L, s=s, bnd=BND[bnd], full=True)
    assert nerr(S.cpu().numpy(), S_ref) < TOL_S
    # the split calls compose to the same energies
    Ed = api.sal_interpolate_lattice(api.sal_lattice_energy(to_dev(V), p), shape, p)
    for m in range(3):
        assert nerr(Ed[m].cpu().numpy(), E_ref[m]) < TOL_MAP


def test_stride_one_lattice_is_every_voxel():
    V = to_dev(synth.make_volume((20, 21, 40), seed=9))
    p = api.params(L=7, stride=1)
    Ec = api.sal_lattice_energy(V, p)
    E = api.sal_spectral_energy(V, p)
    assert Ec.shape == E.shape
    assert float((Ec - E).abs().max()) <= 2e-5 * float(E.abs().max())


def test_stride_needs_the_calls_with_room_for_the_lattice():
    V = to_dev(synth.make_volume((16, 16, 32), seed=10))
    p = api.params(L=7, stride=2)
    with pytest.raises(api.N.SalError) as ei:
        api.sal_spectral_energy(V, p)
    assert ei.value.status == api.N.SAL_ERR_UNSUPPORTED
    with pytest.raises(api.N.SalError) as ei:
        api.sal_saliency(V, api.params(L=7, stride=2, precision="bf16"))
    assert ei.value.status == api.N.SAL_ERR_UNSUPPORTED


def test_strided_host_buffers_equal_device_call():
    V = synth.make_volume((70, 40, 66), seed=11)
    p = api.params(L=7, stride=3)
    S_dev, _ = api.sal_saliency(to_dev(V), p)
    Vh = torch.from_numpy(V).pin_memory()
    S_host = api.sal_saliency_host(Vh, p)
    torch.cuda.synchronize()
    assert torch.equal(S_host, S_dev.cpu())
