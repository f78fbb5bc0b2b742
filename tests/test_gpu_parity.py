"""Parity of the CUDA path (through the C ABI) with the FP64 CPU oracle, element by element.

Tolerance of the FP32 path: normwise relative max error 1e-4 on S (max |S - S_ref| /
max |S_ref|), and 2e-5 on each E_m and S_m map; both derived from FP32 arithmetic
(unit roundoff 6e-8) accumulated over O(L^3) terms.
"""
import numpy as np
import pytest
import torch

import oracle as O
from paper_1901_11095_gb300 import api, synth

pytestmark = pytest.mark.gpu

DEV = "cuda:0"
TOL_S = 1e-4
TOL_MAP = 2e-5


def nerr(got, ref):
    got = np.asarray(got, dtype=np.float64)
    ref = np.asarray(ref, dtype=np.float64)
    scale = np.abs(ref).max()
    return float(np.abs(got - ref).max() / (scale if scale > 0 else 1.0))


def to_dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).to(DEV)


BND = {"reflect": O.REFLECT, "periodic": O.PERIODIC}
STC = {"26": O.STENCIL_26, "line": O.STENCIL_LINE}

CASES = [
    # shape, L, boundary, stencil, sigma, seed
    ((64, 64, 64), 7, "reflect", "26", 1.0, 0),      # the small cube of the plain FP32 workload
    ((37, 45, 70), 5, "reflect", "26", 1.0, 1),      # ragged: no axis a tile multiple
    ((20, 17, 33), 9, "periodic", "line", 1.5, 2),
    ((13, 29, 31), 3, "reflect", "line", 0.8, 3),
    ((12, 21, 40), 11, "periodic", "26", 1.0, 4),
    ((14, 15, 36), 13, "reflect", "26", 2.0, 5),
    ((16, 18, 35), 15, "reflect", "line", 1.0, 6),
]


@pytest.mark.parametrize("shape,L,bnd,stc,sigma,seed", CASES)
def test_spectral_energy_matches_oracle(shape, L, bnd, stc, sigma, seed):
    V = synth.make_volume(shape, seed=seed)
    E = api.sal_spectral_energy(to_dev(V), api.params(L=L, boundary=bnd)).cpu().numpy()
    E_ref = O.energy(V, L, bnd=BND[bnd])
    for m in range(3):
        assert nerr(E[m], E_ref[m]) < TOL_MAP, (m, nerr(E[m], E_ref[m]))


@pytest.mark.parametrize("shape,L,bnd,stc,sigma,seed", CASES)
def test_saliency_matches_oracle(shape, L, bnd, stc, sigma, seed):
    V = synth.make_volume(shape, seed=seed)
    p = api.params(L=L, boundary=bnd, stencil=stc, sigma=sigma)
    stats = torch.empty(9, dtype=torch.float64, device=DEV)
    S, _ = api.sal_saliency(to_dev(V), p, stats=stats)
    S_ref, E_ref, Sm_ref, st_ref = O.saliency(V, L=L, bnd=BND[bnd], stencil=STC[stc], sigma=sigma, full=True)
    assert nerr(S.cpu().numpy(), S_ref) < TOL_S
    st = stats.cpu().numpy().reshape(3, 3)
    for m in range(3):      # normwise: min and max carry the error of their map, relative to its scale
        np.testing.assert_allclose(st[m, :2], st_ref[m, :2], rtol=0, atol=TOL_MAP * np.abs(Sm_ref[m]).max())
    np.testing.assert_allclose(st[:, 2], st_ref[:, 2], rtol=1e-4)


@pytest.mark.parametrize("shape", [(1, 1, 1), (2, 3, 1), (5, 1, 7), (1, 40, 1), (3, 3, 3)])
@pytest.mark.parametrize("bnd", ["reflect", "periodic"])
def test_degenerate_small_volumes(shape, bnd):
    V = synth.make_volume(shape, seed=9)
    p = api.params(L=5, boundary=bnd)
    E = api.sal_spectral_energy(to_dev(V), p).cpu().numpy()
    E_ref = O.energy(V, 5, bnd=BND[bnd])
    for m in range(3):
        assert np.abs(E[m] - E_ref[m]).max() <= TOL_MAP * max(np.abs(E_ref).max(), 1e-30)
    S, _ = api.sal_saliency(to_dev(V), p)
    S_ref = O.saliency(V, L=5, bnd=BND[bnd])
    assert np.abs(S.cpu().numpy() - S_ref).max() <= TOL_S * max(np.abs(S_ref).max(), 1.0)


@pytest.mark.parametrize("val", [0.0, 1.0, -3.75])
def test_constant_volume_is_exactly_zero(val):
    V = np.full((19, 23, 41), val, dtype=np.float32)
    Vd = to_dev(V)
    p = api.params(L=7)
    E = api.sal_spectral_energy(Vd, p)
    assert bool((E == 0).all())
    S, _ = api.sal_saliency(Vd, p)
    assert bool((S == 0).all())


@pytest.mark.parametrize("L,k", [(5, (1, 2, 0)), (7, (2, 0, 3)), (9, (4, 1, 2))])
def test_plane_wave_closed_form_on_gpu(L, k):
    shape = (2 * L, 2 * L, 4 * L)
    V = synth.plane_wave(shape, k, L)
    E = api.sal_spectral_energy(to_dev(V), api.params(L=L, boundary="periodic")).cpu().numpy()
    rho = np.sqrt(k[0] ** 2 + k[1] ** 2 + k[2] ** 2)
    n = L ** 3 - 1
    expect = [np.hypot(k[1], k[2]) / rho / n, np.hypot(k[0], k[2]) / rho / n, np.hypot(k[0], k[1]) / rho / n]
    for m in range(3):
        assert np.abs(E[m] - expect[m]).max() < 2e-7


@pytest.mark.parametrize("L,bnd", [(3, "reflect"), (7, "periodic"), (11, "reflect")])
def test_local_spectra_and_project_match_oracle(L, bnd):
    V = synth.make_volume((15, 14, 13), seed=12)
    p = api.params(L=L, boundary=bnd)
    lo, ext = (0, 10, 9), (3, 4, 4)      # touches the t = 0 and y = Y-1 faces
    mag = api.sal_local_spectra(to_dev(V), p, lo, ext).cpu().numpy()
    for a in range(ext[0]):
        for b in range(ext[1]):
            for c in range(ext[2]):
                ref = O.local_spectrum(V, lo[0] + a, lo[1] + b, lo[2] + c, L, BND[bnd])
                assert nerr(mag[a, b, c], ref) < TOL_MAP
    # projection of the same float32 spectra on both sides
    E = api.sal_project(to_dev(mag), L).cpu().numpy()
    E_ref = O.project(mag.astype(np.float64).reshape(-1, L, L, L), L)
    for m in range(3):
        assert nerr(E[m], E_ref[m]) < TOL_MAP


@pytest.mark.parametrize("stc,L,bnd,sigma,shape", [
    ("26", 7, "reflect", 1.0, (21, 19, 67)), ("line", 7, "periodic", 1.3, (21, 19, 67)),
    ("line", 15, "reflect", 2.0, (21, 19, 67)), ("26", 5, "periodic", 0.6, (21, 19, 67)),
    # several chunks of planes along t, the last one ragged; ragged x and y blocks
    ("26", 7, "reflect", 1.0, (150, 11, 70)), ("26", 5, "periodic", 0.8, (129, 9, 131)),
    # the line kernel is compiled once per half-width h = 1 .. 7: every one of them, on
    # ragged shapes (Y not a multiple of 4, so the stores take the per-column path)
    ("line", 3, "reflect", 0.9, (19, 10, 37)), ("line", 5, "reflect", 1.1, (18, 17, 66)),
    ("line", 9, "periodic", 1.5, (25, 12, 71)), ("line", 11, "reflect", 1.7, (23, 13, 65)),
    ("line", 13, "periodic", 1.9, (27, 16, 90)),
    # the line kernels over several chunks of 128 planes, the last one ragged
    ("line", 7, "reflect", 1.0, (150, 11, 70)), ("line", 13, "periodic", 1.9, (140, 9, 67)),
    ("line", 3, "periodic", 0.8, (257, 5, 41)),
])
def test_directional_compare_matches_oracle(stc, L, bnd, sigma, shape):
    rng = np.random.default_rng(5)
    E = rng.uniform(0.0, 1.0, size=(3,) + shape).astype(np.float32)
    p = api.params(L=L, boundary=bnd, stencil=stc, sigma=sigma)
    Sm, st = api.sal_directional_compare(to_dev(E), p)
    Sm_ref = O.dcs(E.astype(np.float64), bnd=BND[bnd], stencil=STC[stc], L=L, sigma=sigma)
    Smh = Sm.cpu().numpy()
    for m in range(3):
        assert nerr(Smh[m], Sm_ref[m]) < TOL_MAP
    st_ref = O.stats(Sm_ref)
    sth = st.cpu().numpy().reshape(3, 3)
    for m in range(3):
        np.testing.assert_allclose(sth[m, :2], st_ref[m, :2], rtol=0, atol=TOL_MAP * np.abs(Sm_ref[m]).max())
    np.testing.assert_allclose(sth[:, 2], st_ref[:, 2], rtol=1e-5)
    # the FP64 min / max reductions are exact on the maps the kernel wrote
    for m in range(3):
        assert sth[m, 0] == float(Sm[m].min()) and sth[m, 1] == float(Sm[m].max())


@pytest.mark.parametrize("a,b,c", [(1 / 3, 1 / 3, 1 / 3), (0.5, 0.3, 0.2), (1.0, 0.0, 0.0)])
def test_combine_matches_oracle(a, b, c):
    rng = np.random.default_rng(6)
    Sm = rng.uniform(0.2, 2.0, size=(3, 9, 10, 37)).astype(np.float32)
    Sm[2] = np.float32(0.75)                       # a constant map normalises to 0
    st_ref = O.stats(Sm.astype(np.float64))
    p = api.params(a=a, b=b, c=c)
    S = api.sal_combine(to_dev(Sm), to_dev(st_ref.reshape(9)), p).cpu().numpy()
    S_ref = O.combine(Sm.astype(np.float64), st_ref, a, b, c)
    assert np.abs(S - S_ref).max() < 2e-6


def test_repeat_calls_are_identical():
    V = to_dev(synth.make_volume((40, 33, 65), seed=7))
    p = api.params(L=7)
    a, _ = api.sal_saliency(V, p)
    b, _ = api.sal_saliency(V, p)
    assert torch.equal(a, b)


def test_stream_argument_is_used():
    V = to_dev(synth.make_volume((30, 30, 64), seed=8))
    p = api.params(L=5)
    s = torch.cuda.Stream()
    ref, _ = api.sal_saliency(V, p)
    with torch.cuda.stream(s):
        out, _ = api.sal_saliency(V, p, stream=s)
    s.synchronize()
    assert torch.equal(out, ref)
