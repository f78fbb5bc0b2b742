"""Pins of the FP64 oracle's local spectrum, weights and energies (Sec. 2, Eq. 1-4).

Each check ties the oracle to something other than itself: numpy's FFT and numpy.pad
(library special cases), brute force, Parseval, conjugate symmetry and closed forms.
"""
import os

import numpy as np
import pytest

import oracle as O
from paper_1901_11095_gb300 import synth

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


@pytest.mark.parametrize("n", [1, 2, 3, 5, 8])
@pytest.mark.parametrize("bnd,mode", [(O.REFLECT, "reflect"), (O.PERIODIC, "wrap")])
def test_ext_index_matches_numpy_pad(n, bnd, mode):
    base = np.arange(n)
    pad = 3 * n + 4
    if n == 1 and mode == "reflect":
        ref = np.zeros(2 * pad + 1, dtype=int)          # a single sample reflects onto itself
    else:
        ref = np.pad(base, pad, mode=mode)
    got = np.array([O.ext_index(i, n, bnd) for i in range(-pad, n + pad)])
    np.testing.assert_array_equal(got, ref)


def _cube(V, t, x, y, L, mode):
    h = (L - 1) // 2
    P = np.pad(V.astype(np.float64), h, mode=mode)
    return P[t:t + L, x:x + L, y:y + L]


@pytest.mark.parametrize("L", [3, 5, 7])
@pytest.mark.parametrize("bnd,mode", [(O.REFLECT, "reflect"), (O.PERIODIC, "wrap")])
def test_spectrum_matches_numpy_fftn(L, bnd, mode):
    V = synth.make_volume((11, 9, 10), seed=3)
    rng = np.random.default_rng(0)
    pts = [(0, 0, 0), (10, 8, 9), (5, 4, 5)] + [tuple(int(v) for v in rng.integers(0, s)) for s in [(11, 9, 10)] * 3]
    for (t, x, y) in pts:
        got = O.local_spectrum(V, t, x, y, L, bnd)
        ref = np.abs(np.fft.fftshift(np.fft.fftn(_cube(V, t, x, y, L, mode)))) / L ** 3
        np.testing.assert_allclose(got, ref, rtol=0, atol=1e-14)


@pytest.mark.parametrize("L", [3, 5])
def test_brute_equals_separable(L):
    V = synth.make_volume((7, 6, 8), seed=5)
    for (t, x, y) in [(0, 0, 0), (3, 2, 4), (6, 5, 7)]:
        for bnd in (O.REFLECT, O.PERIODIC):
            a = O.local_spectrum(V, t, x, y, L, bnd, brute=True)
            b = O.local_spectrum(V, t, x, y, L, bnd, brute=False)
            np.testing.assert_allclose(a, b, rtol=0, atol=1e-14)


@pytest.mark.parametrize("L", [3, 5, 7, 9])
def test_parseval_and_conjugate_symmetry(L):
    V = synth.make_volume((12, 12, 12), seed=7)
    for (t, x, y) in [(1, 2, 3), (11, 0, 6)]:
        mag = O.local_spectrum(V, t, x, y, L)
        f = _cube(V, t, x, y, L, "reflect")
        # Parseval for F = L^-3 DFT(f): sum |F|^2 = L^-3 sum f^2
        assert np.isclose((mag ** 2).sum(), (f ** 2).sum() / L ** 3, rtol=1e-12)
        # real input: |F(-k)| = |F(k)|
        np.testing.assert_allclose(mag, mag[::-1, ::-1, ::-1], rtol=0, atol=1e-15)


@pytest.mark.parametrize("L", [3, 5, 7, 11])
def test_weight_identities(L):
    w = O.weights(L)
    h = (L - 1) // 2
    ssum = (w ** 2).sum(axis=0)
    dc = np.zeros((L, L, L), dtype=bool)
    dc[h, h, h] = True
    # w_t^2 + w_x^2 + w_y^2 = ((nu^2+omega^2) + (mu^2+omega^2) + (mu^2+nu^2)) / rho^2 = 2
    np.testing.assert_allclose(ssum[~dc], 2.0, rtol=1e-14)
    assert (w[:, h, h, h] == 0).all()
    assert (w >= 0).all() and (w <= 1 + 1e-15).all()
    # on the f_t axis the t-projection vanishes and the other two are 1 (Fig. 2 geometry)
    for k in range(1, h + 1):
        np.testing.assert_allclose(w[:, h + k, h, h], [0, 1, 1], atol=1e-15)
        np.testing.assert_allclose(w[:, h, h - k, h], [1, 0, 1], atol=1e-15)
        np.testing.assert_allclose(w[:, h, h, h + k], [1, 1, 0], atol=1e-15)
    # symmetric under the sign of each index, and w_t <-> w_x when mu <-> nu
    np.testing.assert_allclose(w, w[:, ::-1, :, :], atol=0)
    np.testing.assert_allclose(w, w[:, :, ::-1, :], atol=0)
    np.testing.assert_allclose(w[0], np.transpose(w[1], (1, 0, 2)), atol=1e-15)


def _golden_rows():
    rows = []
    with open(os.path.join(GOLDEN, "plane_wave_energies.txt")) as fh:
        for line in fh:
            if line.strip() and not line.startswith("#"):
                v = line.split()
                rows.append((int(v[0]), (int(v[1]), int(v[2]), int(v[3])), [float(s) for s in v[4:7]]))
    return rows


@pytest.mark.parametrize("L,k,expect", _golden_rows())
def test_plane_wave_energy_closed_form(L, k, expect):
    shape = (2 * L, 2 * L, L)
    V = synth.plane_wave(shape, k, L)
    E = O.energy(V, L, bnd=O.PERIODIC)
    for m in range(3):
        np.testing.assert_allclose(E[m], expect[m], rtol=0, atol=2e-8)


def test_energy_matches_fftn_on_padded_volume():
    L = 5
    V = synth.make_volume((9, 8, 7), seed=11)
    E = O.energy(V, L)
    w = O.weights(L)
    P = np.pad(V.astype(np.float64), 2, mode="reflect")
    for (t, x, y) in [(0, 0, 0), (4, 3, 2), (8, 7, 6), (2, 7, 0)]:
        mag = np.abs(np.fft.fftshift(np.fft.fftn(P[t:t + L, x:x + L, y:y + L]))) / L ** 3
        mag[2, 2, 2] = 0.0
        for m in range(3):
            assert np.isclose(E[m, t, x, y], (w[m] * mag).sum() / (L ** 3 - 1), rtol=1e-12)


def test_project_and_energy_at_agree_with_energy():
    L = 5
    V = synth.make_volume((8, 9, 10), seed=2)
    E = O.energy(V, L)
    coords = [(0, 0, 0), (7, 8, 9), (3, 4, 5), (1, 8, 0)]
    Ea = O.energy_at(V, coords, L)
    mags = np.stack([O.local_spectrum(V, *c, L) for c in coords])
    Ep = O.project(mags, L)
    for i, c in enumerate(coords):
        np.testing.assert_allclose(Ea[:, i], E[(slice(None),) + c], rtol=1e-14)
        np.testing.assert_allclose(Ep[:, i], E[(slice(None),) + c], rtol=1e-14)


def test_brute_energy_equals_separable_energy():
    V = synth.make_volume((6, 5, 7), seed=4)
    a = O.energy(V, 3, brute=True)
    b = O.energy(V, 3, brute=False)
    np.testing.assert_allclose(a, b, rtol=1e-12, atol=1e-15)


@pytest.mark.parametrize("stencil,L,bnd", [(O.STENCIL_26, 5, O.REFLECT), (O.STENCIL_LINE, 7, O.PERIODIC),
                                          (O.STENCIL_26, 3, O.PERIODIC)])
def test_maps_at_agrees_with_whole_volume(stencil, L, bnd):
    V = synth.make_volume((9, 11, 10), seed=6)
    S, E, Sm, _ = O.saliency(V, L=L, bnd=bnd, stencil=stencil, sigma=1.4, full=True)
    coords = [(0, 0, 0), (8, 10, 9), (4, 5, 5), (0, 10, 3), (8, 0, 9)]
    Ea, Sa = O.maps_at(V, coords, L, bnd=bnd, stencil=stencil, sigma=1.4)
    for i, c in enumerate(coords):
        np.testing.assert_allclose(Ea[:, i], E[(slice(None),) + c], rtol=1e-13)
        np.testing.assert_allclose(Sa[:, i], Sm[(slice(None),) + c], rtol=1e-12, atol=1e-16)
