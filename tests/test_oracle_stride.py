"""Pins of the oracle's coarse-stride cubes (Sec. 2, first step: the local cube slides with
more than 50 % overlap): the lattice of cube centres, the trilinear interpolation back to
every voxel (exact on trilinear fields, equal to scipy's regular-grid interpolation), and the
reduction to the stride-1 method."""
import numpy as np
import pytest
from scipy.interpolate import RegularGridInterpolator

import oracle as O
from paper_1901_11095_gb300 import synth


def _lattice(n, s):
    return [min(i * s, n - 1) for i in range(O.lattice_size(n, s))]


@pytest.mark.parametrize("n,s", [(1, 2), (2, 2), (7, 3), (8, 3), (9, 3), (10, 3), (64, 2), (65, 2), (17, 7)])
def test_lattice_covers_both_ends_with_step_s(n, s):
    c = _lattice(n, s)
    assert c[0] == 0 and c[-1] == n - 1
    assert len(c) == len(set(c))
    steps = np.diff(c)
    assert (steps[:-1] == s).all() if len(steps) > 1 else True
    assert all(1 <= d <= s for d in steps)


def test_interpolation_is_exact_on_trilinear_fields():
    # f = (a + b t)(c + d x)(e + g y) is trilinear: interpolation from any lattice reproduces it
    T, X, Y, s = 11, 9, 14, 3
    t, x, y = (np.arange(n, dtype=np.float64) for n in (T, X, Y))
    f = lambda tt, xx, yy: (0.5 + 1.5 * tt) * (2.0 - 0.25 * xx) * (-1.0 + 0.75 * yy)
    lt, lx, ly = (np.array(_lattice(n, s), dtype=np.float64) for n in (T, X, Y))
    Ec = np.stack([f(*np.meshgrid(lt, lx, ly, indexing="ij")), 3.0 + 0 * f(*np.meshgrid(lt, lx, ly, indexing="ij"))])
    out = O.interp_lattice(Ec, (T, X, Y), s)
    np.testing.assert_allclose(out[0], f(*np.meshgrid(t, x, y, indexing="ij")), rtol=1e-12, atol=1e-12)
    np.testing.assert_allclose(out[1], 3.0, rtol=1e-14)


def test_interpolation_equals_scipy_regular_grid():
    rng = np.random.default_rng(0)
    T, X, Y, s = 13, 10, 17, 4
    grids = [np.array(_lattice(n, s), dtype=np.float64) for n in (T, X, Y)]
    Ec = rng.standard_normal((2,) + tuple(len(g) for g in grids))
    out = O.interp_lattice(Ec, (T, X, Y), s)
    pts = np.stack(np.meshgrid(*(np.arange(n) for n in (T, X, Y)), indexing="ij"), axis=-1).reshape(-1, 3)
    for m in range(2):
        ref = RegularGridInterpolator(grids, Ec[m], method="linear")(pts).reshape(T, X, Y)
        np.testing.assert_allclose(out[m], ref, rtol=1e-12, atol=1e-12)


def test_lattice_energies_are_the_cubes_at_the_centres():
    V = synth.make_volume((12, 11, 15), seed=3)
    L, s = 5, 2
    Ec = O.energy_lattice(V, L, s)
    E = O.energy(V, L)
    lt, lx, ly = (_lattice(n, s) for n in V.shape)
    np.testing.assert_allclose(Ec, E[:, lt][:, :, lx][:, :, :, ly], rtol=1e-12, atol=1e-15)
    # and the interpolated field passes through them
    Es = O.energy_strided(V, L, s)
    np.testing.assert_allclose(Es[:, lt][:, :, lx][:, :, :, ly], Ec, rtol=1e-12, atol=1e-15)


def test_stride_one_is_the_plain_method():
    V = synth.make_volume((10, 12, 9), seed=4)
    np.testing.assert_allclose(O.energy_strided(V, 5, 1), O.energy(V, 5), rtol=0, atol=0)
    np.testing.assert_allclose(O.saliency_strided(V, L=5, s=1), O.saliency(V, L=5), rtol=0, atol=0)


def test_strided_constant_volume_gives_zero_and_plane_wave_energies_are_exact():
    V = np.full((9, 10, 11), 2.5, dtype=np.float32)
    S, E, Sm, _ = O.saliency_strided(V, L=5, s=2, full=True)
    assert (E == 0).all() and (S == 0).all()
    # a periodic plane wave along t has the same E at every cube: interpolation keeps it exact
    L, mu0 = 5, 1
    T = 3 * L
    t = np.arange(T)
    V = np.broadcast_to(np.cos(2 * np.pi * mu0 * t / L)[:, None, None], (T, 8, 9)).astype(np.float32)
    E = O.energy_strided(np.ascontiguousarray(V), L, 2, bnd=O.PERIODIC)
    np.testing.assert_allclose(E[0], 0.0, atol=1e-9)
    np.testing.assert_allclose(E[1], 1.0 / (L ** 3 - 1), rtol=1e-6)     # V holds float32-rounded cosines
    np.testing.assert_allclose(E[2], 1.0 / (L ** 3 - 1), rtol=1e-6)
