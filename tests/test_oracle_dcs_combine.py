"""Pins of the oracle's directional centre-surround (Eq. 5), normalisation and Eq. 6,
and whole-method invariants: constant volume, shift equivariance, axis swap, scale."""
import itertools
import math

import numpy as np
import pytest

import oracle as O
from paper_1901_11095_gb300 import synth


def _offsets(stencil, m, L):
    if stencil == O.STENCIL_26:
        return [o for o in itertools.product((-1, 0, 1), repeat=3) if o != (0, 0, 0)]
    h = (L - 1) // 2
    out = []
    for k in range(-h, h + 1):
        if k:
            o = [0, 0, 0]
            o[m] = k
            out.append(tuple(o))
    return out


@pytest.mark.parametrize("stencil,L", [(O.STENCIL_26, 7), (O.STENCIL_LINE, 5), (O.STENCIL_LINE, 9)])
@pytest.mark.parametrize("sigma", [0.7, 1.0, 2.5])
def test_dcs_constant_field_closed_form(stencil, L, sigma):
    # E == e everywhere: S_m = e * Q^-1 sum_o (1 - g(o))
    e = np.array([0.3, 1.7, 2.0])
    E = np.ones((3, 9, 8, 10)) * e[:, None, None, None]
    S = O.dcs(E, stencil=stencil, L=L, sigma=sigma)
    for m in range(3):
        offs = _offsets(stencil, m, L)
        expect = e[m] * sum(1 - math.exp(-sum(c * c for c in o) / (2 * sigma * sigma)) for o in offs) / len(offs)
        np.testing.assert_allclose(S[m], expect, rtol=1e-13)


@pytest.mark.parametrize("stencil,L", [(O.STENCIL_26, 7), (O.STENCIL_LINE, 7)])
def test_dcs_spike_closed_form(stencil, L):
    # one spike of height A on zeros: at the spike S = A; at a neighbour v = s - o, S = g(o) A / Q
    sigma, A = 1.3, 2.0
    shape = (11, 12, 13)
    s = (5, 6, 7)
    E = np.zeros((3,) + shape)
    E[:, s[0], s[1], s[2]] = A
    S = O.dcs(E, stencil=stencil, L=L, sigma=sigma, bnd=O.PERIODIC)
    for m in range(3):
        offs = _offsets(stencil, m, L)
        Q = len(offs)
        assert np.isclose(S[m][s], A, rtol=1e-14)
        expect = np.zeros(shape)
        expect[s] = A
        for o in offs:
            v = tuple(s[i] - o[i] for i in range(3))
            expect[v] += math.exp(-sum(c * c for c in o) / (2 * sigma * sigma)) * A / Q
        np.testing.assert_allclose(S[m], expect, rtol=1e-13, atol=1e-300)


def test_dcs_reflect_boundary_closed_form():
    # spike at t = 1 seen from t = 0 through both the t-1 (reflected onto t=1) and t+1 neighbours
    sigma, A = 1.0, 1.0
    E = np.zeros((3, 6, 5, 5))
    E[:, 1, 2, 2] = A
    S = O.dcs(E, stencil=O.STENCIL_26, sigma=sigma, bnd=O.REFLECT)
    g1 = math.exp(-1 / (2 * sigma ** 2))
    assert np.isclose(S[0, 0, 2, 2], 2 * g1 * A / 26, rtol=1e-14)
    S = O.dcs(E, stencil=O.STENCIL_LINE, L=5, sigma=sigma, bnd=O.REFLECT)
    # line along t, offsets -2..2: from t=0, t-1 -> 1 (spike), t+1 = 1 (spike), t-2 -> 2, t+2 = 2
    assert np.isclose(S[0, 0, 2, 2], 2 * g1 * A / 4, rtol=1e-14)
    # the x and y line maps do not see the spike from (0, 2, 2)
    assert S[1, 0, 2, 2] == 0.0 and S[2, 0, 2, 2] == 0.0


def test_stats_and_combine():
    rng = np.random.default_rng(0)
    Sm = rng.uniform(0.5, 3.0, size=(3, 4, 5, 6))
    Sm[2] = 1.25                                   # a constant map normalises to 0
    st = O.stats(Sm)
    for m in range(3):
        assert st[m, 0] == Sm[m].min() and st[m, 1] == Sm[m].max()
        assert np.isclose(st[m, 2], math.fsum(Sm[m].ravel()), rtol=1e-14)
    a, b, c = 0.5, 0.3, 0.2
    S = O.combine(Sm, st, a, b, c)
    n0 = (Sm[0] - Sm[0].min()) / (Sm[0].max() - Sm[0].min())
    n1 = (Sm[1] - Sm[1].min()) / (Sm[1].max() - Sm[1].min())
    np.testing.assert_allclose(S, a * n0 + b * n1, rtol=1e-13, atol=1e-15)


def test_constant_volume_gives_zero_saliency():
    for val in (0.0, 1.0, -3.75):
        V = np.full((9, 10, 11), val, dtype=np.float32)
        S, E, Sm, st = O.saliency(V, L=5, full=True)
        assert (E == 0).all() and (Sm == 0).all() and (S == 0).all()


@pytest.mark.parametrize("stencil", [O.STENCIL_26, O.STENCIL_LINE])
def test_shift_equivariance_periodic(stencil):
    V = synth.make_volume((12, 10, 14), seed=8)
    S = O.saliency(V, L=5, bnd=O.PERIODIC, stencil=stencil)
    k = (3, -4, 5)
    S2 = O.saliency(np.roll(V, k, axis=(0, 1, 2)), L=5, bnd=O.PERIODIC, stencil=stencil)
    np.testing.assert_allclose(S2, np.roll(S, k, axis=(0, 1, 2)), rtol=0, atol=1e-12)


def test_axis_swap_symmetry():
    V = synth.make_volume((10, 12, 12), seed=9)
    Vs = np.ascontiguousarray(np.transpose(V, (0, 2, 1)))
    S, E, _, _ = O.saliency(V, L=5, full=True)
    S2, E2, _, _ = O.saliency(Vs, L=5, full=True)
    np.testing.assert_allclose(E2[1], np.transpose(E[2], (0, 2, 1)), rtol=1e-12)
    np.testing.assert_allclose(E2[2], np.transpose(E[1], (0, 2, 1)), rtol=1e-12)
    np.testing.assert_allclose(E2[0], np.transpose(E[0], (0, 2, 1)), rtol=1e-12)
    np.testing.assert_allclose(S2, np.transpose(S, (0, 2, 1)), atol=1e-12)


def test_scale_and_sign_invariance():
    V = synth.make_volume((10, 9, 11), seed=10)
    S = O.saliency(V, L=5)
    for alpha in (-2.0, 0.125, 8.0):          # powers of two and a sign flip: V * alpha is exact in float32
        S2 = O.saliency((V * np.float32(alpha)).astype(np.float32), L=5)
        np.testing.assert_allclose(S2, S, atol=1e-12)
    # any other factor rounds V once in float32 (relative 6e-8), which S inherits
    S3 = O.saliency((V * np.float32(-2.5)).astype(np.float32), L=5)
    np.testing.assert_allclose(S3, S, atol=1e-5)


def test_saliency_range():
    V = synth.make_volume((16, 16, 16), seed=1)
    S = O.saliency(V, L=7)
    assert S.min() >= 0 and S.max() <= 1 + 1e-12
