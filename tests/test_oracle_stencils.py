"""Pins of the oracle's tunable directional comparisons (Eq. 5 with the neighbourhood of
Fig. 3 and the text after Eq. 5): the d x 1 line along the t-x diagonal and caller-given
offsets with explicit weights.  Closed forms (constant field, spike, linear ramp) fix the
direction, the sign and the axis order of every offset."""
import math

import numpy as np
import pytest

import oracle as O


def _diag_offsets(L):
    h = (L - 1) // 2
    return [(k, k, 0) for k in range(-h, h + 1) if k]


@pytest.mark.parametrize("L,sigma", [(5, 1.0), (7, 0.8), (9, 2.0)])
def test_diag_constant_field_closed_form(L, sigma):
    # E == e: S_m = e * Q^-1 sum_k (1 - exp(-2 k^2 / (2 sigma^2))), Q = L - 1, the same for every map
    e = np.array([0.4, 1.1, 3.0])
    E = np.ones((3, 10, 9, 8)) * e[:, None, None, None]
    S = O.dcs(E, stencil=O.STENCIL_DIAG_TX, L=L, sigma=sigma)
    h = (L - 1) // 2
    gsum = sum(1 - math.exp(-2 * k * k / (2 * sigma * sigma)) for k in range(1, h + 1))
    for m in range(3):
        np.testing.assert_allclose(S[m], e[m] * 2 * gsum / (L - 1), rtol=1e-13)


def test_diag_spike_lies_on_the_t_x_diagonal():
    # spike of height A at s on zeros (periodic): S = A at s, g(o) A / Q at s - o for o = (k, k, 0),
    # zero everywhere else (in particular on the t-y diagonal and the t axis)
    L, sigma, A = 7, 1.4, 2.5
    shape = (15, 14, 13)
    s = (7, 6, 5)
    E = np.zeros((3,) + shape)
    E[:, s[0], s[1], s[2]] = A
    S = O.dcs(E, stencil=O.STENCIL_DIAG_TX, L=L, sigma=sigma, bnd=O.PERIODIC)
    expect = np.zeros(shape)
    expect[s] = A
    for o in _diag_offsets(L):
        expect[s[0] - o[0], s[1] - o[1], s[2] - o[2]] += math.exp(-(o[0] ** 2 + o[1] ** 2) / (2 * sigma ** 2)) * A / (L - 1)
    for m in range(3):
        np.testing.assert_allclose(S[m], expect, rtol=1e-13, atol=1e-300)


def test_diag_linear_ramp_sees_t_plus_x_only():
    # E = alpha t + beta x + gamma y with unit weights (user stencil of the diagonal offsets):
    # at an interior voxel |E(v) - E(v + (k, k, 0))| = |alpha + beta| |k|, whatever gamma is
    L = 7
    alpha, beta, gamma = 0.3, -1.1, 5.0
    T, X, Y = 12, 11, 10
    t, x, y = np.meshgrid(np.arange(T), np.arange(X), np.arange(Y), indexing="ij")
    E = np.stack([alpha * t + beta * x + gamma * y] * 3).astype(np.float64)
    offs = _diag_offsets(L)
    S = O.dcs_user(E, [offs] * 3, [[1.0] * len(offs)] * 3)
    h = 3
    expect = abs(alpha + beta) * 2 * sum(range(1, h + 1)) / (L - 1)
    inner = S[:, h:T - h, h:X - h, :]
    np.testing.assert_allclose(inner, expect, rtol=1e-12)


def test_user_stencil_single_asymmetric_offset():
    # one offset o = (1, -2, 3) with weight w on map t, (0, 0, -1) on map x, (2, 0, 0) on map y:
    # a spike of height A at s gives S = A at s (|A - w * 0|) and |w| A at s - o (|0 - w A|)
    A, w = 1.5, -0.7
    shape = (9, 10, 11)
    s = (4, 5, 6)
    offs = [[(1, -2, 3)], [(0, 0, -1)], [(2, 0, 0)]]
    E = np.zeros((3,) + shape)
    E[:, s[0], s[1], s[2]] = A
    S = O.dcs_user(E, offs, [[w]] * 3, bnd=O.PERIODIC)
    for m in range(3):
        o = offs[m][0]
        expect = np.zeros(shape)
        expect[s] = A
        expect[(s[0] - o[0]) % shape[0], (s[1] - o[1]) % shape[1], (s[2] - o[2]) % shape[2]] = abs(w) * A
        np.testing.assert_allclose(S[m], expect, rtol=1e-14, atol=0)


def test_user_stencil_reflect_boundary():
    # at t = 0 the offset (-1, 0, 0) reads t = 1 (whole-sample reflection), (-2, 0, 0) reads t = 2
    E = np.zeros((3, 6, 4, 5))
    E[:, 1] = 2.0
    E[:, 2] = 7.0
    S = O.dcs_user(E, [[(-1, 0, 0)], [(-2, 0, 0)], [(-1, 0, 0), (-2, 0, 0)]], [[1.0], [1.0], [1.0, 0.5]])
    np.testing.assert_allclose(S[0, 0], 2.0, rtol=0)
    np.testing.assert_allclose(S[1, 0], 7.0, rtol=0)
    np.testing.assert_allclose(S[2, 0], (2.0 + 3.5) / 2, rtol=1e-15)


def test_maps_at_diag_matches_whole_volume():
    from paper_1901_11095_gb300 import synth
    V = synth.make_volume((14, 13, 12), seed=4)
    L = 5
    _, E, Sm, _ = O.saliency(V, L=L, stencil=O.STENCIL_DIAG_TX, sigma=1.2, full=True)
    rng = np.random.default_rng(1)
    c = np.stack([rng.integers(0, s, 40) for s in V.shape], axis=1)
    c = np.concatenate([c, [[0, 0, 0], [13, 12, 11], [0, 12, 5]]])
    Ea, Sa = O.maps_at(V, c, L, stencil=O.STENCIL_DIAG_TX, sigma=1.2)
    np.testing.assert_allclose(Ea, E[:, c[:, 0], c[:, 1], c[:, 2]], rtol=1e-12, atol=1e-15)
    np.testing.assert_allclose(Sa, Sm[:, c[:, 0], c[:, 1], c[:, 2]], rtol=1e-12, atol=1e-15)
