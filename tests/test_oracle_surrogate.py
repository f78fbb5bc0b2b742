"""Pins of the FP64 reference of the surrogate's layers: convolution against scipy's
correlate (a library special case), GELU against the normal CDF, gradients by the adjoint
identity and by central finite differences."""
import numpy as np
import pytest
from scipy import ndimage, special

import oracle as O


def test_conv3d_matches_scipy_correlate():
    rng = np.random.default_rng(0)
    x = rng.standard_normal((2, 6, 5, 7))
    w = rng.standard_normal((3, 2, 3, 3, 3))
    b = rng.standard_normal(3)
    got = O.conv3d(x, w, b)
    for co in range(3):
        ref = b[co] + sum(ndimage.correlate(x[ci], w[co, ci], mode="mirror") for ci in range(2))
        np.testing.assert_allclose(got[co], ref, rtol=1e-12, atol=1e-12)
    got = O.conv3d(x, w, b, bnd=O.PERIODIC)
    for co in range(3):
        ref = b[co] + sum(ndimage.correlate(x[ci], w[co, ci], mode="wrap") for ci in range(2))
        np.testing.assert_allclose(got[co], ref, rtol=1e-12, atol=1e-12)


def test_gelu_against_normal_cdf():
    x = np.linspace(-6, 6, 97)
    np.testing.assert_allclose(O.gelu(x), x * special.ndtr(x), rtol=1e-13, atol=1e-15)
    h = 1e-5
    num = (x + h) * special.ndtr(x + h) - (x - h) * special.ndtr(x - h)
    np.testing.assert_allclose(O.gelu_grad(x), num / (2 * h), rtol=1e-7, atol=1e-9)


def test_conv_gradients_adjoint_identities():
    rng = np.random.default_rng(1)
    x = rng.standard_normal((3, 5, 4, 6))
    w = rng.standard_normal((2, 3, 3, 3, 3))
    g = rng.standard_normal((2, 5, 4, 6))
    gw, gb, gx = O.conv3d_grad(x, w, g)
    y = O.conv3d(x, w)
    # <conv(x), g> is linear in x and in w: its derivatives are the input and weight gradients
    assert np.isclose(np.sum(y * g), np.sum(x * gx), rtol=1e-12)
    assert np.isclose(np.sum(y * g), np.sum(w * gw), rtol=1e-12)
    np.testing.assert_allclose(gb, g.sum(axis=(1, 2, 3)), rtol=1e-13)


def _params(widths, rng):
    out = []
    for l in range(len(widths) - 1):
        out.append(rng.standard_normal(widths[l + 1] * widths[l] * 27) * 0.3)
        out.append(rng.standard_normal(widths[l + 1]) * 0.1)
    return np.concatenate(out)


def test_surrogate_gradient_by_finite_differences():
    rng = np.random.default_rng(2)
    widths = [1, 2, 2, 3]
    x = rng.standard_normal((1, 4, 3, 5))
    target = rng.standard_normal((3, 4, 3, 5))
    mask = (rng.uniform(size=(4, 3, 5)) > 0.3).astype(np.float64)
    params = _params(widths, rng)
    loss, grads = O.surrogate_loss_grad(x, widths, params, target, mask)
    out = O.surrogate_forward(x, widths, params)
    assert np.isclose(loss, 0.5 * np.sum(mask * (out - target) ** 2), rtol=1e-13)
    h = 1e-6
    for i in rng.choice(params.size, 40, replace=False):
        pp, pm = params.copy(), params.copy()
        pp[i] += h
        pm[i] -= h
        lp = 0.5 * np.sum(mask * (O.surrogate_forward(x, widths, pp) - target) ** 2)
        lm = 0.5 * np.sum(mask * (O.surrogate_forward(x, widths, pm) - target) ** 2)
        assert np.isclose(grads[i], (lp - lm) / (2 * h), rtol=1e-5, atol=1e-7), i
