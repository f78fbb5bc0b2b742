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


def _compose_forward(x, widths, params, mode):
    """The layer stack written out from its parts: scipy's correlate for each 3x3x3 tap sum,
    the bias of each output channel read from the flat layout (weights [Cout][Cin][3][3][3],
    then biases [Cout], layer by layer), x * Phi(x) between layers and nothing after the last."""
    off = 0
    a = np.asarray(x, dtype=np.float64)
    n = len(widths) - 1
    for l in range(n):
        cin, cout = widths[l], widths[l + 1]
        w = params[off:off + cout * cin * 27].reshape(cout, cin, 3, 3, 3)
        off += cout * cin * 27
        b = params[off:off + cout]
        off += cout
        z = np.stack([b[co] + sum(ndimage.correlate(a[ci], w[co, ci], mode=mode) for ci in range(cin))
                      for co in range(cout)])
        a = z * special.ndtr(z) if l + 1 < n else z
    assert off == params.size
    return a


@pytest.mark.parametrize("widths", [[1, 3, 2], [1, 4, 3, 3], [2, 3, 4, 3]])
def test_surrogate_forward_composed_from_library_parts(widths):
    rng = np.random.default_rng(3)
    x = rng.standard_normal((widths[0], 5, 6, 4))
    params = _params(widths, rng)
    params[-widths[-1]:] += 3.0          # output biases far from zero: a bias read at the wrong offset shows
    for bnd, mode in ((O.REFLECT, "mirror"), (O.PERIODIC, "wrap")):
        got = O.surrogate_forward(x, widths, params, bnd=bnd)
        ref = _compose_forward(x, widths, params, mode)
        np.testing.assert_allclose(got, ref, rtol=1e-12, atol=1e-12)


def test_surrogate_forward_has_no_activation_after_the_last_layer():
    # one layer of a single centre tap with weight 1 and bias -2: the output is x - 2, negative
    # values included (a GELU after it would bend them towards zero)
    widths = [1, 1]
    w = np.zeros(27)
    w[13] = 1.0
    params = np.concatenate([w, [-2.0]])
    x = np.linspace(-3, 3, 2 * 3 * 4).reshape(1, 2, 3, 4)
    np.testing.assert_allclose(O.surrogate_forward(x, widths, params), x - 2.0, rtol=0, atol=1e-15)
    # two such layers: GELU sits between them only
    params2 = np.concatenate([w, [0.5], w, [0.0]])
    z = x + 0.5
    np.testing.assert_allclose(O.surrogate_forward(x, [1, 1, 1], params2), z * special.ndtr(z), rtol=1e-13,
                               atol=1e-15)
