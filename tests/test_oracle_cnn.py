"""Pins of the warm-start network oracle: scipy correlation, finite differences,
Adam's closed-form first step, bfloat16 rounding."""

import numpy as np
import pytest
from scipy.signal import correlate2d

from oracle import cnn_oracle as C


def test_single_channel_conv_is_correlation():
    g = np.random.default_rng(0)
    x = g.standard_normal((1, 13, 17, 1))
    w = g.standard_normal((3, 3, 1, 1))
    out = C.conv3x3(x, w, np.array([0.25]))
    ref = correlate2d(x[0, :, :, 0], w[:, :, 0, 0], mode="same", boundary="fill") + 0.25
    np.testing.assert_allclose(out[0, :, :, 0], ref, rtol=1e-13, atol=1e-13)


def test_multi_channel_conv_is_sum_of_correlations():
    g = np.random.default_rng(1)
    x = g.standard_normal((2, 9, 11, 3))
    w = g.standard_normal((3, 3, 3, 2))
    out = C.conv3x3(x, w, np.zeros(2))
    for n in range(2):
        for o in range(2):
            ref = sum(correlate2d(x[n, :, :, i], w[:, :, i, o], mode="same") for i in range(3))
            np.testing.assert_allclose(out[n, :, :, o], ref, rtol=1e-12, atol=1e-12)


def _tiny_net(g, chans=(5, 4, 4, 1)):
    return [(g.standard_normal((3, 3, a, b)) * 0.4, g.standard_normal(b) * 0.1)
            for a, b in zip(chans[:-1], chans[1:])]


def test_network_gradients_match_finite_differences():
    g = np.random.default_rng(2)
    params = _tiny_net(g)
    x = g.standard_normal((2, 6, 7, 5))
    t = g.standard_normal((2, 6, 7))

    def loss(ps):
        out, _, _ = C.forward(ps, x)
        return C.mse_loss(out, t)[0]

    out, inputs, pre = C.forward(params, x)
    _, dout = C.mse_loss(out, t)
    grads = C.backward(params, inputs, pre, dout)
    eps = 1e-6
    for li in range(len(params)):
        for which in (0, 1):
            arr = params[li][which]
            idx = [tuple(g.integers(0, s) for s in arr.shape) for _ in range(4)]
            for ix in idx:
                plus = [(w.copy(), b.copy()) for w, b in params]
                minus = [(w.copy(), b.copy()) for w, b in params]
                plus[li][which][ix] += eps
                minus[li][which][ix] -= eps
                fd = (loss(plus) - loss(minus)) / (2 * eps)
                assert abs(grads[li][which][ix] - fd) <= 1e-6 * max(1.0, abs(fd)) + 1e-9


def test_input_gradient_matches_finite_differences():
    g = np.random.default_rng(3)
    w = g.standard_normal((3, 3, 2, 3))
    x = g.standard_normal((1, 5, 6, 2))
    dout = g.standard_normal((1, 5, 6, 3))
    dx, _, _ = C.conv3x3_backward(x, w, dout)
    eps = 1e-6
    for ix in [(0, 0, 0, 0), (0, 4, 5, 1), (0, 2, 3, 0)]:
        xp, xm = x.copy(), x.copy()
        xp[ix] += eps
        xm[ix] -= eps
        fd = (np.sum(C.conv3x3(xp, w, np.zeros(3)) * dout) -
              np.sum(C.conv3x3(xm, w, np.zeros(3)) * dout)) / (2 * eps)
        assert abs(dx[ix] - fd) <= 1e-7 * max(1.0, abs(fd))


def test_adam_first_step_closed_form():
    g = np.array([3.0, -0.5, 1e-3, 0.0])
    p, m, v = C.adam_step(np.zeros(4), g, np.zeros(4), np.zeros(4), 1, lr=0.01)
    # bias-corrected moments equal g and g^2 after one step
    np.testing.assert_allclose(p, -0.01 * g / (np.abs(g) + 1e-8), rtol=1e-12)


@pytest.mark.parametrize("v,exp", [(1.0, 1.0), (1.0078125, 1.0078125), (1.00390625, 1.0),
                                   (1.01171875, 1.015625), (1.001953125, 1.0),
                                   (1.005859375, 1.0078125), (-3.140625, -3.140625)])
def test_bf16_rounding(v, exp):
    # bfloat16 keeps 7 fraction bits: spacing 2^-7 at 1.  1 + 2^-8 is a tie and
    # goes to the even neighbour 1.0; 1 + 3 * 2^-8 ties up to 1 + 2^-6;
    # 1 + 2^-9 is below half a step; 1 + 3 * 2^-9 is above half a step.
    assert C.bf16_round(np.array([v]))[0] == exp


def test_descriptors_of_delta_and_gaussian_psfs():
    K = 31
    delta = np.zeros((1, 1, K, K))
    delta[0, 0, K // 2, K // 2] = 1.0
    d = C.psf_descriptors(delta)[0, 0]
    np.testing.assert_allclose(d, [0.0, 10.0, 0.0], atol=1e-15)
    # 2-D Gaussian of std s: E[r^2] = 2 s^2 (well inside the support)
    s = 2.0
    yy, xx = np.mgrid[0:K, 0:K] - K // 2
    h = np.exp(-0.5 * (yy ** 2 + xx ** 2) / s ** 2)
    d = C.psf_descriptors((h / h.sum())[None, None])[0, 0]
    assert abs(d[0] - np.sqrt(2) * s / 8.0) < 1e-6


def test_feature_maps_interpolate_descriptors():
    from oracle import dv_oracle as O
    g = np.random.default_rng(4)
    K = 5
    psfs = g.uniform(0, 1, (2, 3, K, K))
    y = g.uniform(0, 1, (20, 30))
    wr, wc = O.bilinear_weights(24, 2), O.bilinear_weights(34, 3)
    f = C.warmstart_features(y, psfs, 0.01, wr, wc)
    d = C.psf_descriptors(psfs)
    # at a grid corner the map equals that PSF's descriptor; elsewhere it is a convex mix
    np.testing.assert_allclose(f[0, 0, 1:4], d[0, 0], rtol=1e-12)
    np.testing.assert_allclose(f[23, 33, 1:4], d[1, 2], rtol=1e-12)
    assert np.all(f[..., 1] >= d[..., 0].min() - 1e-12) and np.all(f[..., 1] <= d[..., 0].max() + 1e-12)
    np.testing.assert_allclose(f[2:-2, 2:-2, 0], y)
    np.testing.assert_allclose(f[..., 4], 1.0)
