"""Pins of the oracle's evaluation measures (reading R19, Sec. IV-C): SNR in
closed form, SSIM against its definition evaluated window by window, its
closed form on constant images, identity and symmetry."""

import numpy as np
import pytest

from oracle import dv_oracle as O


def test_snr_closed_form():
    g = np.random.default_rng(1)
    ref = g.uniform(0, 1, (20, 30))
    x = ref + 0.01
    assert O.snr_db(x, ref) == pytest.approx(10 * np.log10(np.sum(ref ** 2) / (600 * 1e-4)),
                                             rel=1e-12)
    assert O.snr_db(ref, ref) == float("inf")


def test_ssim_window_is_the_unit_sum_gaussian():
    w = O.ssim_window()
    assert w.shape == (11, 11) and w.sum() == pytest.approx(1.0, abs=1e-15)
    assert w[5, 5] / w[5, 6] == pytest.approx(np.exp(1 / (2 * 1.5 ** 2)), rel=1e-12)
    np.testing.assert_allclose(w, w.T, rtol=0, atol=0)


def test_ssim_equals_the_window_by_window_definition():
    g = np.random.default_rng(2)
    x, r = g.uniform(0, 1, (15, 17)), g.uniform(0, 1, (15, 17))
    w = O.ssim_window()
    c1, c2 = 0.01 ** 2, 0.03 ** 2
    vals = []
    for i in range(15 - 10):
        for j in range(17 - 10):
            a, b = x[i:i + 11, j:j + 11], r[i:i + 11, j:j + 11]
            ma, mb = np.sum(w * a), np.sum(w * b)
            va, vb = np.sum(w * (a - ma) ** 2), np.sum(w * (b - mb) ** 2)
            cab = np.sum(w * (a - ma) * (b - mb))
            vals.append((2 * ma * mb + c1) * (2 * cab + c2) / ((ma ** 2 + mb ** 2 + c1) * (va + vb + c2)))
    assert O.ssim(x, r) == pytest.approx(np.mean(vals), rel=1e-12)


def test_ssim_constant_images_and_identity():
    a, b = 0.3, 0.7
    x, r = np.full((30, 40), a), np.full((30, 40), b)
    c1 = 0.01 ** 2
    assert O.ssim(x, r) == pytest.approx((2 * a * b + c1) / (a * a + b * b + c1), rel=1e-12)
    g = np.random.default_rng(3)
    y = g.uniform(0, 1, (25, 33))
    z = g.uniform(0, 1, (25, 33))
    assert O.ssim(y, y) == pytest.approx(1.0, abs=1e-12)
    assert O.ssim(y, z) == pytest.approx(O.ssim(z, y), abs=1e-14)
    assert O.ssim(y, z) < 0.5
