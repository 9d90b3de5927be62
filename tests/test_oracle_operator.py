"""Pins of the oracle's interpolation weights and shift-variant operator
(Sec. II-B, Eq. (2), Fig. 1) against closed forms, scipy routines and invariants."""

import json
import os

import numpy as np
import pytest
from scipy.signal import convolve2d, correlate2d

from oracle import dv_oracle as O
from tests.oracle_helpers import dense_H

pytestmark = pytest.mark.filterwarnings("ignore::DeprecationWarning")


def _rand_psfs(g, Gr, Gc, K):
    p = g.uniform(0.0, 1.0, (Gr, Gc, K, K))
    return p / p.sum(axis=(2, 3), keepdims=True)


def test_tent_weights_golden(golden_dir):
    d = json.load(open(os.path.join(golden_dir, "tent_weights_n5_G3.json")))
    np.testing.assert_allclose(O.bilinear_weights(d["n"], d["G"]), np.array(d["weights"]),
                               rtol=0, atol=1e-15)


@pytest.mark.parametrize("n,G", [(136, 3), (2078, 8), (97, 2), (40, 1), (1001, 17)])
def test_weights_partition_of_unity(n, G):
    w = O.bilinear_weights(n, G)
    assert w.min() >= 0.0 and w.max() <= 1.0
    assert np.max(np.abs(w.sum(axis=0) - 1.0)) <= 1e-12
    # at most two neighbouring grid points are active at any pixel (first order)
    assert np.max((w > 0).sum(axis=0)) <= 2


def test_uniform_blocks_golden(golden_dir):
    d = json.load(open(os.path.join(golden_dir, "uniform_blocks.json")))
    for c in d["cases"]:
        assert O.uniform_blocks(c["n"], c["count"], c["overlap"]) == [tuple(b) for b in c["blocks"]]


def test_equal_psfs_reduce_to_convolution():
    """With one PSF everywhere the weights sum to 1 and H is ordinary 'valid' convolution."""
    g = np.random.default_rng(11)
    K, Gr, Gc = 5, 3, 4
    x = g.uniform(0, 1, (37, 41))
    h = g.uniform(0, 1, (K, K))
    h /= h.sum()
    psfs = np.broadcast_to(h, (Gr, Gc, K, K)).copy()
    wr, wc = O.bilinear_weights(37, Gr), O.bilinear_weights(41, Gc)
    y = O.apply_H(x, psfs, wr, wc)
    ref = convolve2d(x, h, mode="valid")
    np.testing.assert_allclose(y, ref, rtol=1e-12, atol=1e-14)
    pts = [(0, 0), (5, 7), (32, 36), (17, 3)]
    np.testing.assert_allclose(O.apply_H_at(x, psfs, wr, wc, pts),
                               [ref[i, j] for i, j in pts], rtol=1e-12)
    # the adjoint is the 'full' correlation
    r = g.standard_normal(ref.shape)
    gt = correlate2d(r, h, mode="full")
    np.testing.assert_allclose(O.apply_Ht(r, psfs, wr, wc), gt, rtol=1e-12, atol=1e-13)
    ptx = [(0, 0), (36, 40), (4, 39), (20, 20)]
    np.testing.assert_allclose(O.apply_Ht_at(r, psfs, wr, wc, ptx), [gt[i, j] for i, j in ptx],
                               rtol=1e-12, atol=1e-13)


def test_delta_psf_is_crop():
    K = 7
    g = np.random.default_rng(3)
    x = g.uniform(0, 1, (30, 25))
    psfs = np.zeros((2, 3, K, K))
    psfs[:, :, K // 2, K // 2] = 1.0
    y = O.apply_H(x, psfs, O.bilinear_weights(30, 2), O.bilinear_weights(25, 3))
    np.testing.assert_allclose(y, x[K // 2:-(K // 2), K // 2:-(K // 2)], rtol=1e-14)


def test_impulse_response_interpolates_grid_psfs():
    """Sec. II-B: the PSF at a grid point is the sampled PSF, and between two grid
    points it is their first-order (linear) interpolation."""
    K, n = 5, 41            # grid spacing 10 with G = 5: points at 0, 10, 20, 30, 40
    g = np.random.default_rng(5)
    psfs = _rand_psfs(g, 5, 5, K)
    wr, wc = O.bilinear_weights(n, 5), O.bilinear_weights(n, 5)
    # impulse exactly at grid point (20, 30)
    x = np.zeros((n, n))
    x[20, 30] = 1.0
    y = O.apply_H(x, psfs, wr, wc)
    exp = np.zeros_like(y)
    exp[20 - K + 1:21, 30 - K + 1:31] = psfs[2, 3]
    np.testing.assert_allclose(y, exp, atol=1e-15)
    # impulse 3/10 of the way from grid row 1 (R=10) to grid row 2 (R=20), column on grid 1
    x = np.zeros((n, n))
    x[13, 10] = 1.0
    y = O.apply_H(x, psfs, wr, wc)
    exp = np.zeros_like(y)
    exp[13 - K + 1:14, 10 - K + 1:11] = 0.7 * psfs[1, 1] + 0.3 * psfs[2, 1]
    np.testing.assert_allclose(y, exp, atol=1e-15)


def test_dense_matrix_brute_force():
    """Shift-variant H and H^T against a matrix assembled column by column with
    scipy.signal.convolve2d."""
    g = np.random.default_rng(7)
    K, Gr, Gc = 3, 3, 2
    nxr, nxc = 11, 9
    psfs = g.uniform(-0.2, 1.0, (Gr, Gc, K, K))
    wr, wc = O.bilinear_weights(nxr, Gr), O.bilinear_weights(nxc, Gc)
    M = dense_H(psfs, wr, wc)
    x = g.standard_normal((nxr, nxc))
    r = g.standard_normal((nxr - K + 1, nxc - K + 1))
    np.testing.assert_allclose(O.apply_H(x, psfs, wr, wc).ravel(), M @ x.ravel(), rtol=1e-12,
                               atol=1e-13)
    np.testing.assert_allclose(O.apply_Ht(r, psfs, wr, wc).ravel(), M.T @ r.ravel(), rtol=1e-12,
                               atol=1e-13)
    pts = [(0, 0), (8, 6), (3, 2)]
    np.testing.assert_allclose(O.apply_H_at(x, psfs, wr, wc, pts),
                               [(M @ x.ravel()).reshape(9, 7)[i, j] for i, j in pts], rtol=1e-12)
    ptx = [(0, 0), (10, 8), (5, 1)]
    np.testing.assert_allclose(O.apply_Ht_at(r, psfs, wr, wc, ptx),
                               [(M.T @ r.ravel()).reshape(nxr, nxc)[i, j] for i, j in ptx],
                               rtol=1e-12, atol=1e-13)
    # the step-size bound really bounds ||H||^2 for nonnegative PSFs
    pp = np.abs(psfs)
    assert O.lipschitz_bound_H(pp) >= np.linalg.norm(dense_H(pp, wr, wc), 2) ** 2 * (1 - 1e-12)


@pytest.mark.parametrize("K,G,shape", [(7, (3, 3), (60, 52)), (9, (3, 3), (136, 136)),
                                       (3, (1, 1), (12, 20))])
def test_adjoint_identity(K, G, shape):
    g = np.random.default_rng(K)
    psfs = g.uniform(-0.5, 1.0, G + (K, K))
    wr, wc = O.bilinear_weights(shape[0], G[0]), O.bilinear_weights(shape[1], G[1])
    x = g.standard_normal(shape)
    r = g.standard_normal((shape[0] - K + 1, shape[1] - K + 1))
    lhs = np.vdot(O.apply_H(x, psfs, wr, wc), r)
    rhs = np.vdot(x, O.apply_Ht(r, psfs, wr, wc))
    assert abs(lhs - rhs) <= 1e-13 * max(1.0, abs(lhs)) * 10
