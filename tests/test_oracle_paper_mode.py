"""Pins of the oracle's one-PSF-per-block mode (reading R18, Sec. III-A and
III-C): the block geometry, the tile operator against scipy's valid
convolution, the reduction to the interpolated model when every PSF is the
same, and the consensus weights as first-order interpolation tents."""

import numpy as np
import pytest
from scipy.signal import convolve2d

from oracle import dv_oracle as O


@pytest.mark.parametrize("ny,K,G", [(128, 9, 3), (2048, 31, 8), (150, 15, 2), (301, 9, 5),
                                    (8192, 63, 16)])
def test_paper_blocks_span_three_cells(ny, K, G):
    blocks = O.paper_blocks(ny, K, G)
    n = ny + K - 1
    cell = n / G
    xt = [(s, e + K - 1) for s, e in blocks]
    assert blocks[0][0] == 0 and blocks[-1][1] == ny
    for i, (x0, x1) in enumerate(xt):
        lo, hi = max(0.0, (i - 0.5) * cell), min(n, (i + 1.5) * cell)
        assert abs(x0 - lo) <= 1 and abs(x1 - hi) <= 1       # cells i - 1 .. i + 1
        if i + 1 < G:
            # neighbours share one cell, and the y-blocks leave no gap
            assert abs((x1 - xt[i + 1][0]) - cell) <= 1
            assert blocks[i + 1][0] <= blocks[i][1]
        if i + 2 < G:
            assert xt[i + 2][0] >= x1                          # only neighbours overlap


def test_per_tile_operator_is_valid_convolution():
    g = np.random.default_rng(3)
    lay = O.paper_layout(60, 52, 7, 3, 2)
    psfs = g.uniform(0, 1, (3, 2, 7, 7))
    for tr, tc in lay.tiles:
        xi = g.uniform(0, 1, (lay.xrows[tr][1] - lay.xrows[tr][0],
                              lay.xcols[tc][1] - lay.xcols[tc][0]))
        p, wr, wc = O.tile_operator(lay, tr, tc, psfs, "per_tile")
        ref = convolve2d(xi, psfs[tr, tc], mode="valid")
        np.testing.assert_allclose(O.apply_H(xi, p, wr, wc), ref, rtol=1e-12, atol=1e-12)


def test_equal_psfs_reduce_to_the_interpolated_model():
    """With every PSF equal, H_i is the shift-invariant blur in both models
    (the tents sum to 1), so the solves coincide."""
    g = np.random.default_rng(4)
    K, G = 7, (3, 3)
    lay = O.paper_layout(64, 64, K, *G)
    h = g.uniform(0, 1, (K, K))
    h /= h.sum()
    psfs = np.broadcast_to(h, G + (K, K)).copy()
    y = g.uniform(0, 1, (64, 64))
    a, ia = O.solve(y, psfs, lay, 1e-3, 1 / 60, 0.4, 1.0, 3, 4, inner_increment=2,
                    weights="per_tile")
    b, ib = O.solve(y, psfs, lay, 1e-3, 1 / 60, 0.4, 1.0, 3, 4, inner_increment=2)
    np.testing.assert_allclose(a, b, rtol=1e-12, atol=1e-12)
    np.testing.assert_allclose(ia.taus, ib.taus, rtol=1e-14)


def test_paper_consensus_weights_are_tents():
    """On the paper's blocks an interior tile has no exclusive part: its
    weight ramps up across the cell shared with one neighbour and down across
    the other, and the weights of all tiles sum to 1."""
    lay = O.paper_layout(300, 300, 9, 5, 5)
    for om in lay.omega_r[1:-1]:
        d = np.diff(om)
        peak = int(np.argmax(om))
        # strictly up to the peak, then down (two equal peak pixels at most)
        assert np.all(d[:peak] > 0) and d[peak] <= 0 and np.all(d[peak + 1:] < 0)
        assert om.min() > 0 and om.max() < 1
    tot = np.zeros(lay.nx[0])
    for (s, e), om in zip(lay.xrows, lay.omega_r):
        tot[s:e] += om
    np.testing.assert_allclose(tot, 1.0, rtol=1e-14)
