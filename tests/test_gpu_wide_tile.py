"""Algorithm 1 at the scale of the 8192 x 8192 workload against the FP64 oracle.

The GPU runs two outer iterations (one projected-gradient step each) of the
consensus solve over all 81 uneven tiles of the 8254^2-pixel x grid, with the
16 x 16 grid of 63 x 63 Moffat PSFs and per-pixel noise weights W (Eq. (3)),
and exports the D-R state (x_i, u_i).  The oracle recomputes the state on a
128 x 128 window that straddles the overlap band of two neighbouring tiles,
so both the Local-Solver steps and the consensus average of Lemma 1 over two
covering tiles (Sec. III-B) are checked element by element.

A projected-gradient step at a pixel reads the iterate within 2 (K - 1) + 1 =
125 pixels (H, then H^T, then the prior's difference stencil), so after two
steps the window depends on its 250-pixel surround only.  The oracle therefore
runs its Local-Solver on crops of each tile: the window grown by 250 pixels
(first outer iteration), then by 125 (second), clipped to the tile, with the
tile's own step size, consensus weights and noise weights.  Where a crop ends
at the tile's edge it is the tile's edge; elsewhere the crop's edge lies
farther from the window than the dependency reaches.  The observed image is a
seeded star field with Poisson + Gaussian noise drawn directly (not through a
CUDA operator)."""

import numpy as np
import pytest

from oracle import dv_oracle as O
from tests.gpu_common import assert_close, need_gpu

pytestmark = pytest.mark.gpu

FFT = 2
REACH = 125          # 2 (K - 1) + 1 for K = 63


def _tile_views(stack, lay):
    """Tile arrays of an exported x-shaped stack (tiles in row-major order,
    rows padded to 32 floats, tiles starting on 32-float boundaries)."""
    out, off = {}, 0
    for tr, tc in lay.tiles:
        rs, cs = lay.xslice(tr, tc)
        nr, nc = rs.stop - rs.start, cs.stop - cs.start
        pitch = -(-nc // 32) * 32
        out[(tr, tc)] = stack[off:off + nr * pitch].reshape(nr, pitch)[:, :nc]
        off += -(-(nr * pitch) // 32) * 32
    return out


def test_wide8192_two_outer_iterations_on_a_window_across_two_tiles():
    torch, dv = need_gpu()
    from paper_1705_06603_gb300.synth import WORKLOADS, poisson_gaussian, psf_grid_for, star_field
    w = WORKLOADS["wide8192"]
    K = w.K
    psfs = psf_grid_for(w)
    y, W = poisson_gaussian(star_field((w.hy, w.wy), 21, dtype=np.float64), w.poisson_peak,
                            w.noise_sigma, 22)
    y32, W32 = y.astype(np.float32), W.astype(np.float32)

    plan = dv.Plan(w.hy, w.wy, psfs.astype(np.float32), n_tiles=w.n_tiles, overlap=w.overlap,
                   tile_bounds=(w.yrows, w.ycols), lam=w.lam, delta=w.delta, gamma=w.gamma,
                   rho=w.rho, n_outer=2, n_inner=1, path=FFT, noise_w=W32)
    assert plan.info.path == FFT
    plan.solve(torch.from_numpy(y32).cuda(), stats=False)
    xs = torch.empty(plan.info.stack_elems, device="cuda")
    us = torch.empty_like(xs)
    assert dv.dv_state_export(plan.handle, xs, us) == 2
    torch.cuda.synchronize()
    plan.close()
    lay = O.make_layout(w.hy, w.wy, K, *w.n_tiles, w.overlap, w.yrows, w.ycols)
    gx, gu = _tile_views(xs.cpu().numpy(), lay), _tile_views(us.cpu().numpy(), lay)
    # the oracle sees the values the GPU was given
    y64, W64 = y32.astype(np.float64), W32.astype(np.float64)
    ps64 = psfs.astype(np.float32).astype(np.float64)

    # window: rows inside tile row 4's exclusive band, columns across the overlap
    # of tile columns 4 and 5 (one column covered by each tile alone on either side)
    tiles = [(4, 4), (4, 5)]
    (r0a, r1a), (r0b, r1b) = lay.xrows[3], lay.xrows[5]
    rmid = (lay.xrows[4][0] + lay.xrows[4][1]) // 2
    c_lo, c_hi = lay.xcols[5][0] - 1, lay.xcols[4][1] + 1
    win_r, win_c = (rmid - 64, rmid + 64), (c_lo, c_hi)
    assert win_r[0] - 2 * REACH >= r1a and win_r[1] + 2 * REACH <= r0b
    assert lay.xcols[3][1] <= win_c[0] - 2 * REACH and lay.xcols[6][0] >= win_c[1] + 2 * REACH

    wr_all = O.bilinear_weights(lay.nx[0], w.grid[0])
    wc_all = O.bilinear_weights(lay.nx[1], w.grid[1])
    x0 = O.start_image(y64, K)

    def crop(t, grow):
        """Global x ranges of the window grown by `grow`, clipped to tile t."""
        (ta, tb), (tc0, tc1) = lay.xrows[t[0]], lay.xcols[t[1]]
        return ((max(ta, win_r[0] - grow), min(tb, win_r[1] + grow)),
                (max(tc0, win_c[0] - grow), min(tc1, win_c[1] + grow)))

    def step(t, rr, cc, wv, uv):
        """One Local-Solver step of tile t on the x crop rr x cc (global
        coordinates) from the crop arrays wv, uv."""
        (ta, _), (tc0, _) = lay.xrows[t[0]], lay.xcols[t[1]]
        ys = (slice(rr[0], rr[1] - K + 1), slice(cc[0], cc[1] - K + 1))
        om = lay.omega(*t)[rr[0] - ta:rr[1] - ta, cc[0] - tc0:cc[1] - tc0]
        tau = O.tile_step(lay, *t, ps64, W64, w.lam, w.gamma)
        return O.local_solve(wv, uv, y64[ys], W64[ys], ps64, wr_all[:, rr[0]:rr[1]],
                             wc_all[:, cc[0]:cc[1]], w.gamma * om, w.lam, w.delta, tau, 1)

    def zbar(vals):
        """Lemma 1 over the covering tiles: vals[t] = (2 x - u) on tile t's
        window part (global array with NaN elsewhere); the oracle's consensus
        average over the layout with those tiles filled in."""
        vs = []
        for t in lay.tiles:
            rs, cs = lay.xslice(*t)
            v = np.zeros((rs.stop - rs.start, cs.stop - cs.start))
            if t in vals:
                v[:] = np.nan_to_num(vals[t][rs, cs])
            vs.append(v)
        return O.consensus_average(lay, vs, [w.gamma * lay.omega(*t) for t in lay.tiles])

    # outer iteration 1 on each tile's crop (valid on the window grown by REACH)
    x1, u0 = {}, {}
    for t in tiles:
        rr, cc = crop(t, 2 * REACH)
        u0[t] = x0.copy()
        x1[t] = np.full(lay.nx, np.nan)
        x1[t][rr[0]:rr[1], cc[0]:cc[1]] = step(t, rr, cc, x0[rr[0]:rr[1], cc[0]:cc[1]],
                                               x0[rr[0]:rr[1], cc[0]:cc[1]])
    z1 = zbar({t: 2 * x1[t] - u0[t] for t in tiles})
    u1 = {t: u0[t] + w.rho * (z1 - x1[t]) for t in tiles}
    # outer iteration 2
    x2 = {}
    for t in tiles:
        rr, cc = crop(t, REACH)
        x2[t] = np.full(lay.nx, np.nan)
        x2[t][rr[0]:rr[1], cc[0]:cc[1]] = step(t, rr, cc, x1[t][rr[0]:rr[1], cc[0]:cc[1]],
                                               u1[t][rr[0]:rr[1], cc[0]:cc[1]])
    z2 = zbar({t: 2 * x2[t] - u1[t] for t in tiles})
    for t in tiles:
        rr, cc = crop(t, 0)
        (ta, _), (tc0, _) = lay.xrows[t[0]], lay.xcols[t[1]]
        sl = (slice(rr[0], rr[1]), slice(cc[0], cc[1]))
        tl = (slice(rr[0] - ta, rr[1] - ta), slice(cc[0] - tc0, cc[1] - tc0))
        u2 = u1[t][sl] + w.rho * (z2[sl] - x2[t][sl])
        assert np.isfinite(x2[t][sl]).all() and np.isfinite(u2).all()
        assert_close(gx[t][tl], x2[t][sl], 1e-5)
        assert_close(gu[t][tl], u2, 1e-5)
