"""Pins of the oracle's Huber prior (Sec. IV-A), consensus weights and Lemma 1
(Sec. III-B), projected-gradient Local-Solver, and Algorithm 1 as a whole."""

import json
import os

import numpy as np
import pytest

from oracle import dv_oracle as O
from tests.oracle_helpers import dense_D, dense_H, huber_terms, lbfgsb_min


# --------------------------------------------------------------------------- prior


def test_huber_golden(golden_dir):
    d = json.load(open(os.path.join(golden_dir, "huber_single_pixel_3x3.json")))
    x = np.array(d["x"], dtype=float)
    for c in d["cases"]:
        assert abs(O.huber_value(x, c["delta"]) - c["phi"]) <= 1e-15
        if "grad" in c:
            np.testing.assert_allclose(O.huber_gradient(x, c["delta"]), np.array(c["grad"], float),
                                       atol=1e-15)


def test_huber_large_delta_is_quadratic():
    g = np.random.default_rng(1)
    x = g.standard_normal((9, 13))
    q = 0.5 * (np.sum(np.diff(x, axis=0) ** 2) + np.sum(np.diff(x, axis=1) ** 2))
    assert abs(O.huber_value(x, 1e6) - q) <= 1e-12 * q


def test_huber_small_delta_is_scaled_tv():
    g = np.random.default_rng(2)
    x = g.standard_normal((8, 10))
    dr = np.zeros_like(x)
    dr[:-1] = np.diff(x, axis=0)
    dc = np.zeros_like(x)
    dc[:, :-1] = np.diff(x, axis=1)
    s = np.hypot(dr, dc)
    delta = 1e-9
    # every nonzero gradient is far above delta: phi = sum delta (s - delta/2)
    nz = s > 0
    exp = np.sum(delta * (s[nz] - 0.5 * delta))
    assert abs(O.huber_value(x, delta) - exp) <= 1e-12 * exp


@pytest.mark.parametrize("delta", [0.05, 0.5, 5.0])
def test_huber_gradient_finite_differences(delta):
    g = np.random.default_rng(3)
    x = g.uniform(0, 1, (7, 6))
    gr = O.huber_gradient(x, delta)
    eps = 1e-6
    fd = np.zeros_like(x)
    for i in range(x.shape[0]):
        for j in range(x.shape[1]):
            xp, xm = x.copy(), x.copy()
            xp[i, j] += eps
            xm[i, j] -= eps
            fd[i, j] = (O.huber_value(xp, delta) - O.huber_value(xm, delta)) / (2 * eps)
    np.testing.assert_allclose(gr, fd, rtol=1e-6, atol=1e-8)


# --------------------------------------------------------------------------- consensus


def test_consensus_profiles_golden(golden_dir):
    d = json.load(open(os.path.join(golden_dir, "consensus_profiles_two_tiles.json")))
    prof = O.consensus_profiles([tuple(r) for r in d["xranges"]])
    for p, e in zip(prof, d["profiles"]):
        np.testing.assert_allclose(p, e, atol=1e-15)


@pytest.mark.parametrize("wl", ["disks128", "stars2048", "wide8192"])
def test_consensus_weights_partition_and_positivity(wl):
    from paper_1705_06603_gb300.synth import WORKLOADS
    w = WORKLOADS[wl]
    lay = O.make_layout(w.hy, w.wy, w.K, *w.n_tiles, w.overlap, w.yrows, w.ycols)
    for axis_ranges, prof in ((lay.xrows, lay.omega_r), (lay.xcols, lay.omega_c)):
        n = max(e for _, e in axis_ranges)
        tot = np.zeros(n)
        cover = np.zeros(n, int)
        for (s, e), p in zip(axis_ranges, prof):
            assert p.min() > 0.0 and p.max() <= 1.0 + 1e-15
            tot[s:e] += p
            cover[s:e] += 1
        assert np.max(np.abs(tot - 1.0)) <= 1e-12
        # exactly 1 where only one tile covers the pixel
        for (s, e), p in zip(axis_ranges, prof):
            only = cover[s:e] == 1
            np.testing.assert_array_equal(p[only], 1.0)


def test_lemma_pixel_golden(golden_dir):
    d = json.load(open(os.path.join(golden_dir, "consensus_lemma_pixel.json")))
    lay = O.Layout(1, 1, 1, [(0, 1)], [(0, 1), (0, 1)])   # two tiles on one pixel
    x = [np.array([[v]]) for v in d["x"]]
    u = [np.array([[v]]) for v in d["u"]]
    al = [np.array([[v]]) for v in d["alpha"]]
    z = O.consensus_average(lay, [2 * a - b for a, b in zip(x, u)], al)
    assert abs(z[0, 0] - d["zbar"]) <= 1e-15
    un = [b + d["rho"] * (z - a) for a, b in zip(x, u)]
    np.testing.assert_allclose([v[0, 0] for v in un], d["u_next"], atol=1e-15)


def test_consensus_is_weighted_mean_and_argmin():
    """Lemma 1: the prox of the consensus indicator is the alpha-weighted mean,
    checked against numpy.average and by perturbing the minimiser."""
    g = np.random.default_rng(4)
    lay = O.make_layout(20, 24, 5, 2, 3, 6)
    vs = [g.standard_normal((r.stop - r.start, c.stop - c.start))
          for r, c in (lay.xslice(*t) for t in lay.tiles)]
    als = [g.uniform(0.1, 2.0, v.shape) for v in vs]
    z = O.consensus_average(lay, vs, als)
    for R in range(0, lay.nx[0], 3):
        for C in range(0, lay.nx[1], 4):
            vals, ws = [], []
            for n, t in enumerate(lay.tiles):
                rs, cs = lay.xslice(*t)
                if rs.start <= R < rs.stop and cs.start <= C < cs.stop:
                    vals.append(vs[n][R - rs.start, C - cs.start])
                    ws.append(als[n][R - rs.start, C - cs.start])
            assert abs(z[R, C] - np.average(vals, weights=ws)) <= 1e-13
            q = lambda w: sum(a * (w - v) ** 2 for a, v in zip(ws, vals))
            assert q(z[R, C]) <= min(q(z[R, C] + 1e-4), q(z[R, C] - 1e-4))


def test_consensus_fixed_point_invariant():
    """If all tiles agree and u = x, then zbar = x and the dual update is a no-op."""
    g = np.random.default_rng(5)
    lay = O.make_layout(30, 30, 3, 3, 3, 5)
    xg = g.uniform(0, 1, lay.nx)
    xs = [xg[lay.xslice(*t)] for t in lay.tiles]
    al = [0.4 * lay.omega(*t) for t in lay.tiles]
    z = O.consensus_average(lay, [2 * x - x for x in xs], al)
    np.testing.assert_allclose(z, xg, rtol=1e-14)
    np.testing.assert_allclose(O.assemble(lay, xs), xg, rtol=1e-14)


# --------------------------------------------------------------------------- local solver


def _tiny_problem(seed, hy=10, wy=12, K=3, G=(2, 2), tiles=(2, 2), overlap=4, delta=10.0):
    g = np.random.default_rng(seed)
    lay = O.make_layout(hy, wy, K, *tiles, overlap)
    psfs = g.uniform(0.2, 1.0, G + (K, K))
    psfs /= psfs.sum(axis=(2, 3), keepdims=True)
    xt = g.uniform(0, 1, lay.nx)
    wr, wc = O.bilinear_weights(lay.nx[0], G[0]), O.bilinear_weights(lay.nx[1], G[1])
    y = O.apply_H(xt, psfs, wr, wc) + 0.01 * g.standard_normal((hy, wy))
    return lay, psfs, wr, wc, y


def test_projected_gradient_decreases_prox_objective():
    lay, psfs, wr, wc, y = _tiny_problem(6, delta=0.05)
    lam, delta, gamma = 0.05, 0.05, 0.7
    tr, tc = 1, 0
    wri, wci = O.tile_weights(lay, tr, tc, wr, wc)
    yi = y[lay.yslice(tr, tc)]
    g = np.random.default_rng(8)
    w = g.uniform(0, 1, (wri.shape[1], wci.shape[1]))
    u = g.uniform(0, 1, w.shape)
    al = gamma * lay.omega(tr, tc)
    tau = O.tile_step(lay, tr, tc, psfs, None, lam, gamma)
    prev = O.prox_objective(w, u, yi, None, psfs, wri, wci, al, lam, delta)
    for _ in range(40):
        w = O.local_solve(w, u, yi, None, psfs, wri, wci, al, lam, delta, tau, 1)
        cur = O.prox_objective(w, u, yi, None, psfs, wri, wci, al, lam, delta)
        assert cur <= prev + 1e-13 * abs(prev)
        prev = cur
    assert w.min() >= 0.0


def test_local_solver_reaches_prox_minimiser():
    lay, psfs, wr, wc, y = _tiny_problem(9)
    lam, delta, gamma = 0.02, 0.3, 1.0
    tr, tc = 0, 1
    wri, wci = O.tile_weights(lay, tr, tc, wr, wc)
    yi = y[lay.yslice(tr, tc)]
    shape = (wri.shape[1], wci.shape[1])
    g = np.random.default_rng(10)
    u = g.uniform(-0.2, 1, shape)
    al = gamma * lay.omega(tr, tc)
    tau = O.tile_step(lay, tr, tc, psfs, None, lam, gamma)
    w = O.local_solve(u.copy(), u, yi, None, psfs, wri, wci, al, lam, delta, tau, 3000)
    M = dense_H(psfs, wri, wci)
    Dr, Dc = dense_D(*shape)

    def fg(v):
        r = M @ v - yi.ravel()
        hv, hg = huber_terms(Dr, Dc, v, delta)
        d = v - u.ravel()
        return (0.5 * r @ r + lam * hv + 0.5 * np.sum(al.ravel() * d * d),
                M.T @ r + lam * hg + al.ravel() * d)

    ref = lbfgsb_min(fg, np.maximum(u.ravel(), 0))
    np.testing.assert_allclose(w.ravel(), ref, atol=2e-6)


# --------------------------------------------------------------------------- Algorithm 1


def _consensus_minimiser(lay, psfs, wr, wc, y, lam, delta):
    """Brute-force argmin_{x >= 0} sum_i f_i(C_i x) with dense matrices."""
    blocks = []
    for tr, tc in lay.tiles:
        wri, wci = O.tile_weights(lay, tr, tc, wr, wc)
        rs, cs = lay.xslice(tr, tc)
        idx = (np.arange(lay.nx[0])[rs, None] * lay.nx[1] + np.arange(lay.nx[1])[None, cs]).ravel()
        blocks.append((idx, dense_H(psfs, wri, wci), dense_D(rs.stop - rs.start, cs.stop - cs.start),
                       y[lay.yslice(tr, tc)].ravel()))

    def fg(v):
        f, gr = 0.0, np.zeros_like(v)
        for idx, M, (Dr, Dc), yi in blocks:
            xi = v[idx]
            r = M @ xi - yi
            hv, hg = huber_terms(Dr, Dc, xi, delta)
            f += 0.5 * r @ r + lam * hv
            np.add.at(gr, idx, M.T @ r + lam * hg)
        return f, gr

    return lbfgsb_min(fg, np.full(lay.nx[0] * lay.nx[1], 0.5)).reshape(lay.nx), fg


def _dr_pin(oracle_module):
    """Run Algorithm 1 on a tiny problem and measure its distance to the
    brute-force consensus minimiser (max abs error, relative objective gap)."""
    lay, psfs, wr, wc, y = _tiny_problem(12)
    lam, delta = 0.02, 10.0
    ref, fg = _consensus_minimiser(lay, psfs, wr, wc, y, lam, delta)
    xhat, info = oracle_module.solve(y, psfs, lay, lam, delta, gamma=0.5, rho=1.0, n_outer=60,
                                     n_inner=40)
    Fs = fg(ref.ravel())[0]
    return np.abs(xhat - ref).max(), (fg(xhat.ravel())[0] - Fs) / Fs, info, xhat, (y, psfs, lay,
                                                                                   lam, delta, fg)


def test_douglas_rachford_reaches_consensus_minimiser():
    """Sec. III-B: with accurate local solves the D-R iterates converge to a
    minimiser of Eq. (4).  D-R converges sublinearly here (tile-boundary pixels
    are weakly determined), so the pin is the objective gap plus a distance
    bound; the planted-mistake test below shows plausible mistakes land >= 0.1
    away."""
    err, gap, info, xhat, (y, psfs, lay, lam, delta, fg) = _dr_pin(O)
    assert err <= 3e-3 and 0.0 <= gap <= 1e-5
    # the oracle's objective equals the dense brute-force objective at x_hat
    F, _, _ = O.objective(xhat, y, psfs, lay, lam, delta)
    assert abs(F - fg(xhat.ravel())[0]) <= 1e-12 * abs(F)
    assert info.primal[-1] < 1e-2 * info.primal[0]


@pytest.mark.parametrize("mistake", ["unweighted_mean", "convolution_for_adjoint", "prior_sign"])
def test_planted_mistakes_fail_the_pin(monkeypatch, mistake):
    """Plant a plausible mistake in the oracle (CPU only) and check that the D-R
    pin above rejects it."""
    if mistake == "unweighted_mean":
        good = O.consensus_average
        monkeypatch.setattr(O, "consensus_average",
                            lambda lay, vs, al: good(lay, vs, [np.ones_like(a) for a in al]))
    elif mistake == "convolution_for_adjoint":
        good_ht = O.apply_Ht
        monkeypatch.setattr(O, "apply_Ht",
                            lambda r, p, wr, wc: good_ht(r, p[:, :, ::-1, ::-1], wr, wc))
    else:
        good_hg = O.huber_gradient
        monkeypatch.setattr(O, "huber_gradient", lambda x, d: -good_hg(x, d))
    err, gap, *_ = _dr_pin(O)
    assert not (err <= 3e-3 and gap <= 1e-5)


def test_single_tile_is_centralised_solver():
    """With one tile the consensus step is trivial (zbar = 2x - u, u <- x for
    rho = 1) and Algorithm 1 is the proximal-point method on Eq. (3)."""
    g = np.random.default_rng(13)
    K, G = 3, (2, 3)
    lay = O.make_layout(9, 10, K, 1, 1, 0)
    psfs = g.uniform(0.2, 1.0, G + (K, K))
    psfs /= psfs.sum(axis=(2, 3), keepdims=True)
    wr, wc = O.bilinear_weights(lay.nx[0], G[0]), O.bilinear_weights(lay.nx[1], G[1])
    y = O.apply_H(g.uniform(0, 1, lay.nx), psfs, wr, wc) + 0.01 * g.standard_normal((9, 10))
    lam, delta = 0.03, 0.2
    ref, _ = _consensus_minimiser(lay, psfs, wr, wc, y, lam, delta)
    xhat, info = O.solve(y, psfs, lay, lam, delta, gamma=0.05, rho=1.0, n_outer=30, n_inner=100,
                         inner_increment=10)
    np.testing.assert_allclose(info.us[0], info.xs[0], atol=1e-14)
    np.testing.assert_allclose(xhat, ref, atol=1e-7)


# --------------------------------------------------------------------------- residuals


def test_dual_and_primal_residuals_golden(golden_dir):
    """Two outer iterations of Algorithm 1 derived by hand (one tile, H = I,
    no prior): iterates, duals and both residuals of the oracle's solve."""
    d = json.load(open(os.path.join(golden_dir, "dual_residual_two_iterations.json")))
    y = np.array(d["y"], dtype=float)
    lay = O.make_layout(y.shape[0], y.shape[1], 1, 1, 1, 0)
    psfs = np.ones((1, 1, 1, 1))
    assert abs(O.tile_step(lay, 0, 0, psfs, None, d["lambda"], d["gamma"]) - d["tau"]) <= 1e-15
    for k in (1, 2):
        _, info = O.solve(y, psfs, lay, d["lambda"], 1.0 / 60.0, d["gamma"], d["rho"], k, 1,
                          x0=np.array(d["x0"], dtype=float))
        np.testing.assert_allclose(info.xs[0], d["x"][k - 1], atol=1e-15)
        np.testing.assert_allclose(info.us[0], d["u"][k - 1], atol=1e-15)
        np.testing.assert_allclose(info.primal, d["primal"][:k], atol=1e-15)
        np.testing.assert_allclose(info.dual, d["dual"][:k], atol=1e-15)


def test_dual_residual_alpha_metric_reading():
    """Reading of the dual residual: the unweighted ||zbar^k - zbar^(k-1)||
    the oracle reports times rho sqrt(gamma) is the product-space norm
    rho ||zbar^k - zbar^(k-1)||_alpha summed over the tiles, because
    sum_i alpha_i(l) = gamma sum_i omega_i(l) = gamma at every x pixel."""
    from paper_1705_06603_gb300.synth import WORKLOADS
    w = WORKLOADS["disks128"]
    lay = O.make_layout(w.hy, w.wy, w.K, *w.n_tiles, w.overlap, w.yrows, w.ycols)
    g = np.random.default_rng(11)
    dz = g.standard_normal(lay.nx)
    gamma, rho = 0.4, 1.7
    prod = sum(np.sum(gamma * lay.omega(tr, tc) * dz[lay.xslice(tr, tc)] ** 2)
               for tr, tc in lay.tiles)
    assert abs(rho * np.sqrt(prod) - rho * np.sqrt(gamma) * np.linalg.norm(dz)) <= \
        1e-12 * rho * np.sqrt(gamma) * np.linalg.norm(dz)
