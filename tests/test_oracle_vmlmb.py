"""Pins of the oracle's VMLM-B Local-Solver (reading R20, Sec. IV-B): its
first iteration is exactly one projected-gradient step, every accepted step
decreases the prox objective and keeps w >= 0, it reaches the L-BFGS-B
minimiser of Phi_i computed with dense matrices, faster than projected
gradient, and Algorithm 1 with it reaches the brute-force consensus
minimiser like the projected-gradient version."""

import numpy as np

from oracle import dv_oracle as O
from tests.oracle_helpers import dense_D, dense_H, huber_terms, lbfgsb_min
from tests.test_oracle_prior_solver import _consensus_minimiser, _tiny_problem


def _tile(seed, lam=0.02, delta=0.3, gamma=1.0):
    lay, psfs, wr, wc, y = _tiny_problem(seed)
    tr, tc = 0, 1
    wri, wci = O.tile_weights(lay, tr, tc, wr, wc)
    yi = y[lay.yslice(tr, tc)]
    shape = (wri.shape[1], wci.shape[1])
    g = np.random.default_rng(seed + 1)
    u = g.uniform(-0.2, 1, shape)
    al = gamma * lay.omega(tr, tc)
    tau = O.tile_step(lay, tr, tc, psfs, None, lam, gamma)
    return lay, psfs, wri, wci, yi, u, al, tau, lam, delta, shape


def test_first_iteration_is_the_projected_gradient_step():
    lay, psfs, wri, wci, yi, u, al, tau, lam, delta, _ = _tile(9)
    w0 = np.maximum(u, 0.0)
    a = O.local_solve_vmlmb(w0, u, yi, None, psfs, wri, wci, al, lam, delta, tau, 1)
    b = O.local_solve(w0, u, yi, None, psfs, wri, wci, al, lam, delta, tau, 1)
    np.testing.assert_allclose(a, b, rtol=0, atol=0)


def test_vmlmb_decreases_and_stays_feasible():
    lay, psfs, wri, wci, yi, u, al, tau, lam, delta, _ = _tile(13, lam=0.05, delta=0.05)
    w = np.maximum(u, 0.0)
    prev = O.prox_objective(w, u, yi, None, psfs, wri, wci, al, lam, delta)
    for _ in range(15):
        w = O.local_solve_vmlmb(w, u, yi, None, psfs, wri, wci, al, lam, delta, tau, 2)
        cur = O.prox_objective(w, u, yi, None, psfs, wri, wci, al, lam, delta)
        assert cur <= prev + 1e-13 * abs(prev)
        assert w.min() >= 0.0
        prev = cur


def test_vmlmb_reaches_prox_minimiser_faster_than_pg():
    lay, psfs, wri, wci, yi, u, al, tau, lam, delta, shape = _tile(9)
    M = dense_H(psfs, wri, wci)
    Dr, Dc = dense_D(*shape)

    def fg(v):
        r = M @ v - yi.ravel()
        hv, hg = huber_terms(Dr, Dc, v, delta)
        d = v - u.ravel()
        return (0.5 * r @ r + lam * hv + 0.5 * np.sum(al.ravel() * d * d),
                M.T @ r + lam * hg + al.ravel() * d)

    ref = lbfgsb_min(fg, np.maximum(u.ravel(), 0))
    fref = fg(ref)[0]
    w0 = np.maximum(u, 0.0)
    vm = O.local_solve_vmlmb(w0, u, yi, None, psfs, wri, wci, al, lam, delta, tau, 200)
    np.testing.assert_allclose(vm.ravel(), ref, atol=2e-6)
    n = 40
    gap_vm = fg(O.local_solve_vmlmb(w0, u, yi, None, psfs, wri, wci, al, lam, delta, tau, n)
                .ravel())[0] - fref
    gap_pg = fg(O.local_solve(w0, u, yi, None, psfs, wri, wci, al, lam, delta, tau, n)
                .ravel())[0] - fref
    assert gap_vm < 0.1 * gap_pg


def test_algorithm1_with_vmlmb_reaches_consensus_minimiser():
    lay, psfs, wr, wc, y = _tiny_problem(12)
    lam, delta = 0.02, 10.0
    ref, fg = _consensus_minimiser(lay, psfs, wr, wc, y, lam, delta)
    xhat, _ = O.solve(y, psfs, lay, lam, delta, gamma=0.5, rho=1.0, n_outer=60, n_inner=15,
                      local_solver="vmlmb", vm_memory=5)
    Fs = fg(ref.ravel())[0]
    assert (fg(xhat.ravel())[0] - Fs) / Fs <= 1e-5
    assert np.abs(xhat - ref).max() <= 3e-3


def test_stop_at_objective_resolution_lands_at_the_minimiser():
    """Reading R21: a tile ends its VMLM-B solve once -g'd <= stop_rel |Phi|.
    For a quasi-Newton direction -g'd is about twice the remaining gap, so the
    stopped iterate lies within a few stop_rel |Phi| of the dense L-BFGS-B
    minimiser's objective; the stop fires (well before the iteration budget)
    and, until it does, the solve is the plain VMLM-B."""
    lay, psfs, wri, wci, yi, u, al, tau, lam, delta, shape = _tile(9)
    M = dense_H(psfs, wri, wci)
    Dr, Dc = dense_D(*shape)

    def fg(v):
        r = M @ v - yi.ravel()
        hv, hg = huber_terms(Dr, Dc, v, delta)
        d = v - u.ravel()
        return (0.5 * r @ r + lam * hv + 0.5 * np.sum(al.ravel() * d * d),
                M.T @ r + lam * hg + al.ravel() * d)

    ref = lbfgsb_min(fg, np.maximum(u.ravel(), 0))
    fref = fg(ref)[0]
    w0 = np.maximum(u, 0.0)
    for eta in (1e-4, 1e-7):
        st = {}
        vm = O.local_solve_vmlmb(w0, u, yi, None, psfs, wri, wci, al, lam, delta, tau, 400,
                                 stop_rel=eta, stats=st)
        k = st["stopped_at"]
        assert k is not None and k < 400
        assert len(st["trials"]) == k
        assert 0.0 <= fg(vm.ravel())[0] - fref <= 5.0 * eta * abs(fref)
        # identical to the unstopped solve run for the same number of iterations
        same = O.local_solve_vmlmb(w0, u, yi, None, psfs, wri, wci, al, lam, delta, tau, k)
        np.testing.assert_array_equal(vm, same)
    st = {}
    O.local_solve_vmlmb(w0, u, yi, None, psfs, wri, wci, al, lam, delta, tau, 30, stats=st)
    assert st["stopped_at"] is None and len(st["trials"]) == 30
    # the exact (FP64) line search accepts the first trial almost always
    assert np.mean(st["trials"]) <= 1.5
