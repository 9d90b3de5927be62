"""Shared helpers of the GPU tests: problem builders on seeded synthetic inputs
and comparison metrics.  Expected values always come from the oracle."""

import numpy as np
import pytest

from oracle import dv_oracle as O
from paper_1705_06603_gb300.synth import WORKLOADS, psf_grid_for, scene_for, gaussian_noise


def need_gpu():
    import torch
    if not torch.cuda.is_available():
        pytest.fail("this test needs a CUDA GPU")
    from paper_1705_06603_gb300 import build
    build.build()
    from paper_1705_06603_gb300 import dv
    return torch, dv


def rel_l2(a, b):
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


def rel_rmse(a, b):
    return rel_l2(a, b)


def random_psfs(g, G, K, negative=False):
    p = g.uniform(-0.3 if negative else 0.0, 1.0, G + (K, K))
    if not negative:
        p /= p.sum(axis=(2, 3), keepdims=True)
    return p.astype(np.float32)


def workload_case(name, n_outer=None, n_inner=None):
    """Observed image of a named workload: y = H x_true + noise with the
    oracle's operator (so no CUDA output feeds the oracle)."""
    w = WORKLOADS[name]
    psfs = psf_grid_for(w).astype(np.float32)
    x = scene_for(w)
    nxr, nxc = w.nx
    wr, wc = O.bilinear_weights(nxr, w.grid[0]), O.bilinear_weights(nxc, w.grid[1])
    y = O.apply_H(x, psfs.astype(np.float64), wr, wc)
    y = (y + gaussian_noise(y.shape, w.noise_sigma, w.noise_seed)).astype(np.float32)
    return w, psfs, y, x


def oracle_solve(w, psfs, y, n_outer, n_inner, **kw):
    lay = O.make_layout(w.hy, w.wy, w.K, *w.n_tiles, w.overlap, w.yrows, w.ycols)
    xhat, info = O.solve(y.astype(np.float64), psfs.astype(np.float64), lay, w.lam, w.delta,
                         w.gamma, w.rho, n_outer, n_inner, **kw)
    return lay, xhat, info


def max_abs_err(a, b):
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    return float(np.max(np.abs(a - b))) if a.size else 0.0


def assert_close(a, b, tol):
    """The GPU result a against the oracle's b: relative L2 error <= tol, and
    element by element |a - b| <= 10 tol max|b| (a wrong row, column or block
    edge that a norm over the whole image would dilute fails the second)."""
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    assert a.shape == b.shape, (a.shape, b.shape)
    e = rel_l2(a, b)
    assert e <= tol, f"relative L2 error {e:.3e} > {tol:.1e}"
    scale = float(np.max(np.abs(b))) if b.size else 0.0
    m = max_abs_err(a, b)
    assert m <= 10.0 * tol * scale, (f"max |error| {m:.3e} > 10 x {tol:.1e} x max|ref| "
                                     f"({scale:.3e}) at {np.unravel_index(np.argmax(np.abs(a - b)), a.shape)}")
