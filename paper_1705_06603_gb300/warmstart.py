"""Training driver of the learned warm start.

The network learns the correction from the observed image to the image the
plain method converges to: pairs (features, x_hat - y_pad) are produced by the
library itself (dv_consensus_solve from the blurred-image start) on seeded
synthetic scenes with randomly drawn Moffat PSF grids and noise levels, then
the network is trained with Adam on random crops (dv_cnn_train_step).  Every
step runs in libdv; this module only draws inputs and moves tensors.
"""

from __future__ import annotations

import numpy as np

from . import dv
from .synth import gaussian_noise, moffat_psf_grid, rng, star_field


def random_case(seed, size, K, grid):
    """A seeded scene (star field), Moffat PSF grid with random width / shape
    ranges, and noise level."""
    g = rng(10_000 + seed)
    nx = size + K - 1
    x = star_field((nx, nx), seed, star_density=g.uniform(5e-4, 3e-3),
                   blob_density=g.uniform(5e-5, 4e-4))
    psfs = moffat_psf_grid(grid[0], grid[1], K, fwhm_center=g.uniform(1.5, 3.0),
                           fwhm_corner=g.uniform(3.0, 5.5), beta_center=g.uniform(3.0, 4.5),
                           beta_corner=g.uniform(2.2, 3.2)).astype(np.float32)
    sigma = float(g.uniform(0.003, 0.01))
    return x, psfs, sigma


def make_pair(seed, size=96, K=15, grid=(3, 3), n_tiles=(2, 2), overlap=16, n_outer=40,
              n_inner=10, lam=1e-3, delta=1.0 / 60.0, gamma=0.4, psfs=None, sigma=None):
    """(features [nx, nx, 5], target [nx, nx], y, psfs, sigma) of one seeded case
    (CUDA tensors); psfs / sigma, when given, replace the random draws."""
    import torch
    x, rpsfs, rsigma = random_case(seed, size, K, grid)
    psfs = rpsfs if psfs is None else np.ascontiguousarray(psfs, dtype=np.float32)
    sigma = rsigma if sigma is None else float(sigma)
    plan = dv.Plan(size, size, psfs, n_tiles=n_tiles, overlap=overlap, lam=lam, delta=delta,
                   gamma=gamma, n_outer=n_outer, n_inner=n_inner, noise_sigma=sigma)
    y = plan.apply_H(torch.from_numpy(x).cuda())
    y += torch.from_numpy(gaussian_noise(y.shape, sigma, 20_000 + seed, np.float32)).cuda()
    xhat, _ = plan.solve(y, stats=False)
    feat = torch.empty(plan.nx + (dv.CNN_IN_CH,), device="cuda")
    dv.dv_warmstart_features(plan.handle, y, feat)
    torch.cuda.synchronize()
    plan.close()
    return feat, xhat - feat[..., 0], y, psfs, sigma


def train(cnn, pairs, steps, batch=8, crop=64, lr=1e-3, seed=0, log_every=0):
    """Adam on random crops of the pairs; returns the loss history."""
    import torch
    g = rng(30_000 + seed)
    losses = []
    for it in range(steps):
        xs, ts = [], []
        for _ in range(batch):
            f, t = pairs[int(g.integers(len(pairs)))]
            H, W = t.shape
            r0 = int(g.integers(0, H - crop + 1))
            c0 = int(g.integers(0, W - crop + 1))
            xs.append(f[r0:r0 + crop, c0:c0 + crop])
            ts.append(t[r0:r0 + crop, c0:c0 + crop])
        xb = torch.stack(xs).contiguous()
        tb = torch.stack(ts).contiguous()
        losses.append(cnn.train_step(xb, tb, lr))
        if log_every and (it + 1) % log_every == 0:
            print(f"step {it + 1}: loss {np.mean(losses[-log_every:]):.3e}")
    return losses
