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
from .synth import gaussian_noise, moffat_psf_grid, poisson_gaussian, rng, star_field


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
              n_inner=10, lam=1e-3, delta=1.0 / 60.0, gamma=0.4, psfs=None, sigma=None,
              poisson_peak=0.0):
    """(features [nx, nx, 5], target [nx, nx], y, psfs, sigma) of one seeded case
    (CUDA tensors); psfs / sigma, when given, replace the random draws.  With
    poisson_peak > 0 the noise is Poisson(peak H x) / peak + N(0, sigma^2) and the
    solve weighs the data term with the per-pixel inverse-variance weights."""
    import torch
    x, rpsfs, rsigma = random_case(seed, size, K, grid)
    psfs = rpsfs if psfs is None else np.ascontiguousarray(psfs, dtype=np.float32)
    sigma = rsigma if sigma is None else float(sigma)
    kw = dict(n_tiles=n_tiles, overlap=overlap, lam=lam, delta=delta, gamma=gamma,
              n_outer=n_outer, n_inner=n_inner, noise_sigma=sigma)
    plan = dv.Plan(size, size, psfs, **kw)
    y = plan.apply_H(torch.from_numpy(x).cuda())
    if poisson_peak > 0:
        yb, W = poisson_gaussian(y.cpu().numpy(), poisson_peak, sigma, 20_000 + seed)
        y.copy_(torch.from_numpy(yb.astype(np.float32)))
        plan.close()
        plan = dv.Plan(size, size, psfs, noise_w=W.astype(np.float32), **kw)
    else:
        y += torch.from_numpy(gaussian_noise(y.shape, sigma, 20_000 + seed, np.float32)).cuda()
    xhat, _ = plan.solve(y, stats=False)
    feat = torch.empty(plan.nx + (dv.CNN_IN_CH,), device="cuda")
    dv.dv_warmstart_features(plan.handle, y, feat)
    torch.cuda.synchronize()
    plan.close()
    return feat, xhat - feat[..., 0], y, psfs, sigma


def train(cnn, pairs, steps, batch=8, crop=64, lr=1e-3, seed=0, log_every=0, schedule="const",
          chunk=4000):
    """Adam on random crops of the pairs; returns the loss history.  schedule:
    "const" keeps lr; "cosine" anneals it as lr (1 + cos(pi t / steps)) / 2.
    The crop table is drawn on the host (pair, then row, then column per crop)
    and the steps run inside libdv, `chunk` steps per call."""
    import math
    import torch
    if schedule not in ("const", "cosine"):
        raise ValueError(f"unknown schedule {schedule!r}")
    H, W = pairs[0][1].shape
    if any(t.shape != (H, W) for _, t in pairs):
        raise ValueError("training pairs must share one size")
    feats = torch.stack([f for f, _ in pairs]).contiguous()
    targets = torch.stack([t for _, t in pairs]).contiguous()
    g = rng(30_000 + seed)
    crops = np.empty((steps, batch, 3), dtype=np.int32)
    for it in range(steps):
        for b in range(batch):
            crops[it, b, 0] = int(g.integers(len(pairs)))
            crops[it, b, 1] = int(g.integers(0, H - crop + 1))
            crops[it, b, 2] = int(g.integers(0, W - crop + 1))
    t = np.arange(steps)
    lrs = (np.full(steps, lr) if schedule == "const"
           else 0.5 * lr * (1.0 + np.cos(math.pi * t / max(steps, 1))))
    lrs = np.maximum(lrs, 1e-3 * lr).astype(np.float32)
    losses = []
    for s0 in range(0, steps, chunk):
        s1 = min(steps, s0 + chunk)
        losses.extend(cnn.train_crops(feats, targets, crops[s0:s1], crop, lrs[s0:s1]).tolist())
        if log_every:
            print(f"step {s1}: loss {np.mean(losses[-log_every:]):.3e}")
    return losses
