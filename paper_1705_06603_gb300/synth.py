"""Seeded synthetic inputs: scenes, PSF grids, noise draws and workload shapes.

This module holds none of the deblurring method's arithmetic (no blur operator,
no prior, no solver).  It only draws the inputs that both the CUDA path and the
FP64 oracle consume, so that the two can be compared on identical data.  All
randomness comes from numpy's PCG64 generator seeded explicitly.

The paper evaluates on named photographs (resized and rescaled to 6000
photons/pixel) that are not available here; these generators stand in for them
with sky-like scenes of the same sizes and structure:

  * disks_and_points ... small scene of flat disks and point sources in [0, 1]
  * star_field ......... Poisson-placed stars with power-law fluxes (pdf ~ F^-2)
                         plus elliptical Gaussian blobs on a constant background
  * gaussian/moffat/airy PSF grids whose width grows radially across the field,
    like the radially increasing Gaussian FWHM of the paper's shift-variant
    experiments (Sec. IV).
"""

from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np


def rng(seed: int) -> np.random.Generator:
    return np.random.Generator(np.random.PCG64(seed))


# ---------------------------------------------------------------------------
# Scenes
# ---------------------------------------------------------------------------


def disks_and_points(shape, seed, n_disks=24, n_points=32, r_lo=3.0, r_hi=15.0):
    """Flat disks (radius U[r_lo, r_hi], value U[0.2, 1], max-composited) plus
    single-pixel point sources U[0.5, 1], clipped to [0, 1]."""
    g = rng(seed)
    H, W = shape
    img = np.zeros(shape)
    rr, cc = np.mgrid[0:H, 0:W]
    for _ in range(n_disks):
        r0, c0 = g.uniform(0, H), g.uniform(0, W)
        rad, val = g.uniform(r_lo, r_hi), g.uniform(0.2, 1.0)
        mask = (rr - r0) ** 2 + (cc - c0) ** 2 <= rad * rad
        img[mask] = np.maximum(img[mask], val)
    pr = g.integers(0, H, n_points)
    pc = g.integers(0, W, n_points)
    pv = g.uniform(0.5, 1.0, n_points)
    img[pr, pc] = np.maximum(img[pr, pc], pv)
    return np.clip(img, 0.0, 1.0)


def star_field(shape, seed, star_density=1e-3, flux_lo=0.01, flux_hi=1.0,
               blob_density=2e-5, background=0.01, dtype=np.float32):
    """Stars: Poisson count (density per pixel), uniform positions, fluxes by
    inverse CDF of pdf ~ F^-2 on [flux_lo, flux_hi].  Blobs: elliptical Gaussians
    (amplitude U[0.05, 0.3], major sigma U[3, 30], axis ratio U[0.3, 1],
    angle U[0, pi)).  Constant background; normalised to peak 1."""
    g = rng(seed)
    H, W = shape
    img = np.full(shape, background, dtype=np.float64)
    n_stars = g.poisson(star_density * H * W)
    u = g.uniform(0.0, 1.0, n_stars)
    flux = 1.0 / (1.0 / flux_lo - u * (1.0 / flux_lo - 1.0 / flux_hi))
    sr = g.integers(0, H, n_stars)
    sc = g.integers(0, W, n_stars)
    np.add.at(img, (sr, sc), flux)
    n_blobs = g.poisson(blob_density * H * W)
    for _ in range(n_blobs):
        amp = g.uniform(0.05, 0.3)
        smaj = g.uniform(3.0, 30.0)
        smin = smaj * g.uniform(0.3, 1.0)
        th = g.uniform(0.0, np.pi)
        r0, c0 = g.uniform(0, H), g.uniform(0, W)
        ext = int(np.ceil(4 * smaj))
        ra, rb = max(0, int(r0) - ext), min(H, int(r0) + ext + 1)
        ca, cb = max(0, int(c0) - ext), min(W, int(c0) + ext + 1)
        if ra >= rb or ca >= cb:
            continue
        dr = np.arange(ra, rb)[:, None] - r0
        dc = np.arange(ca, cb)[None, :] - c0
        p = dr * np.cos(th) + dc * np.sin(th)
        q = -dr * np.sin(th) + dc * np.cos(th)
        img[ra:rb, ca:cb] += amp * np.exp(-0.5 * ((p / smaj) ** 2 + (q / smin) ** 2))
    img /= img.max()
    return img.astype(dtype)


# ---------------------------------------------------------------------------
# PSF grids (each PSF normalised to unit sum, centred in a K x K array)
# ---------------------------------------------------------------------------


def _radial_position(Gr, Gc):
    """Distance of each grid point from the field centre, 0 at the centre and 1
    at the corners."""
    a = np.zeros(Gr) if Gr == 1 else np.arange(Gr) / (Gr - 1) - 0.5
    b = np.zeros(Gc) if Gc == 1 else np.arange(Gc) / (Gc - 1) - 0.5
    return np.sqrt(a[:, None] ** 2 + b[None, :] ** 2) / np.sqrt(0.5)


def _kernel_coords(K):
    c = np.arange(K) - K // 2
    return c[:, None].astype(np.float64), c[None, :].astype(np.float64)


def gaussian_psf_grid(Gr, Gc, K, sigma_center, sigma_corner):
    rad = _radial_position(Gr, Gc)
    yy, xx = _kernel_coords(K)
    out = np.empty((Gr, Gc, K, K))
    for a in range(Gr):
        for b in range(Gc):
            s = sigma_center + (sigma_corner - sigma_center) * rad[a, b]
            h = np.exp(-0.5 * (yy * yy + xx * xx) / (s * s))
            out[a, b] = h / h.sum()
    return out


def moffat_psf(K, fwhm, beta):
    yy, xx = _kernel_coords(K)
    alpha = fwhm / (2.0 * np.sqrt(2.0 ** (1.0 / beta) - 1.0))
    h = (1.0 + (yy * yy + xx * xx) / (alpha * alpha)) ** (-beta)
    return h / h.sum()


def airy_psf(K, core_px=2.5, oversample=4):
    """|FFT(circular pupil)|^2 resampled to K x K (first dark ring near core_px)."""
    N = oversample * K
    N += N % 2
    yy, xx = np.mgrid[0:N, 0:N] - N // 2
    # first zero of the Airy pattern at 1.22 N / D pixels for a pupil of diameter D
    D = 1.22 * N / core_px
    pupil = (yy * yy + xx * xx) <= (D / 2) ** 2
    psf = np.abs(np.fft.fftshift(np.fft.fft2(np.fft.ifftshift(pupil)))) ** 2
    c = N // 2
    h = psf[c - K // 2:c + K // 2 + 1, c - K // 2:c + K // 2 + 1]
    return h / h.sum()


def moffat_psf_grid(Gr, Gc, K, fwhm_center=2.0, fwhm_corner=5.0, beta_center=4.5,
                    beta_corner=2.5, airy_fraction=0.0):
    rad = _radial_position(Gr, Gc)
    airy = airy_psf(K) if airy_fraction > 0 else None
    out = np.empty((Gr, Gc, K, K))
    for a in range(Gr):
        for b in range(Gc):
            t = rad[a, b]
            h = moffat_psf(K, fwhm_center + (fwhm_corner - fwhm_center) * t,
                           beta_center + (beta_corner - beta_center) * t)
            if airy is not None:
                h = (1.0 - airy_fraction) * h + airy_fraction * airy
            out[a, b] = h / h.sum()
    return out


# ---------------------------------------------------------------------------
# Noise draws (applied by the caller to its blurred image)
# ---------------------------------------------------------------------------


def gaussian_noise(shape, sigma, seed, dtype=np.float64):
    return (sigma * rng(seed).standard_normal(shape)).astype(dtype)


def poisson_gaussian(blurred, peak, sigma, seed):
    """Poisson(peak * max(b, 0)) / peak + N(0, sigma^2), and the per-pixel
    inverse-variance weights normalised to (0, 1]: W = sigma^2 / (b/peak + sigma^2)."""
    g = rng(seed)
    b = np.maximum(np.asarray(blurred, dtype=np.float64), 0.0)
    y = g.poisson(peak * b) / peak + sigma * g.standard_normal(b.shape)
    var = np.maximum(y, 0.0) / peak + sigma * sigma
    return y, (sigma * sigma) / var


# ---------------------------------------------------------------------------
# Workload shapes (sizes, PSF grids, tilings, parameters)
# ---------------------------------------------------------------------------


@dataclass
class Workload:
    name: str
    hy: int
    wy: int
    K: int
    grid: tuple
    n_tiles: tuple
    overlap: int
    lam: float = 1e-3
    delta: float = 1.0 / 60.0
    gamma: float = 0.4
    rho: float = 1.0
    n_outer: int = 30
    n_inner: int = 10
    noise_sigma: float = 0.01
    poisson_peak: float = 0.0
    yrows: list | None = None
    ycols: list | None = None
    scene_seed: int = 0
    noise_seed: int = 1
    extra: dict = field(default_factory=dict)

    @property
    def nx(self):
        return self.hy + self.K - 1, self.wy + self.K - 1


def _uneven(n_interior, interior, boundary, overlap):
    """y-block bounds: boundary block, n_interior interior blocks, boundary block."""
    sizes = [boundary] + [interior] * n_interior + [boundary]
    out, s = [], 0
    for sz in sizes:
        out.append((s, s + sz))
        s += sz - overlap
    return out


WORKLOADS = {
    # 128x128 disks + points, 3x3 Gaussian 9x9 PSFs, 2x2 tiles / 16 px, 30 x 10
    "disks128": Workload("disks128", 128, 128, 9, (3, 3), (2, 2), 16,
                         noise_sigma=0.01, n_outer=30, n_inner=10,
                         extra={"psf": ("gaussian", 0.8, 2.0)}),
    # 2048x2048 star field, 8x8 Moffat 31x31, 4x4 tiles / 64 px, 100 x 10
    "stars2048": Workload("stars2048", 2048, 2048, 31, (8, 8), (4, 4), 64,
                          noise_sigma=0.005, n_outer=100, n_inner=10,
                          scene_seed=2, noise_seed=3, extra={"psf": ("moffat", 0.0)}),
    # 8192x8192, 16x16 Moffat 63x63, uneven 9x9 tiles (7 x 1024 + 2 x 768) / 64 px
    "wide8192": Workload("wide8192", 8192, 8192, 63, (16, 16), (9, 9), 64,
                         noise_sigma=2e-3, poisson_peak=1e4, n_outer=100, n_inner=10,
                         yrows=_uneven(7, 1024, 768, 64), ycols=_uneven(7, 1024, 768, 64),
                         scene_seed=4, noise_seed=5, extra={"psf": ("moffat", 0.0)}),
    # 32768x32768, 32x32 Moffat + 5% Airy 63x63, 36x36 tiles (34 x 1024 + 2 x 656) / 96 px
    "giga32768": Workload("giga32768", 32768, 32768, 63, (32, 32), (36, 36), 96,
                          noise_sigma=2e-3, poisson_peak=1e4, n_outer=200, n_inner=10,
                          yrows=_uneven(34, 1024, 656, 96), ycols=_uneven(34, 1024, 656, 96),
                          scene_seed=6, noise_seed=7, extra={"psf": ("moffat", 0.05)}),
}


def psf_grid_for(wl: Workload):
    kind = wl.extra.get("psf", ("gaussian", 0.8, 2.0))
    Gr, Gc = wl.grid
    if kind[0] == "gaussian":
        return gaussian_psf_grid(Gr, Gc, wl.K, kind[1], kind[2])
    return moffat_psf_grid(Gr, Gc, wl.K, airy_fraction=kind[1])


def scene_for(wl: Workload, dtype=np.float64):
    if wl.name.startswith("disks"):
        return disks_and_points(wl.nx, wl.scene_seed).astype(dtype)
    return star_field(wl.nx, wl.scene_seed, dtype=dtype)
