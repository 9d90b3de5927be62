"""Full-size operator parity for the two largest workloads: the 8254^2-pixel
x grid with a 16 x 16 grid of 63 x 63 Moffat PSFs and uneven 9 x 9 tiles, and
the 32830^2-pixel (1.08 Gpixel) grid with 32 x 32 Moffat + Airy PSFs and
uneven 36 x 36 tiles.  H and H^T run over the whole image on the FP32 block-FFT
path and on the tensor-core path; the FP64 oracle recomputes seeded sampled
output pixels one K x K window at a time.  Inputs are a constant background
plus seeded point sources, built on the device from host-drawn coordinates, so
neither side needs a host copy of the image."""

import numpy as np
import pytest

from oracle import dv_oracle as O
from tests.gpu_common import assert_close, need_gpu

pytestmark = pytest.mark.gpu

FFT, TENSOR = 2, 3
FP32, TF32, BF16 = 0, 1, 2
TOL = {FP32: 1e-5, TF32: 5e-4, BF16: 3e-3}
BACKGROUND = 0.01


def _points(shape, n, seed):
    g = np.random.default_rng(seed)
    r = g.integers(0, shape[0], n)
    c = g.integers(0, shape[1], n)
    v = g.uniform(0.05, 1.0, n)
    return r, c, v


class _Sparse:
    """Background + point sources; slicing [r0:r1, c0:c1] gives a dense FP64
    window (zero outside the image), for the oracle's per-window sums."""

    def __init__(self, shape, pts):
        self.shape = shape
        self.r, self.c, self.v = pts

    def __getitem__(self, idx):
        rs, cs = idx
        r0, r1, c0, c1 = rs.start, rs.stop, cs.start, cs.stop
        win = np.zeros((r1 - r0, c1 - c0))
        rr0, rr1 = max(r0, 0), min(r1, self.shape[0])
        cc0, cc1 = max(c0, 0), min(c1, self.shape[1])
        win[rr0 - r0:rr1 - r0, cc0 - c0:cc1 - c0] = BACKGROUND
        m = (self.r >= rr0) & (self.r < rr1) & (self.c >= cc0) & (self.c < cc1)
        # float32 values, as on the device
        win[self.r[m] - r0, self.c[m] - c0] = self.v[m].astype(np.float32).astype(np.float64)
        return win


def _device_image(torch, shape, pts):
    x = torch.full(shape, BACKGROUND, dtype=torch.float32, device="cuda")
    r, c, v = pts
    x[torch.from_numpy(r).cuda(), torch.from_numpy(c).cuda()] = torch.from_numpy(
        v.astype(np.float32)).cuda()
    return x


def _check(name, path, prec, n_samples=256, strip=256):
    torch, dv = need_gpu()
    from paper_1705_06603_gb300.synth import WORKLOADS, psf_grid_for
    w = WORKLOADS[name]
    K = w.K
    psfs = psf_grid_for(w).astype(np.float32)
    ps = psfs.astype(np.float64)
    nxr, nxc = w.nx
    plan = dv.Plan(w.hy, w.wy, psfs, n_tiles=w.n_tiles, overlap=w.overlap,
                   tile_bounds=(w.yrows, w.ycols), n_outer=0, n_inner=0, path=path,
                   precision=prec)
    assert plan.info.path == path
    n_pts = max(1000, (nxr * nxc) // 5000)
    xs = _Sparse((nxr, nxc), _points((nxr, nxc), n_pts, 11))
    rs = _Sparse((w.hy, w.wy), _points((w.hy, w.wy), n_pts, 12))
    y = plan.apply_H(_device_image(torch, (nxr, nxc), (xs.r, xs.c, xs.v)))
    g = plan.apply_Ht(_device_image(torch, (w.hy, w.wy), (rs.r, rs.c, rs.v)))
    torch.cuda.synchronize()
    wr = O.bilinear_weights(nxr, w.grid[0])
    wc = O.bilinear_weights(nxc, w.grid[1])
    sg = np.random.default_rng(13)
    # sampled y pixels (corners and block edges included) and a contiguous
    # strip of one row across the first tile boundary (block and band edges)
    b0 = w.yrows[1][0] if w.yrows is not None else w.wy // 2
    sj = np.arange(max(0, b0 - strip // 2), min(w.wy, b0 + strip // 2))
    pi = np.concatenate([[0, w.hy - 1, w.hy // 2], sg.integers(0, w.hy, n_samples),
                         np.full(sj.size, w.hy // 2 + 1)])
    pj = np.concatenate([[0, w.wy - 1, w.wy // 3], sg.integers(0, w.wy, n_samples), sj])
    got, ref = [], []
    for i, j in zip(pi, pj):
        win = xs[i:i + K, j:j + K]
        ref.append(O.apply_H_at(win, ps, wr[:, i:i + K], wc[:, j:j + K], [(0, 0)])[0])
        got.append(float(y[i, j]))
    got, ref = np.array(got), np.array(ref)
    assert_close(got, ref, TOL[prec])
    # sampled x pixels of H^T, and a strip of one x row across the first
    # tile boundary
    sC = np.arange(max(0, b0 - strip // 2), min(nxc, b0 + strip // 2 + K))
    pR = np.concatenate([[0, nxr - 1, nxr // 2], sg.integers(0, nxr, n_samples),
                         np.full(sC.size, nxr // 2 - 1)])
    pC = np.concatenate([[0, nxc - 1, nxc // 3], sg.integers(0, nxc, n_samples), sC])
    got, ref = [], []
    for R, C in zip(pR, pC):
        win = rs[R - K + 1:R + 1, C - K + 1:C + 1]
        wrs = np.zeros((w.grid[0], 2 * K - 1))
        wcs = np.zeros((w.grid[1], 2 * K - 1))
        wrs[:, K - 1] = wr[:, R]
        wcs[:, K - 1] = wc[:, C]
        ref.append(O.apply_Ht_at(win, ps, wrs, wcs, [(K - 1, K - 1)])[0])
        got.append(float(g[R, C]))
    got, ref = np.array(got), np.array(ref)
    assert_close(got, ref, TOL[prec])
    plan.close()


@pytest.mark.parametrize("path,prec", [(FFT, FP32), (TENSOR, BF16), (TENSOR, TF32)])
def test_wide8192_operator_sampled(path, prec):
    _check("wide8192", path, prec)


@pytest.mark.parametrize("path,prec", [(FFT, FP32), (TENSOR, BF16)])
def test_giga32768_operator_sampled(path, prec):
    _check("giga32768", path, prec)
