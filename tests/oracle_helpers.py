"""Independent references used to pin the oracle: dense operators assembled with
scipy's convolution routines, and brute-force minimisers from scipy.optimize.
Nothing here calls the CUDA path."""

import numpy as np
from scipy.optimize import minimize
from scipy.signal import convolve2d


def dense_H(psfs, wr, wc):
    """Matrix of the shift-variant operator, column j = sum_p convolve2d(w_p . e_j, h_p, 'valid')."""
    Gr, Gc, K, _ = psfs.shape
    nxr, nxc = wr.shape[1], wc.shape[1]
    ny, nx = nxr - K + 1, nxc - K + 1
    M = np.zeros((ny * nx, nxr * nxc))
    for j in range(nxr * nxc):
        e = np.zeros(nxr * nxc)
        e[j] = 1.0
        e = e.reshape(nxr, nxc)
        col = np.zeros((ny, nx))
        for a in range(Gr):
            for b in range(Gc):
                col += convolve2d(np.outer(wr[a], wc[b]) * e, psfs[a, b], mode="valid")
        M[:, j] = col.ravel()
    return M


def dense_D(nr, nc):
    """Forward differences with zero on the last row / column, as two matrices."""
    n = nr * nc
    Dr = np.zeros((n, n))
    Dc = np.zeros((n, n))
    for i in range(nr):
        for j in range(nc):
            k = i * nc + j
            if i + 1 < nr:
                Dr[k, k + nc], Dr[k, k] = 1.0, -1.0
            if j + 1 < nc:
                Dc[k, k + 1], Dc[k, k] = 1.0, -1.0
    return Dr, Dc


def huber_terms(Dr, Dc, x, delta):
    """Isotropic Huber value and gradient written with dense difference matrices."""
    dr, dc = Dr @ x, Dc @ x
    s = np.sqrt(dr * dr + dc * dc)
    val = np.sum(np.where(s <= delta, 0.5 * s * s, delta * (s - 0.5 * delta)))
    kap = np.where(s <= delta, 1.0, delta / np.where(s > 0, s, 1.0))
    return val, Dr.T @ (kap * dr) + Dc.T @ (kap * dc)


def lbfgsb_min(fun_grad, x0, maxiter=200000):
    res = minimize(fun_grad, x0, jac=True, method="L-BFGS-B",
                   bounds=[(0.0, None)] * x0.size,
                   options={"maxiter": maxiter, "maxfun": maxiter, "ftol": 1e-16, "gtol": 1e-13,
                            "maxcor": 50})
    return res.x
