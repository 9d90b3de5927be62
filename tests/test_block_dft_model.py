"""The block-DFT factorization of H and H^T (the tensor-core kernels' algorithm,
Sec. II-B's sum of PSF-weighted convolutions on 128 x 128 overlap-save blocks)
written out in float64 numpy and checked against the oracle on one block.

This pins the derivation the kernels implement, independent of the GPU: the
packed half spectrum of a real input (A1's rows: real and imaginary parts of
Y(k), k < 64, interleaved, row 1 holding Y(64)); Z(k) from the two GEMMs
Fr Y'^T, Fi Y'^T; the inverse with the mirror half folded in (weight 2 for
k = 1 .. 63) as [Ur | Ui] = Fr [aSr | aSi] + Fi [aSi | -aSr]; for H^T the
conjugate spectra, the row weights summed over the PSF grid rows inside the
last inverse GEMM and the column weight applied to that sum.  No GPU."""

import numpy as np
import pytest

from oracle import dv_oracle as O
from tests.gpu_common import random_psfs

S = 128
TH = 2.0 * np.pi / S
k_ = np.arange(S)
FR = np.cos(TH * np.outer(k_, k_))      # Fr[n][k]
FI = -np.sin(TH * np.outer(k_, k_))     # Fi[n][k]
ALPHA = np.where((np.arange(65) == 0) | (np.arange(65) == 64), 1.0, 2.0)


def a1_matrix():
    """Rows 2m: Fr(m), 2m + 1: Fi(m) for m = 0 .. 63; row 1 (Fi(0) = 0) holds Fr(64)."""
    A = np.empty((S, S))
    A[0::2] = FR[:64]
    A[1::2] = FI[:64]
    A[1] = FR[64]
    return A


def spectrum(h):
    """Hh(kr, kc) = sum_{m,n} h(m, n) exp(-2 pi i (kr m + kc n) / 128), kr = 0 .. 64."""
    hp = np.zeros((S, S))
    hp[:h.shape[0], :h.shape[1]] = h
    return np.fft.fft2(hp)[:65]


def z_of(Yp):
    """Z(k)[kc] for k = 0 .. 64 from Y' (j x c): P = Fr Y'^T, Q = Fi Y'^T (kc x j)."""
    P, Q = FR @ Yp.T, FI @ Yp.T
    Z = np.empty((65, S), complex)
    Z[0] = P[:, 0] + 1j * Q[:, 0]
    Z[64] = P[:, 1] + 1j * Q[:, 1]
    k = np.arange(1, 64)
    Z[1:64] = (P[:, 2 * k] - Q[:, 2 * k + 1] + 1j * (Q[:, 2 * k] + P[:, 2 * k + 1])).T
    return Z


def inverse(Sk):
    """x[r][c] = Re sum over the full spectrum, from its half k = 0 .. 64 (Sk: 65 x kc)."""
    aS = ALPHA[:, None] * Sk
    Ur = FR[:, :65] @ aS.real + FI[:, :65] @ aS.imag      # [Ur | Ui] = Fr [aSr | aSi] +
    Ui = FR[:, :65] @ aS.imag + FI[:, :65] @ (-aS.real)   #             Fi [aSi | -aSr]
    return (Ur @ FR.T + Ui @ FI.T) / (S * S)              # x = Ur Fr + Ui Fi


def test_half_spectrum_round_trip():
    """Forward with A1 and the two GEMMs, inverse with the folded mirror half:
    the identity on a real 128 x 128 block."""
    g = np.random.default_rng(5)
    x = g.standard_normal((S, S))
    Z = z_of(a1_matrix() @ x)
    assert np.allclose(Z, np.fft.fft2(x)[:65], atol=1e-9)
    assert np.allclose(inverse(Z), x, atol=1e-12)


@pytest.mark.parametrize("K,G", [(15, (3, 3)), (31, (2, 4))])
def test_block_model_matches_oracle_H_and_Ht(K, G):
    """One interior block of H and of H^T from the factorization, against the
    oracle's shift-variant operator and its adjoint on the same image."""
    g = np.random.default_rng(K)
    psfs = random_psfs(g, G, K).astype(np.float64)
    hy, wy = 220, 240
    nxr, nxc = hy + K - 1, wy + K - 1
    wr, wc = O.bilinear_weights(nxr, G[0]), O.bilinear_weights(nxc, G[1])
    b = S - K + 1
    r0, c0 = 37, 51                      # output block origin (H: y coords; H^T: x coords)
    A1 = a1_matrix()

    # H: window of x rows r0 .. r0 + 127; per PSF grid row one forward
    # transform of wr_a x, per PSF the column weight on Y' and the product
    x = g.uniform(0, 1, (nxr, nxc))
    rows = np.arange(r0, r0 + S)
    cols = np.arange(c0, c0 + S)
    xin = np.zeros((S, S))
    vr, vc = rows < nxr, cols < nxc
    xin[np.ix_(vr, vc)] = x[np.ix_(rows[vr], cols[vc])]
    Ssum = np.zeros((65, S), complex)
    for a in range(G[0]):
        wra = np.where(vr, wr[a, np.minimum(rows, nxr - 1)], 0.0)
        Yp = A1 @ (wra[:, None] * xin)
        for bb in range(G[1]):
            wcb = np.where(vc, wc[bb, np.minimum(cols, nxc - 1)], 0.0)
            Ssum += z_of(Yp * wcb[None, :]) * spectrum(psfs[a, bb])
    yblk = inverse(Ssum)[K - 1:, K - 1:]
    yref = O.apply_H(x, psfs, wr, wc)[r0:r0 + b, c0:c0 + b]
    assert np.abs(yblk - yref).max() <= 1e-10 * np.abs(yref).max()

    # H^T: window of r from K - 1 above / left of the output block; one forward
    # transform; per PSF the conjugate spectrum and the inverse, the row
    # weights summed over a inside the last stage, the column weight after
    r = g.standard_normal((hy, wy))
    rrows = np.arange(r0 - (K - 1), r0 - (K - 1) + S)
    rcols = np.arange(c0 - (K - 1), c0 - (K - 1) + S)
    vr2 = (rrows >= 0) & (rrows < hy)
    vc2 = (rcols >= 0) & (rcols < wy)
    rin = np.zeros((S, S))
    rin[np.ix_(vr2, vc2)] = r[np.ix_(rrows[vr2], rcols[vc2])]
    Z = z_of(A1 @ rin)
    gblk = np.zeros((S, S))
    for bb in range(G[1]):
        acc = np.zeros((S, S))
        for a in range(G[0]):
            T = ALPHA[:, None] * Z * np.conj(spectrum(psfs[a, bb]))
            Ur = FR[:, :65] @ T.real + FI[:, :65] @ T.imag
            Ui = FR[:, :65] @ T.imag + FI[:, :65] @ (-T.real)
            wra = wr[a, np.minimum(rows, nxr - 1)] * (rows < nxr)
            acc += (wra[:, None] * Ur) @ FR.T + (wra[:, None] * Ui) @ FI.T
        wcb = wc[bb, np.minimum(cols, nxc - 1)] * (cols < nxc)
        gblk += acc * wcb[None, :] / (S * S)
    gref = O.apply_Ht(r, psfs, wr, wc)[r0:r0 + b, c0:c0 + b]
    assert np.abs(gblk[:b, :b] - gref).max() <= 1e-10 * np.abs(gref).max()
