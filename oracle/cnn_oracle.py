"""FP64 CPU oracle of the learned warm-start network (test infrastructure only).

The warm start maps the observed image and per-pixel PSF descriptor maps to a
correction of the start image of Algorithm 1:
    x0 = max(0, y_pad + net(features)).
The network is a stack of 3 x 3 convolutions with zero padding, ReLU between
layers and none after the last.  Tensors are NHWC: (batch, rows, cols,
channels).  Weights of a layer have shape (3, 3, C_in, C_out) and act as a
correlation:
    out[n, y, x, o] = b[o] + sum_{dy, dx, i} w[dy, dx, i, o] in[n, y+dy-1, x+dx-1, i].
The loss is 1/2 mean over pixels of (out - target)^2; training uses Adam
(Kingma & Ba) with bias correction.  Plain numpy in float64; backward passes
are written out from the chain rule, not from autograd.

Pins (tests/test_oracle_cnn.py): single-channel layers against
scipy.signal.correlate2d, gradients against central finite differences, and
the closed form of Adam's first step (a step of lr * g / (|g| + eps)).
"""

from __future__ import annotations

import numpy as np


def bf16_round(a):
    """Round float values to bfloat16 (round to nearest even) and back to float64."""
    f = np.asarray(a, dtype=np.float32)
    u = f.view(np.uint32).astype(np.uint64)
    lsb = (u >> 16) & 1
    u = ((u + 0x7FFF + lsb) >> 16) << 16
    return u.astype(np.uint32).view(np.float32).astype(np.float64)


def conv3x3(x, w, b):
    """Same-size 3x3 correlation with zero padding.  x (N,H,W,Ci), w (3,3,Ci,Co), b (Co)."""
    N, H, W, Ci = x.shape
    Co = w.shape[3]
    xp = np.zeros((N, H + 2, W + 2, Ci))
    xp[:, 1:H + 1, 1:W + 1, :] = x
    out = np.broadcast_to(b, (N, H, W, Co)).astype(np.float64).copy()
    for dy in range(3):
        for dx in range(3):
            out += xp[:, dy:dy + H, dx:dx + W, :] @ w[dy, dx]
    return out


def conv3x3_backward(x, w, dout):
    """Gradients of conv3x3 with respect to its input, weights and bias."""
    N, H, W, Ci = x.shape
    xp = np.zeros((N, H + 2, W + 2, Ci))
    xp[:, 1:H + 1, 1:W + 1, :] = x
    dxp = np.zeros_like(xp)
    dw = np.zeros_like(w)
    for dy in range(3):
        for dx in range(3):
            patch = xp[:, dy:dy + H, dx:dx + W, :]
            dw[dy, dx] = np.einsum("nhwi,nhwo->io", patch, dout)
            dxp[:, dy:dy + H, dx:dx + W, :] += dout @ w[dy, dx].T
    return dxp[:, 1:H + 1, 1:W + 1, :], dw, dout.sum(axis=(0, 1, 2))


def forward(params, x, act_round=None):
    """Runs the network; params = [(w, b), ...].  Returns (output (N,H,W),
    list of layer inputs, list of pre-activations).  act_round, if given, is
    applied to every stored activation (the GPU keeps them in bfloat16)."""
    inputs, pre = [], []
    h = x
    for li, (w, b) in enumerate(params):
        inputs.append(h)
        z = conv3x3(h, w, b)
        pre.append(z)
        h = np.maximum(z, 0.0) if li + 1 < len(params) else z
        if act_round is not None and li + 1 < len(params):
            h = act_round(h)
    return h[..., 0], inputs, pre


def mse_loss(out, target):
    d = out - target
    return 0.5 * float(np.mean(d * d)), d / d.size


def backward(params, inputs, pre, dout):
    """Gradients of all layers given d loss / d output (N,H,W)."""
    grads = [None] * len(params)
    g = dout[..., None]
    for li in range(len(params) - 1, -1, -1):
        w, _ = params[li]
        if li + 1 < len(params):
            g = g * (pre[li] > 0.0)
        dx, dw, db = conv3x3_backward(inputs[li], w, g)
        grads[li] = (dw, db)
        g = dx
    return grads


def adam_step(p, g, m, v, t, lr, beta1=0.9, beta2=0.999, eps=1e-8):
    """One Adam update (t counts from 1).  Returns (p, m, v)."""
    m = beta1 * m + (1.0 - beta1) * g
    v = beta2 * v + (1.0 - beta2) * g * g
    mh = m / (1.0 - beta1 ** t)
    vh = v / (1.0 - beta2 ** t)
    return p - lr * mh / (np.sqrt(vh) + eps), m, v


# ---------------------------------------------------------------------------
# Input features of the warm start
# ---------------------------------------------------------------------------

N_FEATURES = 5


def psf_descriptors(psfs):
    """Per grid PSF (Gr, Gc, 3): RMS radius / 8 px, 10 x peak value, and the
    fraction of |h| outside radius 3 px (all from |h| normalised to unit sum)."""
    Gr, Gc, K, _ = psfs.shape
    c = K // 2
    yy, xx = np.mgrid[0:K, 0:K]
    r2 = (yy - c) ** 2 + (xx - c) ** 2
    out = np.zeros((Gr, Gc, 3))
    for a in range(Gr):
        for b in range(Gc):
            h = np.abs(psfs[a, b].astype(np.float64))
            s = h.sum()
            if s <= 0:
                continue
            hn = h / s
            out[a, b, 0] = np.sqrt(np.sum(hn * r2)) / 8.0
            out[a, b, 1] = 10.0 * hn.max()
            out[a, b, 2] = np.sum(hn[r2 > 9])
    return out


def warmstart_features(y, psfs, noise_sigma, wr, wc):
    """(nxr, nxc, 5): observed image edge-replicated by K//2, the three PSF
    descriptor maps interpolated with the weights w_p, and 100 x noise sigma."""
    K = psfs.shape[2]
    ypad = np.pad(np.asarray(y, dtype=np.float64), K // 2, mode="edge")
    d = psf_descriptors(psfs)
    f = np.zeros(ypad.shape + (N_FEATURES,))
    f[..., 0] = ypad
    for a in range(psfs.shape[0]):
        for b in range(psfs.shape[1]):
            w = np.outer(wr[a], wc[b])
            for k in range(3):
                f[..., 1 + k] += w * d[a, b, k]
    f[..., 4] = 100.0 * noise_sigma
    return f
