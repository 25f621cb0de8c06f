"""FP64 reference of the learned NCC-weight network (test infrastructure).

This is the oracle of the learned form: a plain NumPy restatement of a
small convolutional network that maps band energies of the full-aperture
angular-spectrum image to the AS-TAX NCC weight map rho_n (Eq. 10-11 give the
target). Only tests/ and the bench's baseline leg import it; the library's
CUDA kernels never do.

Definitions (all arrays float64, NCHW):
* conv3x3 with zero padding 1:
    y[n, o, i, j] = b[o] + sum_{c, u, v} w[o, c, u, v] x[n, c, i + u - 1, j + v - 1]
* its gradients (the adjoint of the above):
    dx[n, c, i, j] = sum_{o, u, v} w[o, c, u, v] dy[n, o, i - u + 1, j - v + 1]
    dw[o, c, u, v] = sum_{n, i, j} dy[n, o, i, j] x[n, c, i + u - 1, j + v - 1]
    db[o]          = sum_{n, i, j} dy[n, o, i, j]
* network: 5 conv3x3 layers 5 -> 32 -> 32 -> 32 -> 32 -> 1, ReLU after the
  first four, and the head rho = eps + (1 - eps) sigmoid(z), so that the
  prediction lies in [eps, 1) like the clamped NCC of Sec. II-A.
* loss: energy-weighted mean squared error against the target map,
    L = (1/n) sum_px w (rho - target)^2,  w = 0.05 + 0.95 min(1, E/max E),
  with E/max E = 10^(4 x0) - 1e-4 recovered from input channel 0 (a fixed
  function of the input): the image is rho^2 E, so the bright pixels matter
  most, and the floor keeps the background supervised.
* Adam (Kingma and Ba 2015) with bias correction.
* features: channel 0 = log10(E / max E + 1e-4) of the full-aperture energy
  E = sum_k |p~|^2 (Eq. 3), channels 1..4 the same for the energy of each
  contiguous quarter of the bins, all divided by 4 so that they lie in [-1, 0].

Parity pins live in tests/test_cnn_oracle.py: the convolution against
scipy.signal.correlate2d, every gradient against central finite
differences, and Adam's first step (lr times the gradient's sign).
"""
from __future__ import annotations

import numpy as np

CHANNELS = (5, 32, 32, 32, 32, 1)
FEATURE_FLOOR = 1e-4
WEIGHT_FLOOR = 0.05


def conv3x3(x, w, b):
    """x [N][C][H][W], w [O][C][3][3], b [O] -> [N][O][H][W]."""
    N, C, H, W = x.shape
    O = w.shape[0]
    xp = np.zeros((N, C, H + 2, W + 2))
    xp[:, :, 1:H + 1, 1:W + 1] = x
    y = np.zeros((N, O, H, W)) + b[None, :, None, None]
    for u in range(3):
        for v in range(3):
            patch = xp[:, :, u:u + H, v:v + W]                      # x[n, c, i+u-1, j+v-1]
            y += np.einsum("oc,nchw->nohw", w[:, :, u, v], patch)
    return y


def conv3x3_backward(x, w, dy):
    """Gradients (dx, dw, db) of conv3x3 for upstream dy."""
    N, C, H, W = x.shape
    xp = np.zeros((N, C, H + 2, W + 2))
    xp[:, :, 1:H + 1, 1:W + 1] = x
    dxp = np.zeros_like(xp)
    dw = np.zeros_like(w)
    for u in range(3):
        for v in range(3):
            patch = xp[:, :, u:u + H, v:v + W]
            dw[:, :, u, v] = np.einsum("nohw,nchw->oc", dy, patch)
            dxp[:, :, u:u + H, v:v + W] += np.einsum("oc,nohw->nchw", w[:, :, u, v], dy)
    db = dy.sum(axis=(0, 2, 3))
    return dxp[:, :, 1:H + 1, 1:W + 1], dw, db


def sigmoid(z):
    return 1.0 / (1.0 + np.exp(-z))


def init_params(seed: int = 0, channels=CHANNELS):
    """He-normal weights, zero biases (the starting point of training)."""
    rng = np.random.default_rng(seed)
    params = []
    for cin, cout in zip(channels[:-1], channels[1:]):
        w = rng.standard_normal((cout, cin, 3, 3)) * np.sqrt(2.0 / (9 * cin))
        params.append((w, np.zeros(cout)))
    return params


def forward(params, x, eps: float = 1e-3):
    """Returns (rho, cache) for features x [N][5][H][W]."""
    acts = [x]
    h = x
    for li, (w, b) in enumerate(params):
        z = conv3x3(h, w, b)
        if li < len(params) - 1:
            h = np.maximum(z, 0.0)
            acts.append(h)
        else:
            s = sigmoid(z)
            return eps + (1.0 - eps) * s, (acts, s)
    raise ValueError("empty network")


def loss_weights(x):
    """Per-pixel loss weight [N][1][H][W] from the input's channel 0."""
    e = np.clip(10.0 ** (4.0 * np.asarray(x, dtype=np.float64)[:, :1]) - FEATURE_FLOOR, 0.0, 1.0)
    return WEIGHT_FLOOR + (1.0 - WEIGHT_FLOOR) * e


def loss_and_grads(params, x, target, eps: float = 1e-3):
    """Energy-weighted mean squared error and its gradients with respect to every (w, b)."""
    rho, (acts, s) = forward(params, x, eps)
    diff = rho - target[:, None] if target.ndim == 3 else rho - target
    n = diff.size
    wgt = loss_weights(x)
    loss = float(np.sum(wgt * diff ** 2) / n)
    dy = 2.0 * wgt * diff / n * (1.0 - eps) * s * (1.0 - s)
    grads = [None] * len(params)
    for li in range(len(params) - 1, -1, -1):
        w, b = params[li]
        dx, dw, db = conv3x3_backward(acts[li], w, dy)
        grads[li] = (dw, db)
        if li > 0:
            dy = dx * (acts[li] > 0.0)
    return loss, grads


def adam_step(p, g, m, v, t, lr=1e-3, beta1=0.9, beta2=0.999, eps=1e-8):
    """One Adam update of p (returns new p, m, v); t counts from 1."""
    m = beta1 * m + (1.0 - beta1) * g
    v = beta2 * v + (1.0 - beta2) * g * g
    mh = m / (1.0 - beta1 ** t)
    vh = v / (1.0 - beta2 ** t)
    return p - lr * mh / (np.sqrt(vh) + eps), m, v


def features(e_bands):
    """e_bands [4][H][W] band energies (quarters of the bins) -> [5][H][W]."""
    e_bands = np.asarray(e_bands, dtype=np.float64)
    e = e_bands.sum(axis=0)
    m = e.max()
    scale = 1.0 / m if m > 0 else 0.0
    out = np.empty((5,) + e.shape)
    out[0] = np.log10(e * scale + FEATURE_FLOOR) / 4.0
    for q in range(4):
        out[1 + q] = np.log10(e_bands[q] * scale + FEATURE_FLOOR) / 4.0
    return out
