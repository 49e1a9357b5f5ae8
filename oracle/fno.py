"""Plain FP64 forward pass of the Fourier-neural-operator start predictor.

Test infrastructure (see ``oracle/__init__.py``): not used by the product.

The learned start is not in arXiv 1701.04685; it predicts the starting strain
fluctuation E for the paper's fixed point (Sec. 4) from the microstructure and
the macroscopic strain, so the iteration only has to remove the prediction's
error.  The network (a Fourier neural operator) is, for input channels x on an
N^3 grid:

    v_0     = P x + p                               (pointwise lift to `width`)
    u_l     = W_l v_l + w_l + K_l v_l,  v_{l+1} = gelu(u_l),   l = 0..L-1
    y       = Q v_L + q                             (pointwise projection)

with the spectral convolution K_l restricted to the modes
kx, ky in {-m..m-1}, kz in {0..m-1}:

    v^(k)   = sum_x v(x) exp(-2 pi i k.x / N)                  (truncated DFT)
    c(k)    = R_l(k) v^(k)                                     (width x width, complex)
    (K v)(x)= N^-3 Re sum_k w(kz) c(k) exp(+2 pi i k.x / N),   w(0) = 1, w(kz > 0) = 2,

which is numpy's irfftn of the zero-padded coefficients.  gelu is the exact
0.5 x (1 + erf(x / sqrt 2)).
"""
from __future__ import annotations

import numpy as np
from scipy.special import erf


def mode_index(N, m):
    """Grid indices of the kept modes along x and y (kx = 0..m-1, then -m..-1)."""
    return np.concatenate([np.arange(m), np.arange(N - m, N)])


class Params:
    """Parameters in the layout of the product: R[l] of shape (2m, 2m, m, width, width)
    complex (mode-major, then output, then input channel)."""

    def __init__(self, cin, cout, width, modes, layers):
        self.cin, self.cout, self.width, self.modes, self.layers = cin, cout, width, modes, layers
        m = modes
        self.P = np.zeros((width, cin))
        self.p = np.zeros(width)
        self.W = np.zeros((layers, width, width))
        self.w = np.zeros((layers, width))
        self.R = np.zeros((layers, 2 * m, 2 * m, m, width, width), dtype=complex)
        self.Q = np.zeros((cout, width))
        self.q = np.zeros(cout)

    def flat(self):
        parts = [self.P, self.p, self.W, self.w, self.R.real, self.R.imag, self.Q, self.q]
        return np.concatenate([a.ravel() for a in parts])

    def set_flat(self, v):
        o = 0
        for name in ("P", "p", "W", "w"):
            a = getattr(self, name)
            a[...] = v[o:o + a.size].reshape(a.shape)
            o += a.size
        n = self.R.size
        self.R = v[o:o + n].reshape(self.R.shape) + 1j * v[o + n:o + 2 * n].reshape(self.R.shape)
        o += 2 * n
        for name in ("Q", "q"):
            a = getattr(self, name)
            a[...] = v[o:o + a.size].reshape(a.shape)
            o += a.size


def gelu(u):
    return 0.5 * u * (1.0 + erf(u / np.sqrt(2.0)))


def spectral(v, R, modes):
    """K v for v of shape (C, N, N, N); R of shape (2m, 2m, m, Cout, Cin)."""
    C, N = v.shape[0], v.shape[1]
    m = modes
    vh = np.fft.rfftn(v, axes=(1, 2, 3))
    ix = mode_index(N, m)
    sel = vh[:, ix][:, :, ix][..., :m]                      # (C, 2m, 2m, m)
    out = np.einsum("abkoi,iabk->oabk", R, sel)             # (Cout, 2m, 2m, m)
    full = np.zeros((R.shape[3], N, N, N // 2 + 1), dtype=complex)
    full[:, ix[:, None], ix[None, :], :m] = out
    return np.fft.irfftn(full, s=(N, N, N), axes=(1, 2, 3))


def forward(params, x):
    """y for one sample x of shape (cin, N, N, N)."""
    v = np.einsum("oc,cxyz->oxyz", params.P, x) + params.p[:, None, None, None]
    for l in range(params.layers):
        u = (np.einsum("oi,ixyz->oxyz", params.W[l], v) + params.w[l][:, None, None, None]
             + spectral(v, params.R[l], params.modes))
        v = gelu(u)
    return np.einsum("oc,cxyz->oxyz", params.Q, v) + params.q[:, None, None, None]


def loss(params, xs, ts):
    """Mean squared error over a batch: mean over samples, channels and voxels."""
    tot, cnt = 0.0, 0
    for x, t in zip(xs, ts):
        y = forward(params, x)
        tot += np.sum((y - t) ** 2)
        cnt += y.size
    return tot / cnt
