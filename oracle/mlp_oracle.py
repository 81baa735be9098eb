"""FP64 CPU oracle of the warm-start network (test infrastructure only: the tests call it; the
product path never does).

Plain numpy, following the definition written in the library header: widths
d_0 -> d_1 (ReLU) ... -> d_L, parameters flat per layer (W [out][in] row-major, then b),
inputs and targets standardised per column, loss = mean squared error over rows and
outputs.  Gradients are central finite differences of that loss, nothing else.
"""
from __future__ import annotations

import numpy as np


def layer_slices(dims):
    """[(W slice, b slice, out, in)] per layer of the flat parameter vector."""
    out, off = [], 0
    for l in range(1, len(dims)):
        nw = dims[l] * dims[l - 1]
        out.append((slice(off, off + nw), slice(off + nw, off + nw + dims[l]), dims[l], dims[l - 1]))
        off += nw + dims[l]
    return out


def n_params(dims):
    return sum(dims[l] * dims[l - 1] + dims[l] for l in range(1, len(dims)))


def forward(params, dims, X, x_mu=None, x_sd=None, y_mu=None, y_sd=None, standardised_out=False):
    """Network output for rows X (FP64).  With standardised_out the output is left in the
    standardised target units (what the loss compares)."""
    p = np.asarray(params, np.float64)
    H = np.asarray(X, np.float64)
    if x_mu is not None:
        H = (H - x_mu) / x_sd
    L = len(dims) - 1
    for l, (ws, bs, o, i) in enumerate(layer_slices(dims), start=1):
        H = H @ p[ws].reshape(o, i).T + p[bs]
        if l < L:
            H = np.maximum(H, 0.0)
    if standardised_out or y_mu is None:
        return H
    return H * y_sd + y_mu


def loss(params, dims, X, Y, x_mu=None, x_sd=None, y_mu=None, y_sd=None):
    Yh = forward(params, dims, X, x_mu, x_sd, standardised_out=True)
    T = np.asarray(Y, np.float64)
    if y_mu is not None:
        T = (T - y_mu) / y_sd
    return float(np.mean((Yh - T) ** 2))


def fd_grad(params, dims, X, Y, idx, eps=1e-6, **norm):
    """Central differences of the loss at the parameter indices idx."""
    p = np.asarray(params, np.float64).copy()
    g = np.zeros(len(idx))
    for k, i in enumerate(idx):
        old = p[i]
        p[i] = old + eps
        lp = loss(p, dims, X, Y, **norm)
        p[i] = old - eps
        lm = loss(p, dims, X, Y, **norm)
        p[i] = old
        g[k] = (lp - lm) / (2 * eps)
    return g
