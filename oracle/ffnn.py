"""Multi-layer feed-forward network with ln cosh activations (Sec. 2.2.2: FFNN
machines built from dense layers y = W x + b and Lncosh activations, with a
sum output; an RBM without visible bias is the one-layer case, and stacking
layers generalises it), in FP64 / complex128.

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__``).

    x_0 = sigma,  h_l = W_l x_(l-1) + b_l,  x_l = ln cosh(h_l)   (l = 1 .. L),
    ln psi(sigma) = sum_j x_(L, j).

Readings [r]: the output layer is the sum of the last activations (NetKet's
Sum layer); parameters are ordered layer by layer, W_l row-major [w_l][w_(l-1)]
then b_l; for complex parameters everything is holomorphic.

Log-derivatives (holomorphic, by the chain rule):
    d ln psi / d h_L = tanh(h_L),
    d ln psi / d h_(l-1) = (W_l^T d ln psi / d h_l) * tanh(h_(l-1)),
    d ln psi / d W_l[j][i] = (d ln psi / d h_l)_j x_(l-1, i),  d / d b_l = d / d h_l.
"""
from __future__ import annotations

import numpy as np

from .rbm import lncosh


def n_params(widths) -> int:
    return int(sum(widths[l] * (widths[l - 1] + 1) for l in range(1, len(widths))))


def unpack(params, widths):
    """[(W_l, b_l)] from the flat parameter vector."""
    out, o = [], 0
    for l in range(1, len(widths)):
        wo, wi = widths[l], widths[l - 1]
        W = np.asarray(params[o:o + wo * wi]).reshape(wo, wi)
        o += wo * wi
        b = np.asarray(params[o:o + wo])
        o += wo
        out.append((W, b))
    return out


def forward(params, widths, sigma):
    """(ln psi [ns], pre-activations [h_1 .. h_L], inputs [x_0 .. x_(L-1)])."""
    x = np.asarray(sigma, dtype=np.float64)
    hs, xs = [], []
    for W, b in unpack(params, widths):
        xs.append(x)
        h = x @ W.T + b[None, :]
        hs.append(h)
        x = lncosh(h)
    return x.sum(axis=1), hs, xs


def logpsi(params, widths, sigma):
    return forward(params, widths, sigma)[0]


def logderiv_dense(params, widths, sigma):
    """O [ns, P]: d ln psi(sigma_s) / d alpha_k in the flat parameter order."""
    _, hs, xs = forward(params, widths, sigma)
    layers = unpack(params, widths)
    d = np.tanh(hs[-1])                      # d ln psi / d h_L
    blocks = [None] * len(layers)
    for l in range(len(layers) - 1, -1, -1):
        W, _ = layers[l]
        gw = d[:, :, None] * xs[l][:, None, :]             # [ns, w_l, w_(l-1)]
        blocks[l] = np.concatenate([gw.reshape(len(d), -1), d], axis=1)
        if l > 0:
            d = (d @ W) * np.tanh(hs[l - 1])
    return np.concatenate(blocks, axis=1)


def backward(params, widths, sigma, g):
    """sum_s conj(O_sk) g_s (the conjugate-Wirtinger convention of the RBM
    backward), flat [P]; real parameters: sum_s O_sk Re g_s."""
    o = logderiv_dense(params, widths, sigma)
    if np.iscomplexobj(params):
        return o.conj().T @ np.asarray(g, dtype=np.complex128)
    return o.T @ np.real(np.asarray(g))
