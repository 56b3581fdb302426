"""RBM amplitude and log-derivatives in FP64 / complex128.

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__``).

Sec. 2.2.2 (``RbmSpin``, fully complex parameters; an RBM is a single-layer
FFNN with ln cosh activation):

    ln psi(sigma) = sum_i a_i sigma_i + sum_j ln cosh(theta_j),
    theta = W sigma + b.

Readings where the paper is silent:
* both biases a and b are present (``RbmSpin``);
* no constant M ln 2 is added (it cancels in every ratio, derivative and
  local energy);
* ln cosh is evaluated through the identity ln cosh z = s z + log1p(exp(-2 s z))
  - ln 2 with s = sign(Re z) (cosh is even), which never overflows.

Log-derivatives (Sec. 2.2.5, "obtained analytically for the RBM"),
holomorphic for complex parameters:
    O_{a_i} = sigma_i,  O_{b_j} = tanh(theta_j),  O_{W_ji} = tanh(theta_j) sigma_i,
ordered as the parameter vector (a, b, W row-major).
"""
from __future__ import annotations

import numpy as np

LN2 = float(np.log(2.0))


def lncosh(z):
    """ln cosh z, elementwise, real or complex."""
    z = np.asarray(z)
    s = np.where(np.real(z) >= 0, 1.0, -1.0)
    zz = s * z
    return zz + np.log1p(np.exp(-2.0 * zz)) - LN2


def theta(p, sigma):
    """theta = W sigma + b for a batch sigma [ns, N] -> [ns, M]."""
    sig = np.asarray(sigma, dtype=np.float64)
    return sig @ p.w.T + p.b[None, :]


def logpsi(p, sigma):
    """ln psi for a batch sigma [ns, N] -> [ns] (complex128 if the parameters are)."""
    sig = np.asarray(sigma, dtype=np.float64)
    return sig @ p.a + lncosh(theta(p, sig)).sum(axis=1)


def logderiv_dense(p, sigma):
    """Dense log-derivative matrix O [ns, P], P = N + M + M N."""
    sig = np.asarray(sigma, dtype=np.float64)
    t = np.tanh(theta(p, sig))
    ow = t[:, :, None] * sig[:, None, :]
    dt = np.complex128 if p.is_complex else np.float64
    return np.concatenate([sig.astype(dt), t, ow.reshape(len(sig), -1)], axis=1)


def logderiv_factored(p, sigma):
    """Factored log-derivatives: (sigma, T = tanh theta); O_W = T (x) sigma."""
    sig = np.asarray(sigma, dtype=np.float64)
    return sig, np.tanh(theta(p, sig))


def logpsi_backward(p, sigma, g):
    """Gradient of sum_s g_s ln psi(sigma_s) with respect to (a, b, W):
    the O^T g contraction of the analytic derivatives, returned flat [P]."""
    sig, t = logderiv_factored(p, sigma)
    g = np.asarray(g)
    ga = sig.T @ g
    gb = t.T @ g
    gw = (t * g[:, None]).T @ sig
    return np.concatenate([ga, gb, gw.reshape(-1)])
