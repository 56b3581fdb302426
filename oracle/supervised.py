"""Supervised learning of a target wavefunction (Sec. 2.2.3): the negative log
overlap loss of Eq. 1, its gradient, and the AdaMax update the optimiser list
names (Kingma and Ba, "Adam: a method for stochastic optimization", Algorithm 2).

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__``).

Eq. 1: L = -log( <tar|psi><psi|tar> / (<tar|tar><psi|psi>) ), which is 0 when psi
is proportional to the target and positive otherwise.  Readings [r]:
* Monte Carlo form ("direct sampling of the target"): samples sigma_s drawn
  from |tar|^2 / <tar|tar> with weights w_s, ratios R_s = psi(sigma_s) / tar(sigma_s);
  <tar|psi>/<tar|tar> = <R>, <psi|psi>/<tar|tar> = <|R|^2>, so
  L = -log(|<R>|^2 / <|R|^2>);
* gradient: for holomorphic psi with log-derivatives O (Sec. 2.2.5),
  dL/d conj(alpha) = <O^* |R|^2> / <|R|^2> - <O^* R^*> / <R^*>; the reported
  gradient is twice that (for a real parameter, dL/dalpha = 2 Re of it; for a
  complex one, d/dRe + i d/dIm), and real parameters take the real part;
* full-sum form: the same with every basis state as a sample, w ~ |tar|^2;
* AdaMax treats the real and imaginary parts of a complex parameter as two real
  parameters with their own moments; a parameter whose u is still 0 is not moved.
"""
from __future__ import annotations

import numpy as np

from . import rbm


def _w(ns, weights):
    if weights is None:
        return np.full(ns, 1.0 / ns)
    w = np.asarray(weights, dtype=np.float64)
    return w / w.sum()


def overlap_loss_and_grad(p, sigma, target_vals, weights=None):
    """(L, gradient [P]) of Eq. 1 from samples of the target: ``sigma`` [ns, N],
    ``target_vals`` = tar(sigma_s) (complex), ``weights`` the sample weights
    (None: 1/ns, i.e. samples drawn from |tar|^2)."""
    sig = np.asarray(sigma)
    psi = np.exp(rbm.logpsi(p, sig))
    r = psi / np.asarray(target_vals, dtype=np.complex128)
    w = _w(len(sig), weights)
    mr = w @ r
    mr2 = w @ (np.abs(r) ** 2)
    loss = float(-np.log(np.abs(mr) ** 2 / mr2))
    o = rbm.logderiv_dense(p, sig)
    g = 2.0 * ((o.conj().T @ (w * np.abs(r) ** 2)) / mr2
               - (o.conj().T @ (w * r.conj())) / np.conj(mr))
    if not p.is_complex:
        g = g.real
    return loss, g


def overlap_loss_full(p, configs, target_vals):
    """Eq. 1 summed over an enumerated basis (no sampling)."""
    psi = np.exp(rbm.logpsi(p, configs))
    t = np.asarray(target_vals, dtype=np.complex128)
    ov = np.vdot(t, psi)
    return float(-np.log(np.abs(ov) ** 2 / (np.vdot(t, t).real * np.vdot(psi, psi).real)))


class AdaMax:
    """AdaMax (Kingma and Ba, Algorithm 2) on a real or complex parameter vector:
    m <- b1 m + (1 - b1) g, u <- max(b2 u, |g|),
    theta <- theta - (lr / (1 - b1^t)) m / u."""

    def __init__(self, lr: float = 0.001, beta1: float = 0.9, beta2: float = 0.999):
        self.lr, self.b1, self.b2 = lr, beta1, beta2
        self.t = 0
        self.m = None
        self.u = None

    def step(self, theta, g):
        theta = np.asarray(theta)
        cplx = np.iscomplexobj(theta)
        gr = np.concatenate([np.real(g), np.imag(g)]) if cplx else np.asarray(g, np.float64)
        if self.m is None:
            self.m = np.zeros_like(gr)
            self.u = np.zeros_like(gr)
        self.t += 1
        self.m = self.b1 * self.m + (1.0 - self.b1) * gr
        self.u = np.maximum(self.b2 * self.u, np.abs(gr))
        safe = np.where(self.u > 0, self.u, 1.0)
        d = np.where(self.u > 0, self.lr / (1.0 - self.b1 ** self.t) * self.m / safe, 0.0)
        if cplx:
            k = len(theta)
            d = d[:k] + 1j * d[k:]
        return theta - d
