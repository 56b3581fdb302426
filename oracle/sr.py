"""Energy statistics and stochastic reconfiguration (Sec. 2.2.5: the energy
gradient is estimated together with <H>; SR approximates imaginary-time
evolution and is solved by an exact or an iterative linear solver; the update
is the SGD rule alpha <- alpha - lambda * direction of Eq. 2, Sec. 2.2.3).

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__``).

The paper prints no SR formulas; this follows Sorella's SR, which it cites
(readings marked [r]):
  weights w_s (1/Ns for Monte Carlo samples, |psi|^2/Z in full-sum mode),
  <X> = sum_s w_s X_s,
  S_kl = <O_k^* O_l> - <O_k^*><O_l>,
  F_k  = <O_k^* E_loc> - <O_k^*><E_loc>,
  (S + eps I) delta = F with an absolute diagonal shift eps [r],
  alpha <- alpha - lr * delta.
For real parameters S and F are replaced by their real parts [r].
Statistics [r]: E = <E_loc> (complex mean; Re E is the energy estimate),
variance = <|E_loc - E|^2>, error bar from the means m_g of n_blocks equal blocks
of consecutive samples that are independent of one another:
sigma_E = sqrt(sum_g (Re m_g - Re E)^2 / (n_blocks (n_blocks - 1))).
The chains of one proposal group share their proposal sequence (``sampler``),
so they are not independent of one another; the independent units are whole
groups, and the VMC iteration passes n_blocks = number of groups.
"""
from __future__ import annotations

import numpy as np


def stats(eloc, n_blocks: int):
    """(mean, variance, error bar) of E_loc; samples are chain-major and the
    error bar comes from the means of ``n_blocks`` equal blocks of consecutive
    samples (independent units: chains, or proposal groups of chains)."""
    e = np.asarray(eloc, dtype=np.complex128)
    mean = e.mean()
    var = float(np.mean(np.abs(e - mean) ** 2))
    m = e.reshape(n_blocks, -1).mean(axis=1).real
    if n_blocks > 1:
        err = float(np.sqrt(np.sum((m - mean.real) ** 2) / (n_blocks * (n_blocks - 1))))
    else:
        err = float("nan")
    return complex(mean), var, err


def _w(ns, weights):
    if weights is None:
        return np.full(ns, 1.0 / ns)
    return np.asarray(weights, dtype=np.float64)


def sr_matrices(o, eloc, weights=None, real: bool = False):
    """Dense S [P, P] and F [P] from the dense log-derivative matrix O [ns, P]."""
    o = np.asarray(o)
    e = np.asarray(eloc, dtype=np.complex128)
    w = _w(len(o), weights)
    obar = w @ o
    emean = w @ e
    s = (o.conj().T * w) @ o - np.outer(obar.conj(), obar)
    f = (o.conj().T * w) @ e - obar.conj() * emean
    if real:
        return s.real, f.real
    return s, f


def solve_dense(s, f, diag_shift: float):
    """delta = (S + eps I)^{-1} F by a dense Cholesky factorisation."""
    a = s + diag_shift * np.eye(len(s))
    c = np.linalg.cholesky(a)
    y = np.linalg.solve(c, f)
    return np.linalg.solve(c.conj().T, y)


def sr_matvec_lazy(sigma, t, x, n: int, m: int, weights=None, real: bool = False):
    """S x without forming S, from the factored O = (sigma, T, T (x) sigma):
    y_s = O_s . x = sigma_s . x_a + T_s . x_b + sum_j T_sj (X_W sigma_s)_j,
    S x = sum_s w_s O_s^* (y_s - <y>)  with <y> = obar . x."""
    sig = np.asarray(sigma, dtype=np.float64)
    w = _w(len(sig), weights)
    xa, xb, xw = x[:n], x[n:n + m], x[n + m:].reshape(m, n)
    y = sig @ xa + t @ xb + np.sum(t * (sig @ xw.T), axis=1)
    y = y - w @ y
    wy = w * y
    ra = sig.T @ wy
    rb = t.conj().T @ wy
    rw = (t.conj() * wy[:, None]).T @ sig
    out = np.concatenate([ra, rb, rw.reshape(-1)])
    return out.real if real else out


def force_lazy(sigma, t, eloc, n: int, m: int, weights=None, real: bool = False):
    """F = <O^* (E_loc - <E_loc>)> from the factored O."""
    sig = np.asarray(sigma, dtype=np.float64)
    e = np.asarray(eloc, dtype=np.complex128)
    w = _w(len(sig), weights)
    d = w * (e - w @ e)
    fa = sig.T @ d
    fb = t.conj().T @ d
    fw = (t.conj() * d[:, None]).T @ sig
    out = np.concatenate([fa, fb, fw.reshape(-1)])
    return out.real if real else out


def cg(matvec, f, diag_shift: float, n_iter: int, rtol: float = 1e-12):
    """Conjugate gradient for (S + eps I) x = F from x0 = 0.  Runs n_iter
    iterations unless ||r|| <= rtol ||F|| first.  Returns (x, iterations, ||r||/||F||)."""
    x = np.zeros_like(f)
    r = f.copy()
    p = r.copy()
    rs = np.vdot(r, r).real
    fn = np.sqrt(np.vdot(f, f).real)
    it = 0
    if fn == 0.0:
        return x, 0, 0.0
    for it in range(1, n_iter + 1):
        ap = matvec(p) + diag_shift * p
        alpha = rs / np.vdot(p, ap).real
        x = x + alpha * p
        r = r - alpha * ap
        rs_new = np.vdot(r, r).real
        if np.sqrt(rs_new) <= rtol * fn:
            rs = rs_new
            break
        p = r + (rs_new / rs) * p
        rs = rs_new
    return x, it, float(np.sqrt(rs) / fn)


def sgd_update(params_flat, delta, lr: float):
    """alpha <- alpha - lr * delta (Eq. 2)."""
    return params_flat - lr * delta
