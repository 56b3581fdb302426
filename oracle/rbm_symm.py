"""Symmetric RBM (``RbmSpinSymm``, Sec. 2.2.2) in FP64 / complex128, and SR in
its parameter space.

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__``).

The paper names the symmetric RBM as the RBM variant that captures lattice
symmetries such as translations and inversions, and says nothing more.
Readings [r]:
* a symmetry group G of the lattice is given as a permutation table
  perm[g][i] (the image of site i under g); the hidden units come in alpha
  feature families with one unit per group element, unit (f, g) = f |G| + g;
* the unit (f, g) sees the filter of family f moved by g:
  W[(f, g), i] = Wt[f, perm[g][i]]; the families share a hidden bias
  b[(f, g)] = bt[f], and all sites share one visible bias a_i = at;
* so ln psi(sigma) = at sum_i sigma_i
                    + sum_f sum_g ln cosh(bt_f + sum_i Wt[f, perm[g][i]] sigma_i),
  which is invariant under every g of a group (the permutation h maps the unit
  (f, g) onto the unit (f, g h^-1));
* the log-derivatives with respect to the tied parameters are the sums of the
  untied ones over the units and sites each tied parameter stands for (chain
  rule): O_at = sum_i sigma_i, O_bt_f = sum_g tanh theta_(f,g),
  O_Wt[f, k] = sum_g tanh theta_(f,g) sigma_i with perm[g][i] = k;
* SR runs in the tied parameter space: S, F of Sec. 2.2.5 built from these
  derivatives, i.e. S_t = P^T S P and F_t = P^T F with P the matrix that copies
  a tied parameter into every untied one it stands for.
The parameter vector is ordered (at, bt, Wt row-major), P_t = 1 + alpha + alpha N.
"""
from __future__ import annotations

import numpy as np

from paper_1904_00031_gb300.workloads import RbmParams, RbmSymmParams

from . import rbm as _rbm
from . import sr as _sr


def expand(ps: RbmSymmParams, perm) -> RbmParams:
    """The untied RBM (a [N], b [alpha |G|], W [alpha |G|, N]) a symmetric one stands for."""
    perm = np.asarray(perm)
    ng, n = perm.shape
    a = np.full(n, ps.a[0])
    b = np.repeat(ps.b, ng)
    w = np.empty((ps.alpha * ng, n), dtype=ps.w.dtype)
    for f in range(ps.alpha):
        for g in range(ng):
            for i in range(n):
                w[f * ng + g, i] = ps.w[f, perm[g, i]]
    return RbmParams(a=a, b=b, w=w)


def theta(ps: RbmSymmParams, perm, sigma):
    """theta_(f,g) = bt_f + sum_i Wt[f, perm[g][i]] sigma_i, [ns, alpha |G|]."""
    sig = np.asarray(sigma, dtype=np.float64)
    perm = np.asarray(perm)
    ng = perm.shape[0]
    cols = []
    for f in range(ps.alpha):
        for g in range(ng):
            cols.append(sig @ ps.w[f, perm[g]] + ps.b[f])
    return np.stack(cols, axis=1)


def logpsi(ps: RbmSymmParams, perm, sigma):
    """ln psi [ns] of the symmetric RBM, written directly from its definition."""
    sig = np.asarray(sigma, dtype=np.float64)
    return ps.a[0] * sig.sum(axis=1) + _rbm.lncosh(theta(ps, perm, sig)).sum(axis=1)


def fold(v, n: int, alpha: int, perm):
    """P^T v: sums an untied parameter vector (a, b, W) into the tied one."""
    perm = np.asarray(perm)
    ng = perm.shape[0]
    m = alpha * ng
    v = np.asarray(v)
    va, vb, vw = v[:n], v[n:n + m], v[n + m:].reshape(m, n)
    out = np.zeros(1 + alpha + alpha * n, dtype=v.dtype)
    out[0] = va.sum()
    for f in range(alpha):
        out[1 + f] = vb[f * ng:(f + 1) * ng].sum()
        for g in range(ng):
            for i in range(n):
                out[1 + alpha + f * n + perm[g, i]] += vw[f * ng + g, i]
    return out


def expand_vector(x, n: int, alpha: int, perm):
    """P x: copies a tied parameter vector into the untied layout (a, b, W)."""
    ps = RbmSymmParams.from_flat(np.asarray(x), n, alpha)
    return expand(ps, perm).flat()


def logderiv_dense(ps: RbmSymmParams, perm, sigma):
    """Dense tied log-derivatives [ns, P_t] (chain rule through the ties)."""
    sig = np.asarray(sigma, dtype=np.float64)
    perm = np.asarray(perm)
    ng, n = perm.shape
    t = np.tanh(theta(ps, perm, sig))
    dt = np.complex128 if ps.is_complex else np.float64
    out = np.zeros((len(sig), ps.n_params), dtype=dt)
    out[:, 0] = sig.sum(axis=1)
    for f in range(ps.alpha):
        for g in range(ng):
            tj = t[:, f * ng + g]
            out[:, 1 + f] += tj
            for i in range(n):
                out[:, 1 + ps.alpha + f * n + perm[g, i]] += tj * sig[:, i]
    return out


def sr_direction_dense(ps: RbmSymmParams, perm, sigma, eloc, diag_shift: float,
                       weights=None):
    """(S_t + eps I)^{-1} F_t from the dense tied derivatives (Sec. 2.2.5)."""
    o = logderiv_dense(ps, perm, sigma)
    s, f = _sr.sr_matrices(o, eloc, weights, real=not ps.is_complex)
    return _sr.solve_dense(s, f, diag_shift)


def sr_direction_cg(ps: RbmSymmParams, perm, sigma, eloc, diag_shift: float, n_iter: int,
                    rtol: float, weights=None):
    """The same system solved matrix-free by CG in the tied space: every product
    S_t x = P^T S (P x) goes through the untied factored S (S never formed)."""
    perm = np.asarray(perm)
    n, alpha = ps.n, ps.alpha
    p_full = expand(ps, perm)
    sig, t = _rbm.logderiv_factored(p_full, sigma)
    real = not ps.is_complex
    m = p_full.m

    def matvec(x):
        xf = expand_vector(x, n, alpha, perm)
        return fold(_sr.sr_matvec_lazy(sig, t, xf, n, m, weights, real), n, alpha, perm)

    f = fold(_sr.force_lazy(sig, t, eloc, n, m, weights, real), n, alpha, perm)
    return _sr.cg(matvec, f, diag_shift, n_iter, rtol)
