"""Local energy E_loc(sigma) = sum_sigma' <sigma|H|sigma'> psi(sigma') / psi(sigma)
(Eq. 5, Sec. 2.2.5), for a Hamiltonian given as 1-local site terms and 2-local
bond terms (GraphOperator, Sec. 2.2.1).

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__``).

Two forms:
* ``local_energy_generic`` takes any log-amplitude function and evaluates every
  connected configuration by calling it: the definition written out.
* ``local_energy_rbm`` evaluates ln psi(sigma') of an RBM through the exact
  update theta' = theta - 2 sum_{flipped i} sigma_i W[:, i] (the same value,
  O(M) per connection instead of O(N M)).
"""
from __future__ import annotations

import itertools

import numpy as np

from . import rbm


def _outcomes(op):
    """Every (term kind, sites, matrix) triple of the operator."""
    for t in range(op.n_site_terms):
        yield (int(op.site_idx[t]),), op.site_mat[t]
    for t in range(op.n_bond_terms):
        yield (int(op.bond_i[t]), int(op.bond_k[t])), op.bond_mat[t]


def _idx(s):
    return (1 - np.asarray(s, dtype=np.int64)) // 2  # +1 -> 0, -1 -> 1


def local_energy_generic(logpsi_fn, op, sigma):
    """E_loc for a batch sigma [ns, N] given ``logpsi_fn(batch) -> [ns]``."""
    sigma = np.asarray(sigma, dtype=np.int8)
    ns = len(sigma)
    lp = np.asarray(logpsi_fn(sigma))
    e = np.zeros(ns, dtype=np.complex128)
    for sites, mat in _outcomes(op):
        row = np.zeros(ns, dtype=np.int64)
        for i in sites:
            row = 2 * row + _idx(sigma[:, i])
        for out in itertools.product((0, 1), repeat=len(sites)):
            col = 0
            for o in out:
                col = 2 * col + o
            mel = mat[row, col]
            nz = np.nonzero(mel)[0]
            if len(nz) == 0:
                continue
            sp = sigma[nz].copy()
            for i, o in zip(sites, out):
                sp[:, i] = 1 - 2 * o
            same = np.all(sp == sigma[nz], axis=1)
            ratio = np.ones(len(nz), dtype=np.complex128)
            if np.any(~same):
                d = np.asarray(logpsi_fn(sp[~same])) - lp[nz][~same]
                ratio[~same] = np.exp(d)
            e[nz] += mel[nz] * ratio
    return e


def local_energy_rbm(p, op, sigma):
    """E_loc of the RBM for a batch sigma [ns, N], connections by theta update."""
    sigma = np.asarray(sigma, dtype=np.int8)
    sig = sigma.astype(np.float64)
    ns = len(sigma)
    th = rbm.theta(p, sig)
    base = rbm.lncosh(th).sum(axis=1)
    e = np.zeros(ns, dtype=np.complex128)
    for sites, mat in _outcomes(op):
        row = np.zeros(ns, dtype=np.int64)
        for i in sites:
            row = 2 * row + _idx(sigma[:, i])
        for out in itertools.product((0, 1), repeat=len(sites)):
            col = 0
            for o in out:
                col = 2 * col + o
            mel = mat[row, col]
            nz = np.nonzero(mel)[0]
            if len(nz) == 0:
                continue
            # sites whose spin changes, per sample
            dlog = np.zeros(len(nz), dtype=np.complex128)
            thp = th[nz].copy()
            for i, o in zip(sites, out):
                new = 1 - 2 * o
                si = sig[nz, i]
                flip = si != new
                # sigma_i -> -sigma_i: a_i sigma_i changes by -2 a_i sigma_i,
                # theta changes by -2 sigma_i W[:, i]
                dlog = dlog + np.where(flip, -2.0 * p.a[i] * si, 0.0)
                thp = thp - np.where(flip, 2.0 * si, 0.0)[:, None] * p.w[:, i][None, :]
            dlog = dlog + rbm.lncosh(thp).sum(axis=1) - base[nz]
            e[nz] += mel[nz] * np.exp(dlog)
    return e
