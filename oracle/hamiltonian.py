"""Hamiltonian matrices, exact diagonalisation and Lanczos (Sec. 2.1 ``exact``
module: full ED and Lanczos for benchmarking small systems), plus the closed-form
ground energy of the periodic transverse-field Ising chain.

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__``).

Basis state x (an integer) encodes sigma_i = +1 if bit i of x is 0, -1 if it is 1,
so the local basis index idx(sigma_i) is bit i of x.
"""
from __future__ import annotations

import itertools

import numpy as np
import scipy.sparse as sp
import scipy.sparse.linalg as spla


def basis(n: int, zero_magnetisation: bool = False) -> np.ndarray:
    """All basis integers (ascending); optionally only the S^z = 0 sector."""
    xs = np.arange(1 << n, dtype=np.int64)
    if zero_magnetisation:
        pc = np.array([bin(int(x)).count("1") for x in xs])
        xs = xs[pc == n // 2]
    return xs


def configs(xs: np.ndarray, n: int) -> np.ndarray:
    """Basis integers -> spin configurations int8 [len, n]."""
    bits = (xs[:, None] >> np.arange(n)[None, :]) & 1
    return (1 - 2 * bits).astype(np.int8)


def sparse_h(op, xs: np.ndarray) -> sp.csr_matrix:
    """<x'|H|x> restricted to the sorted basis ``xs`` (an H-invariant subspace).

    Each site term contributes M[idx(s_i)][idx(s'_i)] for the 2 outcomes of
    site i; each bond term M4[2 idx(s_i)+idx(s_k)][2 idx(s'_i)+idx(s'_k)] for the
    4 outcomes of (i, k)."""
    rows, cols, vals = [], [], []

    def add(mel, xp, r):
        nz = np.nonzero(mel)[0]
        xp = xp[nz]
        at = np.searchsorted(xs, xp)
        if np.any(at >= len(xs)) or np.any(xs[np.minimum(at, len(xs) - 1)] != xp):
            raise ValueError("basis is not invariant under the Hamiltonian")
        rows.append(at)
        cols.append(r[nz])
        vals.append(mel[nz])

    r_all = np.arange(len(xs))
    for t in range(op.n_site_terms):
        i = int(op.site_idx[t])
        mat = op.site_mat[t]
        bi = (xs >> i) & 1
        for out in (0, 1):
            xp = (xs & ~(1 << i)) | (out << i)
            add(mat[bi, out], xp, r_all)
    for t in range(op.n_bond_terms):
        i, k = int(op.bond_i[t]), int(op.bond_k[t])
        mat = op.bond_mat[t]
        bi = (xs >> i) & 1
        bk = (xs >> k) & 1
        for oi, ok in itertools.product((0, 1), (0, 1)):
            xp = (xs & ~(1 << i) & ~(1 << k)) | (oi << i) | (ok << k)
            add(mat[2 * bi + bk, 2 * oi + ok], xp, r_all)
    dim = len(xs)
    rows = np.concatenate(rows) if rows else np.zeros(0, np.int64)
    cols = np.concatenate(cols) if cols else np.zeros(0, np.int64)
    vals = np.concatenate(vals) if vals else np.zeros(0, np.complex128)
    # H[x', x] = <x'|H|x>; duplicate entries are summed
    return sp.csr_matrix((vals.astype(np.complex128), (rows, cols)), shape=(dim, dim))


def exact_ground(op, zero_magnetisation: bool = False):
    """Full diagonalisation (dense eigh): (E0, psi0 over ``basis``)."""
    xs = basis(op.n, zero_magnetisation)
    h = sparse_h(op, xs).toarray()
    if np.abs(h.imag).max() == 0:
        h = h.real
    ev, vec = np.linalg.eigh(h)
    return float(ev[0]), vec[:, 0], xs


def lanczos_ground(op, zero_magnetisation: bool = False, tol: float = 1e-12):
    """Lowest eigenpair by Lanczos (scipy ARPACK, implicitly restarted Lanczos)."""
    xs = basis(op.n, zero_magnetisation)
    h = sparse_h(op, xs)
    if h.nnz == 0 or np.abs(h.data.imag).max() == 0:
        h = h.real
    ev, vec = spla.eigsh(h, k=1, which="SA", tol=tol)
    return float(ev[0]), vec[:, 0], xs


def tfim_chain_ground(n: int, J: float, h: float) -> float:
    """Ground energy of H = -J sum Z_i Z_{i+1} - h sum X_i on a periodic chain of
    even n (Pauli units), from the Jordan-Wigner free-fermion solution in the
    antiperiodic (even-parity) sector:
        E0 = - sum_{q = (2k+1) pi / n, k = 0..n-1} sqrt(J^2 + h^2 - 2 J h cos q)."""
    k = np.arange(n)
    q = (2 * k + 1) * np.pi / n
    return float(-np.sum(np.sqrt(J * J + h * h - 2 * J * h * np.cos(q))))
