"""Seeded synthetic inputs shared by the CUDA path, the tests and the CPU oracle.

This module holds problem *definitions* only: lattices and bond lists (the
``Hypercube`` graph and coloured bonds of Sec. 2.2.1), the 1-local / 2-local
operator tables of a ``GraphOperator``-style Hamiltonian (Sec. 2.2.1), RBM
parameter initialisation (``init_random_parameters(seed, sigma)`` of the VMC
listing in Sec. 3.1) and initial Markov-chain configurations.  It contains none
of the method's arithmetic (no amplitudes, ratios, local energies, SR algebra).

Conventions used everywhere in this project
-------------------------------------------
* A spin configuration is sigma in {+1, -1}^N, stored as int8.  +1 is "up".
* The local basis index of a spin is ``idx(+1) = 0``, ``idx(-1) = 1``.
* A site operator is a 2x2 complex matrix ``M[idx(s)][idx(s')] = <s|O|s'>``.
* A bond operator on (i, k) is a 4x4 complex matrix in the basis
  ``2*idx(s_i) + idx(s_k)``, i.e. (++, +-, -+, --).
* Hamiltonians are written with Pauli matrices (not spin-1/2 operators).
* RBM parameters: a in F^N, b in F^M, W in F^{M x N} (row-major, W[j, i]
  couples hidden unit j to site i), F = R or C.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

# --------------------------------------------------------------------------
# Lattices (Sec. 2.2.1: Hypercube graph, edge colours of CustomGraph)
# --------------------------------------------------------------------------


def chain_bonds(n: int) -> np.ndarray:
    """Nearest-neighbour bonds of a periodic chain of n sites: (i, i+1 mod n)."""
    i = np.arange(n, dtype=np.int32)
    return np.stack([i, (i + 1) % n], axis=1).astype(np.int32)


def square_bonds(L: int) -> np.ndarray:
    """Nearest-neighbour (J1) bonds of an L x L periodic square lattice.

    Site s = x + L*y; bonds (x,y)-(x+1,y) then (x,y)-(x,y+1); 2*L*L bonds.
    """
    out = []
    for y in range(L):
        for x in range(L):
            s = x + L * y
            out.append((s, (x + 1) % L + L * y))
    for y in range(L):
        for x in range(L):
            s = x + L * y
            out.append((s, x + L * ((y + 1) % L)))
    return np.asarray(out, dtype=np.int32)


def chain_translations(n: int) -> np.ndarray:
    """Translation group of a periodic chain as a permutation table [n][n]:
    row g maps site i to (i + g) mod n (the lattice symmetries an
    ``RbmSpinSymm`` is built on, Sec. 2.2.2)."""
    i = np.arange(n, dtype=np.int64)
    return np.stack([(i + g) % n for g in range(n)]).astype(np.int32)


def square_translations(L: int) -> np.ndarray:
    """Translation group of an L x L periodic square lattice, [L*L][L*L]: row
    g = dx + L*dy maps site x + L*y to (x+dx mod L) + L*((y+dy) mod L)."""
    x = np.arange(L * L) % L
    y = np.arange(L * L) // L
    rows = [((x + dx) % L) + L * ((y + dy) % L) for dy in range(L) for dx in range(L)]
    return np.stack(rows).astype(np.int32)


@dataclass
class RbmSymmParams:
    """FP64 parameters of a symmetric RBM with ``alpha`` feature families:
    ``a`` [1] (one visible bias), ``b`` [alpha], ``w`` [alpha, N]."""

    a: np.ndarray
    b: np.ndarray
    w: np.ndarray

    @property
    def n(self) -> int:
        return int(self.w.shape[1])

    @property
    def alpha(self) -> int:
        return int(self.b.shape[0])

    @property
    def is_complex(self) -> bool:
        return np.iscomplexobj(self.w)

    @property
    def n_params(self) -> int:
        return 1 + self.alpha + self.alpha * self.n

    def flat(self) -> np.ndarray:
        """Parameter vector in the order (a, b, W row-major)."""
        return np.concatenate([self.a, self.b, self.w.reshape(-1)])

    @staticmethod
    def from_flat(x: np.ndarray, n: int, alpha: int) -> "RbmSymmParams":
        return RbmSymmParams(a=x[:1].copy(), b=x[1:1 + alpha].copy(),
                             w=x[1 + alpha:].reshape(alpha, n).copy())

    def copy(self) -> "RbmSymmParams":
        return RbmSymmParams(self.a.copy(), self.b.copy(), self.w.copy())


def init_symm_params(n: int, alpha: int, is_complex: bool, sigma: float = 0.01,
                     seed: int = 1234) -> RbmSymmParams:
    """Gaussian initialisation N(0, sigma^2) of every real component, as
    ``init_params``."""
    rng = np.random.default_rng(seed)

    def draw(shape):
        re = rng.normal(0.0, sigma, size=shape)
        if not is_complex:
            return re
        return re + 1j * rng.normal(0.0, sigma, size=shape)

    return RbmSymmParams(a=draw(1), b=draw(alpha), w=draw((alpha, n)))


def square_diag_bonds(L: int) -> np.ndarray:
    """Next-nearest-neighbour (J2, colour 1) bonds of an L x L periodic lattice.

    (x,y)-(x+1,y+1) then (x,y)-(x+1,y-1); 2*L*L bonds.
    """
    out = []
    for y in range(L):
        for x in range(L):
            s = x + L * y
            out.append((s, (x + 1) % L + L * ((y + 1) % L)))
    for y in range(L):
        for x in range(L):
            s = x + L * y
            out.append((s, (x + 1) % L + L * ((y - 1) % L)))
    return np.asarray(out, dtype=np.int32)


def sublattice(n: int, L: int | None = None) -> np.ndarray:
    """Bipartite sublattice label (0 = A, 1 = B): parity of x (+ y in 2D)."""
    if L is None:
        return (np.arange(n) % 2).astype(np.int32)
    s = np.arange(n)
    return ((s % L + s // L) % 2).astype(np.int32)


# --------------------------------------------------------------------------
# Operators in the GraphOperator format (Sec. 2.2.1)
# --------------------------------------------------------------------------

_X = np.array([[0, 1], [1, 0]], dtype=np.complex128)
_Y = np.array([[0, -1j], [1j, 0]], dtype=np.complex128)
# Z in the basis (up, down) = (+1, -1)
_Z = np.array([[1, 0], [0, -1]], dtype=np.complex128)


@dataclass
class Operator:
    """A Hamiltonian as a list of 1-local site terms and 2-local bond terms.

    ``site_idx[t]`` / ``site_mat[t]`` (2x2) and ``bond_i[t], bond_k[t]`` /
    ``bond_mat[t]`` (4x4), complex128, conventions in the module docstring.
    """

    n: int
    site_idx: np.ndarray = field(default_factory=lambda: np.zeros(0, np.int32))
    site_mat: np.ndarray = field(default_factory=lambda: np.zeros((0, 2, 2), np.complex128))
    bond_i: np.ndarray = field(default_factory=lambda: np.zeros(0, np.int32))
    bond_k: np.ndarray = field(default_factory=lambda: np.zeros(0, np.int32))
    bond_mat: np.ndarray = field(default_factory=lambda: np.zeros((0, 4, 4), np.complex128))

    @property
    def n_site_terms(self) -> int:
        return int(self.site_idx.shape[0])

    @property
    def n_bond_terms(self) -> int:
        return int(self.bond_i.shape[0])


def ising(n: int, bonds: np.ndarray, h: float, J: float = 1.0) -> Operator:
    """Transverse-field Ising model H = -J sum_<ik> Z_i Z_k - h sum_i X_i."""
    zz = -J * np.kron(_Z, _Z)
    return Operator(
        n=n,
        site_idx=np.arange(n, dtype=np.int32),
        site_mat=np.repeat((-h * _X)[None], n, axis=0),
        bond_i=bonds[:, 0].astype(np.int32).copy(),
        bond_k=bonds[:, 1].astype(np.int32).copy(),
        bond_mat=np.repeat(zz[None], len(bonds), axis=0),
    )


def heisenberg_bond(J: float, marshall: bool) -> np.ndarray:
    """J (X X + Y Y + Z Z) on one bond; with the Marshall rotation of one
    endpoint (a pi rotation about z of sublattice B) the exchange part flips sign."""
    m = J * (np.kron(_X, _X) + np.kron(_Y, _Y) + np.kron(_Z, _Z))
    if marshall:
        m = m.copy()
        m[1, 2] *= -1
        m[2, 1] *= -1
    return m


def heisenberg(n: int, bonds: np.ndarray, J: float = 1.0, marshall: bool = False,
               sub: np.ndarray | None = None) -> Operator:
    """Heisenberg model H = J sum_<ik> (XX + YY + ZZ), optionally Marshall-rotated
    on the bonds that join different sublattices."""
    mats = []
    for (i, k) in bonds:
        rot = marshall and (sub is None or sub[i] != sub[k])
        mats.append(heisenberg_bond(J, rot))
    return Operator(n=n, bond_i=bonds[:, 0].astype(np.int32).copy(),
                    bond_k=bonds[:, 1].astype(np.int32).copy(),
                    bond_mat=np.asarray(mats, dtype=np.complex128))


def j1j2(L: int, J1: float = 1.0, J2: float = 0.5, marshall: bool = True) -> Operator:
    """J1-J2 Heisenberg model on an L x L periodic square lattice; J1 bonds are
    colour 0 (Marshall-rotated), J2 diagonal bonds colour 1 (same sublattice)."""
    n = L * L
    sub = sublattice(n, L)
    b1 = square_bonds(L)
    b2 = square_diag_bonds(L)
    h1 = heisenberg(n, b1, J1, marshall, sub)
    h2 = heisenberg(n, b2, J2, marshall, sub)
    return Operator(n=n,
                    bond_i=np.concatenate([h1.bond_i, h2.bond_i]),
                    bond_k=np.concatenate([h1.bond_k, h2.bond_k]),
                    bond_mat=np.concatenate([h1.bond_mat, h2.bond_mat]))


# --------------------------------------------------------------------------
# RBM parameters and chain initial states
# --------------------------------------------------------------------------


@dataclass
class RbmParams:
    """FP64 RBM parameters. ``a`` [N], ``b`` [M], ``w`` [M, N] (complex128 or float64)."""

    a: np.ndarray
    b: np.ndarray
    w: np.ndarray

    @property
    def n(self) -> int:
        return int(self.a.shape[0])

    @property
    def m(self) -> int:
        return int(self.b.shape[0])

    @property
    def is_complex(self) -> bool:
        return np.iscomplexobj(self.w)

    @property
    def n_params(self) -> int:
        return self.n + self.m + self.n * self.m

    def flat(self) -> np.ndarray:
        """Parameter vector in the order (a, b, W row-major)."""
        return np.concatenate([self.a, self.b, self.w.reshape(-1)])

    @staticmethod
    def from_flat(x: np.ndarray, n: int, m: int) -> "RbmParams":
        return RbmParams(a=x[:n].copy(), b=x[n:n + m].copy(), w=x[n + m:].reshape(m, n).copy())

    def copy(self) -> "RbmParams":
        return RbmParams(self.a.copy(), self.b.copy(), self.w.copy())


def init_params(n: int, m: int, is_complex: bool, sigma: float = 0.01, seed: int = 1234) -> RbmParams:
    """Gaussian initialisation N(0, sigma^2) of every real component
    (``init_random_parameters(seed, sigma)`` in the VMC listing, Sec. 3.1).
    Complex parameters draw their real and imaginary parts independently."""
    rng = np.random.default_rng(seed)

    def draw(shape):
        re = rng.normal(0.0, sigma, size=shape)
        if not is_complex:
            return re
        im = rng.normal(0.0, sigma, size=shape)
        return re + 1j * im

    return RbmParams(a=draw(n), b=draw(m), w=draw((m, n)))


def ffnn_n_params(widths) -> int:
    """Parameters of a dense ln cosh network with layer widths [n, w_1, .., w_L]:
    W_l [w_l][w_(l-1)] and b_l [w_l] per layer."""
    return int(sum(widths[l] * (widths[l - 1] + 1) for l in range(1, len(widths))))


def init_ffnn_params(widths, is_complex: bool, sigma: float = 0.01, seed: int = 1234):
    """Flat FFNN parameters (layer by layer: W_l row-major, then b_l), every real
    component N(0, sigma^2) from a seeded generator."""
    rng = np.random.default_rng(seed)
    p = ffnn_n_params(widths)
    x = sigma * rng.normal(size=p)
    if is_complex:
        x = x + 1j * sigma * rng.normal(size=p)
    return x


def init_chains(nc: int, n: int, zero_magnetisation: bool, seed: int) -> np.ndarray:
    """Initial chain states, int8 [nc, n]: uniform +-1 spins, or a uniformly
    random arrangement of n/2 up and n/2 down spins (total S^z = 0 sector)."""
    rng = np.random.default_rng(seed)
    if not zero_magnetisation:
        return np.where(rng.random((nc, n)) < 0.5, 1, -1).astype(np.int8)
    if n % 2:
        raise ValueError("the S^z = 0 sector needs an even number of sites")
    base = np.array([1] * (n // 2) + [-1] * (n // 2), dtype=np.int8)
    out = np.empty((nc, n), dtype=np.int8)
    for c in range(nc):
        out[c] = rng.permutation(base)
    return out


def random_configs(ns: int, n: int, seed: int, zero_magnetisation: bool = False) -> np.ndarray:
    """Independent random configurations (for kernel parity tests)."""
    return init_chains(ns, n, zero_magnetisation, seed)


def perturb_params(p: RbmParams, scale: float, seed: int) -> RbmParams:
    """A structured (non-near-uniform) parameter state: p + N(0, scale^2) noise.
    Used to exercise amplitudes far from the uniform initial state."""
    rng = np.random.default_rng(seed)

    def noise(x):
        r = rng.normal(0.0, scale, size=x.shape)
        if np.iscomplexobj(x):
            r = r + 1j * rng.normal(0.0, scale, size=x.shape)
        return x + r

    return RbmParams(noise(p.a), noise(p.b), noise(p.w))


# --------------------------------------------------------------------------
# The five workloads
# --------------------------------------------------------------------------


@dataclass
class Workload:
    name: str
    n: int
    m: int
    is_complex: bool
    op: Operator
    move: str                 # "flip" or "exchange"
    sampler_bonds: np.ndarray  # bonds proposed by exchange moves
    zero_magnetisation: bool
    n_chains: int
    samples_per_chain: int
    n_discard: int
    diag_shift: float
    lr: float
    n_cg: int
    seed: int
    group_size: int = 8
    lattice: str = "chain"    # "chain" or "square" (periodic), for its translation group

    @property
    def n_samples(self) -> int:
        return self.n_chains * self.samples_per_chain

    @property
    def n_params(self) -> int:
        return self.n + self.m + self.n * self.m


def workload(name: str, n_chains: int | None = None, samples_per_chain: int | None = None) -> Workload:
    """The five workloads: c1 TFIM N=10; c2 Heisenberg N=40; c3 2D TFIM 10x10;
    c5 J1-J2 20x20 (c4, the batched mixture, is built by ``batched_instances``)."""
    if name == "c1":
        n = 10
        w = Workload("tfim1d_n10_alpha1", n, 10, False, ising(n, chain_bonds(n), h=1.0), "flip",
                     chain_bonds(n), False, 16, 63, 7, 0.01, 0.01, 120, 1234)
    elif name == "c2":
        n = 40
        w = Workload("heisenberg1d_n40_alpha2", n, 80, True,
                     heisenberg(n, chain_bonds(n), 1.0, True, sublattice(n)), "exchange",
                     chain_bonds(n), True, 4096, 4, 1, 0.01, 0.01, 50, 1235)
    elif name == "c3":
        L = 10
        n = L * L
        w = Workload("tfim2d_10x10_alpha4", n, 4 * n, False, ising(n, square_bonds(L), h=3.04),
                     "flip", square_bonds(L), False, 16384, 1, 1, 0.01, 0.01, 50, 1236)
    elif name == "c5":
        L = 20
        n = L * L
        w = Workload("j1j2_20x20_alpha4", n, 4 * n, True, j1j2(L, 1.0, 0.5, True), "exchange",
                     square_bonds(L), True, 16384, 4, 1, 0.01, 0.01, 50, 1237)
    else:
        raise KeyError(name)
    if name in ("c3", "c5"):
        w.lattice = "square"
    if n_chains is not None:
        w.n_chains = n_chains
    if samples_per_chain is not None:
        w.samples_per_chain = samples_per_chain
    return w


def translations(w: Workload) -> np.ndarray:
    """Translation group of a workload's periodic lattice (permutation table)."""
    if w.lattice == "square":
        L = int(round(math.sqrt(w.n)))
        return square_translations(L)
    return chain_translations(w.n)


def batched_instances(n_inst: int = 64, seed: int = 4242, n_chains: int = 1024):
    """Uneven independent 1D problems: N uniform in [16, 100] (even N for the
    Heisenberg instances, which need the S^z = 0 sector), alpha in {1, 2, 4}."""
    rng = np.random.default_rng(seed)
    out = []
    for t in range(n_inst):
        heis = bool(rng.integers(0, 2))
        n = int(rng.integers(16, 101))
        if heis and n % 2:
            n += -1 if n == 100 else 1
        alpha = int(rng.choice([1, 2, 4]))
        m = alpha * n
        if heis:
            op = heisenberg(n, chain_bonds(n), 1.0, True, sublattice(n))
            w = Workload(f"inst{t}_heis_n{n}_a{alpha}", n, m, True, op, "exchange", chain_bonds(n),
                         True, n_chains, 4, 1, 0.01, 0.01, 50, seed + t)
        else:
            op = ising(n, chain_bonds(n), h=1.0)
            w = Workload(f"inst{t}_tfim_n{n}_a{alpha}", n, m, False, op, "flip", chain_bonds(n),
                         False, n_chains, 4, 1, 0.01, 0.01, 50, seed + t)
        out.append(w)
    return out


def n_discard_default(samples_per_chain: int) -> int:
    """Burn-in sweeps per iteration: ceil(0.1 * samples per chain), at least 1."""
    return max(1, math.ceil(0.1 * samples_per_chain))
