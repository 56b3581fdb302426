"""One VMC + SR iteration in the order of Sec. 2.2.5 (sample -> local energies
-> statistics -> log-derivatives and force -> SR solve -> SGD update), FP64.

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__``).

``full_sum=True`` replaces the Monte Carlo average by the exact expectation over
every configuration of the Hilbert space (or its S^z = 0 sector) with weights
|psi|^2 / Z (Eq. 4): a deterministic SR trajectory for small N.
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np

from paper_1904_00031_gb300.workloads import RbmParams

from . import hamiltonian, local_energy, rbm, sampler, sr


@dataclass
class ChainState:
    sigma: np.ndarray  # [nc, N] int8
    counter: int


def vmc_sr_iteration(p: RbmParams, op, chains: ChainState, *, move: str, bonds, group_size: int,
                     seed: int, n_discard: int, samples_per_chain: int, diag_shift: float,
                     lr: float, n_cg: int | None, cg_rtol: float = 1e-12,
                     full_sum_basis: np.ndarray | None = None):
    """Returns (new params, new chain state, info dict)."""
    real = not p.is_complex
    if full_sum_basis is None:
        samples, final, counter, n_acc = sampler.metropolis(
            p, chains.sigma, move, bonds, group_size, seed, chains.counter, n_discard,
            samples_per_chain)
        new_chains = ChainState(final, counter)
        weights = None
        acc = float(n_acc.sum()) / (len(final) * (n_discard + samples_per_chain) * p.n)
        nc = len(final)
    else:
        samples = full_sum_basis
        weights = sampler.exact_distribution(p, samples)
        new_chains = chains
        acc = float("nan")
        nc = None
    eloc = local_energy.local_energy_rbm(p, op, samples)
    if weights is None:
        # independent units of the error bar: whole proposal groups
        blocks = nc // group_size if nc % group_size == 0 else 1
        mean, var, err = sr.stats(eloc, blocks)
    else:
        mean = complex(weights @ eloc)
        var = float(weights @ np.abs(eloc - mean) ** 2)
        err = 0.0
    sig, t = rbm.logderiv_factored(p, samples)
    f = sr.force_lazy(sig, t, eloc, p.n, p.m, weights, real)
    if n_cg is None:
        o = rbm.logderiv_dense(p, samples)
        s, _ = sr.sr_matrices(o, eloc, weights, real)
        delta = sr.solve_dense(s, f, diag_shift)
        iters, resid = 0, 0.0
    else:
        delta, iters, resid = sr.cg(
            lambda x: sr.sr_matvec_lazy(sig, t, x, p.n, p.m, weights, real), f, diag_shift,
            n_cg, cg_rtol)
    newflat = sr.sgd_update(p.flat(), delta, lr)
    newp = RbmParams.from_flat(newflat, p.n, p.m)
    info = dict(energy=mean.real, energy_imag=mean.imag, variance=var, error=err,
                acceptance=acc, cg_iters=iters, cg_resid=resid)
    return newp, new_chains, info


def exact_energy_of(p: RbmParams, op, zero_magnetisation: bool) -> float:
    """<psi|H|psi>/<psi|psi> of the RBM by enumeration and the sparse matrix."""
    xs = hamiltonian.basis(p.n, zero_magnetisation)
    cf = hamiltonian.configs(xs, p.n)
    lp = rbm.logpsi(p, cf)
    psi = np.exp(lp - np.max(np.real(lp)))
    h = hamiltonian.sparse_h(op, xs)
    return float(np.real(np.vdot(psi, h @ psi) / np.vdot(psi, psi)))
