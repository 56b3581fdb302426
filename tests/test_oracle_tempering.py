"""Pins of the parallel-tempering oracle (Sec. 2.2.5; replica exchange):
one replica reduces to the plain Metropolis sampler bit for bit; the exchange
step leaves the product of the replicas' tempered distributions exactly
stationary (its transition matrix, enumerated on a 3-site system); and long
runs reproduce |psi|^(2 beta_r) / Z_r in every replica of the ladder."""
import itertools

import numpy as np
import pytest

from oracle import hamiltonian, rbm, sampler, tempering
from paper_1904_00031_gb300 import workloads as W


@pytest.mark.parametrize("move", ["flip", "exchange"])
def test_one_replica_is_the_plain_sampler(move):
    n = 8
    p = W.init_params(n, 8, True, sigma=0.2, seed=3)
    s0 = W.init_chains(64, n, move == "exchange", 5)
    a = sampler.metropolis(p, s0, move, W.chain_bonds(n), 8, 77, 11, 2, 3)
    b = tempering.parallel_tempering(p, s0, 1, move, W.chain_bonds(n), 8, 77, 11, 0, 2, 3)
    assert np.array_equal(a[0], b[0]) and np.array_equal(a[1], b[1])
    assert a[2] == b[2] and np.array_equal(a[3], b[3]) and b[4].shape == (64, 0)


def _exchange_matrix(L, betas, parity, log_ratio):
    """Exact transition matrix of one exchange step over the joint states."""
    R = len(betas)
    states = list(itertools.product(range(len(L)), repeat=R))
    index = {s: k for k, s in enumerate(states)}
    T = np.zeros((len(states), len(states)))
    for s in states:
        cur = {s: 1.0}
        for r in range(parity, R - 1, 2):
            nxt = {}
            for st, pr in cur.items():
                a = min(1.0, np.exp(log_ratio(betas[r], betas[r + 1], L[st[r]], L[st[r + 1]])))
                sw = list(st)
                sw[r], sw[r + 1] = sw[r + 1], sw[r]
                nxt[tuple(sw)] = nxt.get(tuple(sw), 0.0) + pr * a
                nxt[st] = nxt.get(st, 0.0) + pr * (1.0 - a)
            cur = nxt
        for st, pr in cur.items():
            T[index[s], index[st]] += pr
    return states, T


def test_exchange_step_keeps_the_tempered_product_stationary():
    n, R = 3, 3
    p = W.init_params(n, 4, True, sigma=0.6, seed=8)
    cf = np.array(list(itertools.product([1, -1], repeat=n)), dtype=np.int8)
    L = 2.0 * np.real(rbm.logpsi(p, cf))
    betas = tempering.ladder(R)
    assert np.allclose(betas, [1.0, 2.0 / 3.0, 1.0 / 3.0])
    for parity in (0, 1):
        states, T = _exchange_matrix(L, betas, parity, tempering.swap_log_ratio)
        pi = np.array([np.exp(sum(betas[r] * L[s[r]] for r in range(R))) for s in states])
        pi /= pi.sum()
        assert np.allclose(T.sum(axis=1), 1.0)
        assert np.abs(pi @ T - pi).max() < 1e-14
        # the exchange ratio with its sign flipped is not stationary: the check has teeth
        _, Tb = _exchange_matrix(L, betas, parity, lambda *a: -tempering.swap_log_ratio(*a))
        assert np.abs(pi @ Tb - pi).max() > 1e-4


@pytest.mark.parametrize("move", ["flip", "exchange"])
def test_every_replica_samples_its_tempered_distribution(move):
    n, R, nc = 6, 3, 2048
    sz = move == "exchange"
    p = W.init_params(n, 6, True, sigma=0.35, seed=31)
    xs = hamiltonian.basis(n, sz)
    cf = hamiltonian.configs(xs, n)
    L = 2.0 * np.real(rbm.logpsi(p, cf))
    s0 = W.init_chains(nc * R, n, sz, 12)
    _, fin, _, _, n_swap = tempering.parallel_tempering(p, s0, R, move, W.chain_bonds(n), 8,
                                                        2024, 0, 0, 60, 0)
    assert n_swap.sum() > 0
    betas = tempering.ladder(R)
    for r in range(R):
        target = np.exp(betas[r] * (L - L.max()))
        target /= target.sum()
        ints = ((1 - fin[r::R].astype(np.int64)) // 2) @ (1 << np.arange(n))
        c = np.bincount(np.searchsorted(xs, ints), minlength=len(xs)).astype(np.float64)
        exp = target * nc
        chi2 = np.sum((c - exp) ** 2 / exp)
        dof = len(xs) - 1
        assert chi2 < dof + 5 * np.sqrt(2 * dof), (r, chi2, dof)
    # the ladder's distributions differ enough for the check to tell them apart
    t0 = np.exp(L - L.max())
    t2 = np.exp(betas[2] * (L - L.max()))
    assert np.abs(t0 / t0.sum() - t2 / t2.sum()).max() > 0.02
