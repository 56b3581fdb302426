"""Parallel tempering (replica exchange) over |psi|^2: the sampler option the
paper names to improve sampling efficiency (Sec. 2.2.5, after Swendsen and
Wang's replica Monte Carlo).

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__``).

The paper names the option and nothing more.  Readings [r]:
* each Markov chain is a ladder of R replicas at inverse temperatures
  beta_r = 1 - r / R (r = 0 .. R-1), replica r sampling |psi|^(2 beta_r); the
  beta = 1 replica is the physical one, and only its states are recorded;
* the replicas are numbered chain-major, replica c R + r, and each runs the
  Metropolis sweep of ``sampler`` (same proposals and Philox streams, with
  replica index in place of chain index) at its own beta;
* after every sweep, neighbouring replicas (r, r + 1) exchange states, over
  the pairs starting at r = 0 on even sweeps and r = 1 on odd ones, with
  probability min(1, exp((beta_r - beta_(r+1)) (L(sigma_(r+1)) - L(sigma_r)))),
  L = 2 Re ln psi, which keeps prod_r |psi(sigma_r)|^(2 beta_r) stationary; the
  uniform of pair (r, r + 1) is drawn from stream (replica c R + r, sweep,
  SWAP), accepted iff U < that ratio (strict, as the Metropolis test);
* a sweep of the ladder counts as one sweep of the chain.
"""
from __future__ import annotations

import numpy as np

from . import philox, rbm, sampler


def ladder(n_replicas: int) -> np.ndarray:
    """beta_r = 1 - r / R."""
    return 1.0 - np.arange(n_replicas, dtype=np.float64) / n_replicas


def swap_log_ratio(beta_r, beta_s, l_r, l_s):
    """ln of the exchange ratio of replicas (r, s) holding L values (l_r, l_s)."""
    return (beta_r - beta_s) * (l_s - l_r)


def parallel_tempering(p, sigma0, n_replicas: int, move: str, bonds, group_size: int,
                       seed: int, counter: int, sweep0: int, n_discard: int, n_samples: int,
                       return_margin: bool = False):
    """Run every ladder (rows c R .. c R + R - 1 of ``sigma0``) for n_discard +
    n_samples sweeps.  ``sweep0`` numbers the first sweep (exchange parity and
    SWAP streams).  Returns (samples [nc * n_samples, N] of the beta = 1
    replicas, final replica states [nc R, N], new counter, accepted moves per
    replica [nc R], accepted exchanges per pair [nc, R - 1]) and, if
    ``return_margin``, per ladder the smallest distance to a tie of any of its
    decisions (|ln U - beta 2 Re Delta| of its replicas' moves, |ln U - ln ratio|
    of its exchanges), for trajectory comparisons."""
    sig = np.array(sigma0, dtype=np.int8, copy=True)
    nrep, n = sig.shape
    R = n_replicas
    nc = nrep // R
    betas = np.tile(ladder(R), nc)
    samples = np.zeros((nc, n_samples, n), dtype=np.int8)
    n_acc = np.zeros(nrep, dtype=np.int64)
    n_swap = np.zeros((nc, max(R - 1, 0)), dtype=np.int64)
    margin = np.full(nc, np.inf)
    for k in range(n_discard + n_samples):
        out = sampler.metropolis(p, sig, move, bonds, group_size, seed, counter, 1, 0,
                                 betas=betas, return_margin=return_margin)
        _, sig, counter, acc = out[:4]
        if return_margin:
            margin = np.minimum(margin, out[4].reshape(nc, R).min(axis=1))
        n_acc += acc
        sweep = sweep0 + k
        lval = 2.0 * np.real(rbm.logpsi(p, sig))
        for r in range(sweep % 2, R - 1, 2):
            lo = np.arange(nc) * R + r
            hi = lo + 1
            u = philox.draw(lo, sweep, philox.TAG_SWAP, seed)
            U = philox.uniform53(u[0], u[1])
            lr = swap_log_ratio(betas[lo], betas[hi], lval[lo], lval[hi])
            with np.errstate(over="ignore"):
                ok = U < np.exp(lr)
            if return_margin:
                margin = np.minimum(margin, np.abs(np.log(U) - lr))
            a, b = sig[lo[ok]].copy(), sig[hi[ok]].copy()
            sig[lo[ok]], sig[hi[ok]] = b, a
            la, lb = lval[lo[ok]].copy(), lval[hi[ok]].copy()
            lval[lo[ok]], lval[hi[ok]] = lb, la
            n_swap[:, r] += ok
        if k >= n_discard:
            samples[:, k - n_discard] = sig[np.arange(nc) * R]
    out = (samples.reshape(nc * n_samples, n), sig, counter, n_acc, n_swap)
    return out + (margin,) if return_margin else out
