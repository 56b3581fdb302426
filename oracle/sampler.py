"""Metropolis sampling of |psi(sigma)|^2 (Eq. 4; Sec. 2.2.5: Markov chains built by
the Metropolis algorithm so that detailed balance holds) with single-spin-flip
moves or the nearest-neighbour exchange moves of the VMC listing (Sec. 3.1),
which keep the total magnetisation.

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__``).

The algorithm, step by step (readings of silent points marked [r]):
1. theta = W sigma + b for each chain's current state.
2. A sweep is N proposals [r].  The chain's global step counter numbers the
   proposals.
3. Proposal of step t: one Philox draw per *group* of ``group_size`` chains
   (stream (group, t, SITE)) picks a site i = floor(u N / 2^32) (flip) or a bond
   b = floor(u n_bonds / 2^32) from the exchange bond list [r: the proposal
   index is shared by the chains of a group; every chain still runs a Metropolis
   chain with a uniformly random proposal and keeps detailed balance].
   An exchange of two equal spins is a null move, counted as rejected [r].
4. Log-ratio Delta = ln psi(sigma') - ln psi(sigma) with sigma' the proposal:
   -2 a_i sigma_i (each flipped site) + sum_j [ln cosh theta'_j - ln cosh theta_j],
   theta' = theta - 2 sigma_i W[:, i] (each flipped site).
5. Accept iff U < exp(2 Re Delta), U uniform in [0, 1) from stream
   (chain, t, ACCEPT) [r: strict inequality].  On accept sigma <- sigma',
   theta <- theta'.
6. n_discard burn-in sweeps, then one recorded sample per sweep.  Samples are
   returned chain-major: row c * n_samples + s.
"""
from __future__ import annotations

import numpy as np

from . import philox, rbm


def metropolis(p, sigma0, move: str, bonds, group_size: int, seed: int, counter: int,
               n_discard: int, n_samples: int, return_margin: bool = False, betas=None):
    """Run every chain (rows of ``sigma0``) for n_discard + n_samples sweeps.

    Returns (samples [nc * n_samples, N] int8, final states [nc, N] int8,
    new counter, accepted count per chain [nc]) and, if ``return_margin``, the
    smallest |ln U - 2 Re Delta| over the chain's non-null proposals (how close
    an accept decision came to a tie), for trajectory comparisons.

    ``betas`` [nc] (parallel tempering): chain c samples |psi|^(2 beta_c) and
    accepts iff U < exp(2 beta_c Re Delta); None is beta = 1 for every chain."""
    sigma = np.array(sigma0, dtype=np.int8, copy=True)
    nc, n = sigma.shape
    sig = sigma.astype(np.float64)
    th = rbm.theta(p, sig)
    lc = rbm.lncosh(th)
    chains = np.arange(nc)
    groups = chains // group_size
    n_acc = np.zeros(nc, dtype=np.int64)
    margin = np.full(nc, np.inf)
    samples = np.zeros((nc, n_samples, n), dtype=np.int8)
    bonds = np.asarray(bonds, dtype=np.int64)
    for sweep in range(n_discard + n_samples):
        for q in range(n):
            t = counter + sweep * n + q
            u_site = philox.draw(groups, t, philox.TAG_SITE, seed)[0]
            u_acc = philox.draw(chains, t, philox.TAG_ACCEPT, seed)
            U = philox.uniform53(u_acc[0], u_acc[1])
            if move == "flip":
                i = philox.uniform_index(u_site, n)
                si = sig[chains, i]
                dlog = -2.0 * p.a[i] * si
                thp = th - (2.0 * si)[:, None] * p.w[:, i].T
                valid = np.ones(nc, dtype=bool)
            else:
                b = philox.uniform_index(u_site, len(bonds))
                i, k = bonds[b, 0], bonds[b, 1]
                si, sk = sig[chains, i], sig[chains, k]
                valid = si != sk
                dlog = -2.0 * p.a[i] * si - 2.0 * p.a[k] * sk
                thp = th - (2.0 * si)[:, None] * p.w[:, i].T - (2.0 * sk)[:, None] * p.w[:, k].T
            lcp = rbm.lncosh(thp)
            dlog = dlog + (lcp - lc).sum(axis=1)
            two_re = 2.0 * np.real(dlog)
            if betas is not None:
                two_re = np.asarray(betas, dtype=np.float64) * two_re
            with np.errstate(over="ignore"):
                acc = valid & (U < np.exp(two_re))
            if return_margin:
                with np.errstate(divide="ignore"):
                    m = np.abs(np.log(U) - two_re)
                m = np.where(valid, m, np.inf)
                margin = np.minimum(margin, m)
            sig[acc, i[acc]] *= -1.0
            if move != "flip":
                sig[acc, k[acc]] *= -1.0
            th[acc] = thp[acc]
            lc[acc] = lcp[acc]
            n_acc += acc
        if sweep >= n_discard:
            samples[:, sweep - n_discard] = sig.astype(np.int8)
    out = (samples.reshape(nc * n_samples, n), sig.astype(np.int8),
           counter + (n_discard + n_samples) * n, n_acc)
    if return_margin:
        return out + (margin,)
    return out


def exact_distribution(p, xs_configs):
    """|psi|^2 / Z over an enumerated set of configurations (Eq. 4)."""
    lp = rbm.logpsi(p, xs_configs)
    w = np.exp(2.0 * (np.real(lp) - np.max(np.real(lp))))
    return w / w.sum()
