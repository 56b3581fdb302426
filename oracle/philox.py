"""Philox4x32-10 (Salmon, Moraes, Dror, Shaw, "Parallel random numbers: as easy
as 1, 2, 3", SC'11), written from its published definition, vectorised with numpy.

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__``).

Definition: a 128-bit counter (c0, c1, c2, c3) and a 64-bit key (k0, k1).
One round computes the two 32x32->64 products of c0 and c2 with the
multipliers M0, M1 and outputs (hi(M1*c2) ^ c1 ^ k0, lo(M1*c2),
hi(M0*c0) ^ c3 ^ k1, lo(M0*c0)).  Between rounds the key is bumped by the Weyl
constants (W0, W1).  Ten rounds.

Streams used by the Metropolis sampler (the paper names no generator; this is
the reading this project adopts, identical on both sides):
  key     = (seed mod 2^32, seed >> 32)
  counter = (index, step mod 2^32, step >> 32, tag)
with ``index`` the chain group (tag SITE) or the chain (tag ACCEPT), and
``step`` the chain's global proposal counter.
"""
from __future__ import annotations

import numpy as np

M0 = np.uint64(0xD2511F53)
M1 = np.uint64(0xCD9E8D57)
W0 = np.uint64(0x9E3779B9)
W1 = np.uint64(0xBB67AE85)
MASK32 = np.uint64(0xFFFFFFFF)

TAG_SITE = 0x53495445    # proposal (site or bond) draw, one per chain group and step
TAG_ACCEPT = 0x41434350  # accept/reject uniform, one per chain and step
TAG_SWAP = 0x53574150    # replica-exchange uniform, one per replica and sweep


def philox4x32_10(c0, c1, c2, c3, k0, k1):
    """Apply Philox4x32-10 to arrays of counters; returns four uint32 arrays."""
    c0 = np.asarray(c0, dtype=np.uint64) & MASK32
    c1 = np.asarray(c1, dtype=np.uint64) & MASK32
    c2 = np.asarray(c2, dtype=np.uint64) & MASK32
    c3 = np.asarray(c3, dtype=np.uint64) & MASK32
    k0 = np.asarray(k0, dtype=np.uint64) & MASK32
    k1 = np.asarray(k1, dtype=np.uint64) & MASK32
    for r in range(10):
        if r > 0:
            k0 = (k0 + W0) & MASK32
            k1 = (k1 + W1) & MASK32
        p0 = M0 * c0  # < 2^64: exact in uint64
        p1 = M1 * c2
        hi0, lo0 = p0 >> np.uint64(32), p0 & MASK32
        hi1, lo1 = p1 >> np.uint64(32), p1 & MASK32
        c0, c1, c2, c3 = hi1 ^ c1 ^ k0, lo1, hi0 ^ c3 ^ k1, lo0
    return (c0.astype(np.uint32), c1.astype(np.uint32),
            c2.astype(np.uint32), c3.astype(np.uint32))


def key_of(seed: int):
    seed = int(seed) & 0xFFFFFFFFFFFFFFFF
    return seed & 0xFFFFFFFF, seed >> 32


def draw(index, step: int, tag: int, seed: int):
    """The 4 x uint32 block of stream (index, step, tag) under ``seed``."""
    k0, k1 = key_of(seed)
    index = np.asarray(index, dtype=np.uint64)
    step = int(step)
    return philox4x32_10(index, step & 0xFFFFFFFF, step >> 32, tag, k0, k1)


def uniform_index(u32, n: int):
    """floor(u * n / 2^32): index in [0, n) by the multiply-shift map (the bias,
    at most n / 2^32, is accepted)."""
    return ((np.asarray(u32, dtype=np.uint64) * np.uint64(n)) >> np.uint64(32)).astype(np.int64)


def uniform53(u_hi, u_lo):
    """Double in [0, 1) from 27 high bits of ``u_hi`` and 26 of ``u_lo``."""
    a = (np.asarray(u_hi, dtype=np.uint64) >> np.uint64(5)).astype(np.float64)
    b = (np.asarray(u_lo, dtype=np.uint64) >> np.uint64(6)).astype(np.float64)
    return (a * 67108864.0 + b) * (1.0 / 9007199254740992.0)
