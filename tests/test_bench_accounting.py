"""The bench's work accounting, on the CPU: the mean number of connected
configurations per sample (the local-energy terms whose FLOPs the roofline of
the local-energy stage counts) equals a brute-force count of the nonzero
off-diagonal entries <sigma'|H|sigma> of the Hamiltonian's sparse matrix, and the
stage FLOP counts scale as their formulas say."""
import numpy as np
import pytest

import bench
from oracle import hamiltonian
from paper_1904_00031_gb300 import workloads as W


def brute_connected(op, n, zero_magnetisation):
    xs = hamiltonian.basis(n, zero_magnetisation)
    h = hamiltonian.sparse_h(op, xs).tocsc()
    h.eliminate_zeros()
    counts = np.diff(h.indptr) - (h.diagonal() != 0)  # nonzero entries of column sigma, off the diagonal
    return hamiltonian.configs(xs, n), counts


@pytest.mark.parametrize("name", ["tfim8", "heis8", "j1j2_4x4"])
def test_connected_per_config_matches_brute_force(name):
    if name == "tfim8":
        n, zm = 8, False
        op = W.ising(n, W.chain_bonds(n), h=1.0)
    elif name == "heis8":
        n, zm = 8, True
        op = W.heisenberg(n, W.chain_bonds(n), 1.0, True, W.sublattice(n))
    else:
        n, zm = 16, True
        op = W.j1j2(4)
    sm, counts = brute_connected(op, n, zm)
    rng = np.random.default_rng(3)
    pick = rng.choice(len(sm), size=min(len(sm), 300), replace=False)
    got = bench.connected_per_config(op, sm[pick])
    assert got == pytest.approx(float(counts[pick].mean()), rel=0, abs=1e-12)
    # per configuration as well (a batch of one)
    for q in pick[:20]:
        assert bench.connected_per_config(op, sm[q:q + 1]) == counts[q]


def test_tfim_connects_every_single_flip():
    # a transverse field connects sigma to each of its n single-spin flips
    n = 10
    op = W.ising(n, W.chain_bonds(n), h=0.7)
    sm = W.random_configs(50, n, 1)
    assert bench.connected_per_config(op, sm) == n


def test_stage_flops_formulas():
    w = W.workload("c5")
    f = bench.stage_flops(w, n_nonnull=100.0, n_accept=40.0, n_connected=800.0)
    m, n, ns = w.m, w.n, w.n_samples
    assert f["sample"] == m * (12 * 100.0 + 32 * 40.0)
    assert f["energies"] == ns * 800.0 * m * 14
    assert f["amplitudes"] == ns * 4 * n * m
    assert f["sr"] == ns * 4 * n * m * (2 * w.n_cg + 1)
    # linear in each count
    g = bench.stage_flops(w, n_nonnull=200.0, n_accept=80.0, n_connected=1600.0)
    for k in ("sample", "energies"):
        assert g[k] == pytest.approx(2 * f[k])
