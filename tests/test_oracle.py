"""Pins of the FP64 oracle against things other than itself: published
known-answer vectors, closed forms, textbook ground energies, exact
diagonalisation, finite differences, library routines and brute force."""
import itertools
import os

import numpy as np
import pytest

from oracle import hamiltonian, local_energy, philox, rbm, sampler, sr, vmc
from paper_1904_00031_gb300 import workloads as W

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _rows(name):
    with open(os.path.join(GOLDEN, name)) as f:
        for line in f:
            line = line.strip()
            if line and not line.startswith("#"):
                yield line.split()


# ---------------------------------------------------------------- Philox

def test_philox_known_answers():
    rows = list(_rows("philox4x32_10_kat.txt"))
    assert len(rows) == 3
    for r in rows:
        v = [int(x, 16) for x in r]
        out = philox.philox4x32_10(*v[:6])
        assert [int(o) for o in out] == v[6:]


def test_philox_vectorised_matches_scalar_and_draw_streams():
    idx = np.arange(5)
    a = philox.draw(idx, 123456789012, philox.TAG_ACCEPT, 0x1234567890ABCDEF)
    for c in range(5):
        b = philox.philox4x32_10(c, 123456789012 & 0xFFFFFFFF, 123456789012 >> 32,
                                 philox.TAG_ACCEPT, 0x90ABCDEF, 0x12345678)
        assert [int(x[c]) for x in a] == [int(x) for x in b]


def test_uniform_maps():
    u = np.array([0, 0xFFFFFFFF, 0x80000000], dtype=np.uint32)
    assert list(philox.uniform_index(u, 10)) == [0, 9, 5]
    assert philox.uniform53(0xFFFFFFFF, 0xFFFFFFFF) < 1.0
    assert philox.uniform53(0, 0) == 0.0
    # equidistribution of indices: chi-square over 10 bins, 200k draws
    d = philox.draw(np.arange(200000), 7, philox.TAG_SITE, 99)[0]
    h = np.bincount(philox.uniform_index(d, 10), minlength=10)
    chi2 = np.sum((h - 20000.0) ** 2 / 20000.0)
    assert chi2 < 35.0  # p ~ 1e-4 for 9 dof
    uu = philox.uniform53(*philox.draw(np.arange(200000), 7, philox.TAG_ACCEPT, 99)[:2])
    assert abs(uu.mean() - 0.5) < 0.005 and uu.min() >= 0.0 and uu.max() < 1.0


# ---------------------------------------------------------------- Hamiltonians

def test_golden_ground_energies():
    for model, n, J, h, e0, *_ in _rows("ground_energies.txt"):
        n, J, h, e0 = int(n), float(J), float(h), float(e0)
        if model == "tfim_chain":
            op = W.ising(n, W.chain_bonds(n), h=h, J=J)
            assert abs(hamiltonian.tfim_chain_ground(n, J, h) - e0) < 1e-9
            assert abs(hamiltonian.exact_ground(op)[0] - e0) < 1e-9
        else:
            op = W.heisenberg(n, W.chain_bonds(n), J)
            assert abs(hamiltonian.exact_ground(op)[0] - e0) < 1e-9


@pytest.mark.parametrize("n,h", [(6, 0.5), (8, 3.04), (10, 1.0), (12, 1.7)])
def test_tfim_closed_form(n, h):
    op = W.ising(n, W.chain_bonds(n), h=h)
    e_ed = hamiltonian.lanczos_ground(op)[0] if n > 10 else hamiltonian.exact_ground(op)[0]
    assert abs(e_ed - hamiltonian.tfim_chain_ground(n, 1.0, h)) < 1e-9


def test_sign_conventions_do_not_change_spectrum():
    n = 8
    bonds = W.chain_bonds(n)
    e = [hamiltonian.exact_ground(W.ising(n, bonds, h=hh, J=jj))[0]
         for hh, jj in [(1.3, 1.0), (-1.3, 1.0), (1.3, -1.0)]]
    assert np.allclose(e, e[0], atol=1e-10)
    sub = W.sublattice(n)
    e1 = hamiltonian.exact_ground(W.heisenberg(n, bonds, 1.0), True)[0]
    e2 = hamiltonian.exact_ground(W.heisenberg(n, bonds, 1.0, True, sub), True)[0]
    assert abs(e1 - e2) < 1e-10


def test_lanczos_matches_dense_and_sector():
    n = 12
    op = W.heisenberg(n, W.chain_bonds(n), 1.0, True, W.sublattice(n))
    e_full = hamiltonian.exact_ground(op)[0]
    e_sz = hamiltonian.lanczos_ground(op, True)[0]
    assert abs(e_full - e_sz) < 1e-9  # ground state of an even ring lies in S^z = 0


def test_j1j2_marshall_invariance_and_bonds():
    L = 4
    op = W.j1j2(L, 1.0, 0.5, True)
    assert op.n_bond_terms == 4 * L * L
    deg = np.bincount(np.concatenate([op.bond_i, op.bond_k]), minlength=L * L)
    assert np.all(deg == 8)
    sub = W.sublattice(L * L, L)
    assert np.all(sub[op.bond_i[:2 * L * L]] != sub[op.bond_k[:2 * L * L]])
    assert np.all(sub[op.bond_i[2 * L * L:]] == sub[op.bond_k[2 * L * L:]])
    op_u = W.j1j2(L, 1.0, 0.5, False)
    e1 = hamiltonian.lanczos_ground(op, True)[0]
    e2 = hamiltonian.lanczos_ground(op_u, True)[0]
    assert abs(e1 - e2) < 1e-8


# ---------------------------------------------------------------- RBM

def test_lncosh_against_library():
    rng = np.random.default_rng(0)
    x = rng.normal(0, 2, 1000)
    z = x + 1j * rng.normal(0, 1, 1000)
    assert np.allclose(rbm.lncosh(x), np.log(np.cosh(x)), rtol=1e-13, atol=1e-13)
    ref = np.log(np.cosh(z))
    got = rbm.lncosh(z)
    assert np.allclose(got.real, ref.real, atol=1e-12)
    d = np.angle(np.exp(1j * (got.imag - ref.imag)))  # compare phases mod 2 pi
    assert np.abs(d).max() < 1e-12
    big = np.array([800.0, -800.0, 800.0 + 3j])
    assert np.all(np.isfinite(rbm.lncosh(big)))
    assert abs(rbm.lncosh(np.array([800.0]))[0] - (800.0 - np.log(2))) < 1e-12


def _brute_logpsi(p, s):
    out = []
    for row in s:
        v = complex(np.dot(p.a, row))
        for j in range(p.m):
            th = p.b[j] + sum(p.w[j, i] * row[i] for i in range(p.n))
            v += np.log(np.cosh(complex(th)))
        out.append(v)
    return np.array(out)


@pytest.mark.parametrize("cplx", [False, True])
def test_rbm_special_cases(cplx):
    n, m = 6, 4
    s = W.random_configs(20, n, 1)
    p = W.init_params(n, m, cplx, sigma=0.3, seed=5)
    z = W.RbmParams(np.zeros_like(p.a), np.zeros_like(p.b), np.zeros_like(p.w))
    assert np.allclose(rbm.logpsi(z, s), 0.0)
    pw0 = W.RbmParams(p.a, p.b, np.zeros_like(p.w))
    assert np.allclose(rbm.logpsi(pw0, s), s @ p.a + np.log(np.cosh(p.b)).sum())
    pab0 = W.RbmParams(np.zeros_like(p.a), np.zeros_like(p.b), p.w)
    d = rbm.logpsi(pab0, s) - rbm.logpsi(pab0, -s)
    assert np.abs(np.angle(np.exp(d))).max() < 1e-12 and np.abs(d.real).max() < 1e-12
    p1 = W.init_params(n, 1, cplx, sigma=0.5, seed=6)
    ref = s @ p1.a + np.log(np.cosh(s @ p1.w[0] + p1.b[0]))
    got = rbm.logpsi(p1, s)
    assert np.allclose(got.real, np.real(ref)) and np.allclose(np.exp(1j * got.imag), np.exp(1j * np.imag(ref)))
    got = rbm.logpsi(p, s)
    ref = _brute_logpsi(p, s)
    assert np.allclose(got.real, ref.real, atol=1e-12)
    assert np.abs(np.angle(np.exp(1j * (got.imag - ref.imag)))).max() < 1e-12


@pytest.mark.parametrize("cplx", [False, True])
def test_logderiv_and_backward_by_finite_differences(cplx):
    n, m = 5, 7
    p = W.init_params(n, m, cplx, sigma=0.4, seed=11)
    s = W.random_configs(6, n, 2)
    o = rbm.logderiv_dense(p, s)
    x0 = p.flat()
    h = 1e-6
    fd = np.zeros_like(o)
    for k in range(len(x0)):
        e = np.zeros_like(x0)
        e[k] = h
        lp = rbm.logpsi(W.RbmParams.from_flat(x0 + e, n, m), s)
        lm = rbm.logpsi(W.RbmParams.from_flat(x0 - e, n, m), s)
        fd[:, k] = (lp - lm) / (2 * h)
    assert np.allclose(o, fd, rtol=1e-7, atol=1e-8)
    if cplx:  # holomorphic: derivative along i equals i * O
        k = n + 2
        e = np.zeros_like(x0)
        e[k] = 1j * h
        lp = rbm.logpsi(W.RbmParams.from_flat(x0 + e, n, m), s)
        lm = rbm.logpsi(W.RbmParams.from_flat(x0 - e, n, m), s)
        assert np.allclose((lp - lm) / (2 * h), 1j * o[:, k], rtol=1e-7, atol=1e-8)
    g = np.random.default_rng(3).normal(size=len(s))
    assert np.allclose(rbm.logpsi_backward(p, s, g), g @ fd, rtol=1e-7, atol=1e-8)


# ---------------------------------------------------------------- local energy

def test_local_energy_of_exact_eigenstate_is_constant():
    for op, sz in [(W.ising(8, W.chain_bonds(8), h=0.7), False),
                   (W.heisenberg(8, W.chain_bonds(8), 1.0, True, W.sublattice(8)), True)]:
        e0, v, xs = hamiltonian.exact_ground(op, sz)
        table = {int(x): complex(c) for x, c in zip(xs, v)}
        n = op.n

        def lookup(batch):
            ints = ((1 - batch.astype(np.int64)) // 2) @ (1 << np.arange(n))
            return np.log(np.array([table[int(i)] for i in ints], dtype=np.complex128))

        cf = hamiltonian.configs(xs, n)
        e = local_energy.local_energy_generic(lookup, op, cf)
        assert np.abs(e - e0).max() < 1e-9  # zero-variance property of an eigenstate


@pytest.mark.parametrize("which", ["tfim", "heis", "j1j2"])
def test_rbm_local_energy_update_form_equals_definition(which):
    if which == "tfim":
        op, sz, n = W.ising(7, W.chain_bonds(7), h=1.3), False, 7
    elif which == "heis":
        op, sz, n = W.heisenberg(8, W.chain_bonds(8), 1.0, True, W.sublattice(8)), True, 8
    else:
        op, sz, n = W.j1j2(4, 1.0, 0.5, True), True, 16
    p = W.init_params(n, 2 * n, True, sigma=0.3, seed=21)
    s = W.random_configs(40, n, 4, sz)
    a = local_energy.local_energy_rbm(p, op, s)
    b = local_energy.local_energy_generic(lambda x: rbm.logpsi(p, x), op, s)
    assert np.allclose(a, b, rtol=1e-11, atol=1e-11)


@pytest.mark.parametrize("cplx", [False, True])
def test_full_sum_energy_equals_rayleigh_quotient(cplx):
    n = 8
    op = W.heisenberg(n, W.chain_bonds(n), 1.0, True, W.sublattice(n))
    p = W.init_params(n, n, cplx, sigma=0.2, seed=8)
    xs = hamiltonian.basis(n, True)
    cf = hamiltonian.configs(xs, n)
    w = sampler.exact_distribution(p, cf)
    e = local_energy.local_energy_rbm(p, op, cf)
    assert abs(w @ e - vmc.exact_energy_of(p, op, True)) < 1e-10
    assert abs((w @ e).imag) < 1e-10


# ---------------------------------------------------------------- SR algebra

def _fullsum_setup(cplx, n=6, m=4, seed=9):
    op = W.ising(n, W.chain_bonds(n), h=0.9)
    p = W.init_params(n, m, cplx, sigma=0.3, seed=seed)
    xs = hamiltonian.basis(n)
    cf = hamiltonian.configs(xs, n)
    return op, p, cf


@pytest.mark.parametrize("cplx", [False, True])
def test_force_is_half_the_energy_gradient(cplx):
    op, p, cf = _fullsum_setup(cplx)
    w = sampler.exact_distribution(p, cf)
    e = local_energy.local_energy_rbm(p, op, cf)
    sig, t = rbm.logderiv_factored(p, cf)
    f = sr.force_lazy(sig, t, e, p.n, p.m, w, real=not cplx)
    x0 = p.flat()
    h = 1e-5
    for k in [0, 3, p.n + 1, p.n + p.m + 5, len(x0) - 1]:
        for direction, comp in ([(1.0, np.real)] + ([(1j, np.imag)] if cplx else [])):
            ee = np.zeros_like(x0)
            ee[k] = h * direction
            ep = vmc.exact_energy_of(W.RbmParams.from_flat(x0 + ee, p.n, p.m), op, False)
            em = vmc.exact_energy_of(W.RbmParams.from_flat(x0 - ee, p.n, p.m), op, False)
            assert abs((ep - em) / (2 * h) - 2 * comp(f[k])) < 1e-7


@pytest.mark.parametrize("cplx", [False, True])
def test_sr_matrix_properties_and_solvers(cplx):
    op, p, cf = _fullsum_setup(cplx)
    w = sampler.exact_distribution(p, cf)
    e = local_energy.local_energy_rbm(p, op, cf)
    o = rbm.logderiv_dense(p, cf)
    s, f = sr.sr_matrices(o, e, w, real=not cplx)
    assert np.abs(s - s.conj().T).max() <= 1e-14 * np.abs(s).max()
    assert np.linalg.eigvalsh(s).min() >= -1e-12
    # S is the weighted covariance matrix of O (library routine, real case)
    if not cplx:
        assert np.allclose(s, np.cov(o.T, aweights=w, bias=True), atol=1e-13)
    sig, t = rbm.logderiv_factored(p, cf)
    assert np.allclose(f, sr.force_lazy(sig, t, e, p.n, p.m, w, real=not cplx), atol=1e-13)
    x = np.random.default_rng(1).normal(size=len(f)) + (1j * np.random.default_rng(2).normal(size=len(f)) if cplx else 0)
    assert np.allclose(sr.sr_matvec_lazy(sig, t, x, p.n, p.m, w, real=not cplx), s @ x, atol=1e-12)
    d_dense = sr.solve_dense(s, f, 0.01)
    assert np.allclose(d_dense, np.linalg.solve(s + 0.01 * np.eye(len(s)), f), atol=1e-10)
    d_cg, it, res = sr.cg(lambda v: sr.sr_matvec_lazy(sig, t, v, p.n, p.m, w, not cplx), f, 0.01, 500, 1e-13)
    assert np.allclose(d_cg, d_dense, atol=1e-9) and res <= 1e-13


def test_stats_hand_example():
    e = np.array([1.0, 3.0, 2.0, 6.0])  # two chains: means 2 and 4, overall 3
    mean, var, err = sr.stats(e, 2)
    assert mean == 3.0 and abs(var - 3.5) < 1e-15
    assert abs(err - np.sqrt(((2 - 3) ** 2 + (4 - 3) ** 2) / 2)) < 1e-15


@pytest.mark.parametrize("move", ["flip", "exchange"])
def test_error_bar_matches_spread_over_independent_runs(move):
    """The error bar of one iteration's mean energy, computed from the means of
    whole proposal groups (the independent units of the sampler), must match the
    standard deviation of that mean over independent runs (different seeds and
    chain starts).  160 runs of 64 chains in 8 groups: the ratio of the two is
    known to about 6 %; a wrong normalisation (e.g. n_blocks^2 for
    n_blocks (n_blocks - 1)), a missing square root or per-sample errors that
    ignore autocorrelation miss the band."""
    n, nc, group, nd, spc = 8, 64, 8, 10, 8
    sz = move == "exchange"
    if sz:
        op = W.heisenberg(n, W.chain_bonds(n), 1.0, True, W.sublattice(n))
        p = W.perturb_params(W.init_params(n, 2 * n, True, 0.01, 5), 0.6 / np.sqrt(n), 6)
    else:
        op = W.ising(n, W.chain_bonds(n), h=1.0)
        p = W.perturb_params(W.init_params(n, n, False, 0.01, 5), 0.6 / np.sqrt(n), 6)
    means, errs = [], []
    for run in range(160):
        s0 = W.init_chains(nc, n, sz, 1000 + run)
        samp, _, _, _ = sampler.metropolis(p, s0, move, W.chain_bonds(n), group, 7000 + run, 0, nd,
                                           spc)
        e = local_energy.local_energy_rbm(p, op, samp)
        mean, _, err = sr.stats(e, nc // group)
        means.append(mean.real)
        errs.append(err)
    ratio = np.std(means, ddof=1) / np.sqrt(np.mean(np.square(errs)))
    assert 0.75 < ratio < 1.33, ratio


# ---------------------------------------------------------------- sampler

def test_zero_parameters_accept_every_flip():
    n = 6
    p = W.RbmParams(np.zeros(n), np.zeros(4), np.zeros((4, n)))
    s0 = W.init_chains(16, n, False, 3)
    samples, final, counter, n_acc = sampler.metropolis(p, s0, "flip", W.chain_bonds(n), 4, 77, 0, 1, 2)
    assert np.all(n_acc == 3 * n) and counter == 3 * n


def test_exchange_conserves_magnetisation_and_null_moves():
    n = 8
    p = W.init_params(n, 8, True, sigma=0.0, seed=1)
    s0 = W.init_chains(32, n, True, 3)
    samples, final, counter, n_acc = sampler.metropolis(p, s0, "exchange", W.chain_bonds(n), 8, 5, 10, 0, 5)
    assert np.all(samples.sum(axis=1) == 0) and np.all(final.sum(axis=1) == 0)
    # with psi constant every non-null exchange is accepted: count the null moves independently
    bonds = W.chain_bonds(n)
    sig = s0.astype(np.int64).copy()
    expect = np.zeros(32, dtype=np.int64)
    for t in range(10, 10 + 5 * n):
        b = philox.uniform_index(philox.draw(np.arange(32) // 8, t, philox.TAG_SITE, 5)[0], n)
        i, k = bonds[b, 0], bonds[b, 1]
        ok = sig[np.arange(32), i] != sig[np.arange(32), k]
        sig[ok, i[ok]] *= -1
        sig[ok, k[ok]] *= -1
        expect += ok
    assert np.array_equal(n_acc, expect) and np.array_equal(final, sig)


@pytest.mark.parametrize("move", ["flip", "exchange"])
def test_metropolis_samples_psi_squared(move):
    n = 6
    sz = move == "exchange"
    p = W.init_params(n, 6, True, sigma=0.25, seed=31)  # well-mixing in 20 sweeps
    xs = hamiltonian.basis(n, sz)
    cf = hamiltonian.configs(xs, n)
    pi = sampler.exact_distribution(p, cf)
    s0 = W.init_chains(4096, n, sz, 12)
    samples, *_ = sampler.metropolis(p, s0, move, W.chain_bonds(n), 8, 2024, 0, 100, 10)
    ints = ((1 - samples.astype(np.int64)) // 2) @ (1 << np.arange(n))
    pos = np.searchsorted(xs, ints)
    counts = np.bincount(pos, minlength=len(xs)).astype(np.float64)
    # samples within a chain are correlated: use the per-chain-sweep count as an
    # upper bound on the effective size by testing with one sample per chain
    first = ints.reshape(4096, 10)[:, -1]
    c1 = np.bincount(np.searchsorted(xs, first), minlength=len(xs)).astype(np.float64)
    exp1 = pi * 4096
    chi2 = np.sum((c1 - exp1) ** 2 / exp1)
    dof = len(xs) - 1
    assert chi2 < dof + 5 * np.sqrt(2 * dof)
    assert np.abs(counts / counts.sum() - pi).max() < 0.02


# ---------------------------------------------------------------- VMC + SR

@pytest.mark.parametrize("cplx", [False, True])
def test_full_sum_sr_converges_to_ground_state(cplx):
    n = 6
    op = W.ising(n, W.chain_bonds(n), h=1.0)
    e0 = hamiltonian.tfim_chain_ground(n, 1.0, 1.0)
    p = W.init_params(n, n, cplx, sigma=0.01, seed=1234)
    xs = hamiltonian.configs(hamiltonian.basis(n), n)
    ch = vmc.ChainState(np.zeros((1, n), np.int8), 0)
    energies = []
    for it in range(150):
        p, ch, info = vmc.vmc_sr_iteration(
            p, op, ch, move="flip", bonds=None, group_size=1, seed=0, n_discard=0,
            samples_per_chain=0, diag_shift=0.01, lr=0.05, n_cg=None, full_sum_basis=xs)
        energies.append(info["energy"])
    assert energies[-1] < energies[0]
    assert abs((energies[-1] - e0) / e0) < 2e-3


def test_cg_and_dense_sr_agree_in_an_iteration():
    n = 6
    op = W.ising(n, W.chain_bonds(n), h=1.0)
    p = W.init_params(n, n, False, sigma=0.1, seed=3)
    xs = hamiltonian.configs(hamiltonian.basis(n), n)
    ch = vmc.ChainState(np.zeros((1, n), np.int8), 0)
    kw = dict(move="flip", bonds=None, group_size=1, seed=0, n_discard=0, samples_per_chain=0,
              diag_shift=0.01, lr=0.05, full_sum_basis=xs)
    pa, _, _ = vmc.vmc_sr_iteration(p, op, ch, n_cg=None, **kw)
    pb, _, info = vmc.vmc_sr_iteration(p, op, ch, n_cg=200, cg_rtol=1e-14, **kw)
    assert np.allclose(pa.flat(), pb.flat(), atol=1e-11)


def test_sampled_vmc_iteration_runs_and_is_deterministic():
    w = W.workload("c1", n_chains=8, samples_per_chain=20)
    p = W.init_params(w.n, w.m, w.is_complex, 0.01, w.seed)
    ch = vmc.ChainState(W.init_chains(w.n_chains, w.n, False, w.seed), 0)
    kw = dict(move="flip", bonds=w.sampler_bonds, group_size=4, seed=w.seed, n_discard=2,
              samples_per_chain=20, diag_shift=0.01, lr=0.01, n_cg=None)
    a = vmc.vmc_sr_iteration(p, w.op, ch, **kw)
    b = vmc.vmc_sr_iteration(p, w.op, ch, **kw)
    assert np.array_equal(a[0].flat(), b[0].flat())
    assert a[1].counter == 22 * w.n
    assert abs(a[2]["energy"] - (-10.0)) < 3.0  # near-uniform psi: <H> ~ -h N
