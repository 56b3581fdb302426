"""Pins of the symmetric-RBM oracle (RbmSpinSymm, Sec. 2.2.2) against results
fixed by the mathematics: group axioms of the translation tables, invariance
of psi under the group, finite differences of ln psi, the adjoint relation of
the tie maps, dense against matrix-free SR, and convergence of full-sum SR in
the tied space to the closed-form ground energy of the periodic TFIM chain."""
import numpy as np
import pytest

from oracle import hamiltonian, local_energy, rbm, rbm_symm, sr
from paper_1904_00031_gb300 import workloads as W

GROUPS = {"chain8": (8, lambda: W.chain_translations(8)),
          "square3": (9, lambda: W.square_translations(3))}


def _params(n, alpha, cplx, seed, sigma=0.3):
    return W.init_symm_params(n, alpha, cplx, sigma=sigma, seed=seed)


@pytest.mark.parametrize("name", list(GROUPS))
def test_translation_tables_form_a_group(name):
    n, make = GROUPS[name]
    perm = make()
    assert perm.shape == (n, n)
    rows = {tuple(r) for r in perm}
    assert len(rows) == n
    assert tuple(range(n)) in rows
    for r in perm:
        assert sorted(r) == list(range(n))
        for q in perm:
            assert tuple(r[q]) in rows  # closed under composition


@pytest.mark.parametrize("name", list(GROUPS))
@pytest.mark.parametrize("cplx", [False, True])
def test_psi_is_invariant_under_the_group(name, cplx):
    n, make = GROUPS[name]
    perm = make()
    ps = _params(n, 2, cplx, seed=5)
    sig = W.random_configs(16, n, seed=9)
    lp = rbm_symm.logpsi(ps, perm, sig)
    for h in perm:
        assert np.allclose(rbm_symm.logpsi(ps, perm, sig[:, h]), lp, atol=1e-12)
    # a generic (untied) RBM is not invariant: the check has teeth
    p = W.init_params(n, 2 * n, cplx, sigma=0.3, seed=5)
    assert not np.allclose(rbm.logpsi(p, sig[:, perm[1]]), rbm.logpsi(p, sig), atol=1e-6)


@pytest.mark.parametrize("cplx", [False, True])
def test_expanded_rbm_has_the_same_amplitude(cplx):
    perm = W.square_translations(3)
    ps = _params(9, 3, cplx, seed=2)
    sig = W.random_configs(32, 9, seed=4)
    p = rbm_symm.expand(ps, perm)
    assert p.m == 27 and np.all(p.a == ps.a[0])
    assert np.allclose(rbm.logpsi(p, sig), rbm_symm.logpsi(ps, perm, sig), atol=1e-12)


@pytest.mark.parametrize("cplx", [False, True])
def test_tied_logderiv_by_finite_differences(cplx):
    perm = W.chain_translations(6)
    ps = _params(6, 2, cplx, seed=11)
    sig = W.random_configs(5, 6, seed=12)
    o = rbm_symm.logderiv_dense(ps, perm, sig)
    x0 = ps.flat()
    h = 1e-6
    for k in range(ps.n_params):
        e = np.zeros_like(x0)
        e[k] = h
        up = rbm_symm.logpsi(W.RbmSymmParams.from_flat(x0 + e, 6, 2), perm, sig)
        dn = rbm_symm.logpsi(W.RbmSymmParams.from_flat(x0 - e, 6, 2), perm, sig)
        assert np.allclose((up - dn) / (2 * h), o[:, k], atol=1e-7), k


def test_fold_is_the_transpose_of_expand():
    perm = W.square_translations(3)
    n, alpha = 9, 2
    rng = np.random.default_rng(3)
    m = alpha * len(perm)
    u = rng.normal(size=n + m + n * m) + 1j * rng.normal(size=n + m + n * m)
    x = rng.normal(size=1 + alpha + alpha * n) + 1j * rng.normal(size=1 + alpha + alpha * n)
    lhs = np.dot(rbm_symm.fold(u, n, alpha, perm), x)
    rhs = np.dot(u, rbm_symm.expand_vector(x, n, alpha, perm))
    assert abs(lhs - rhs) < 1e-10
    # chain rule: the tied derivatives are the folded untied ones
    ps = _params(n, alpha, True, seed=8)
    sig = W.random_configs(4, n, seed=1)
    o_full = rbm.logderiv_dense(rbm_symm.expand(ps, perm), sig)
    o_t = rbm_symm.logderiv_dense(ps, perm, sig)
    for s in range(4):
        assert np.allclose(rbm_symm.fold(o_full[s], n, alpha, perm), o_t[s], atol=1e-12)


def _full_sum(ps, perm, op, xs):
    lp = rbm_symm.logpsi(ps, perm, xs)
    w = np.exp(2 * (lp.real - lp.real.max()))
    w /= w.sum()
    e = local_energy.local_energy_rbm(rbm_symm.expand(ps, perm), op, xs)
    return w, e


@pytest.mark.parametrize("cplx", [False, True])
def test_cg_in_the_tied_space_equals_the_dense_solve(cplx):
    n = 6
    perm = W.chain_translations(n)
    op = W.ising(n, W.chain_bonds(n), h=1.0)
    ps = _params(n, 2, cplx, seed=21, sigma=0.1)
    xs = hamiltonian.configs(hamiltonian.basis(n), n)
    w, e = _full_sum(ps, perm, op, xs)
    d = rbm_symm.sr_direction_dense(ps, perm, xs, e, 0.01, weights=w)
    x, _, res = rbm_symm.sr_direction_cg(ps, perm, xs, e, 0.01, 200, 1e-14, weights=w)
    assert res < 1e-12
    assert np.allclose(x, d, atol=1e-10)


def test_full_sum_tied_sr_converges_to_the_tfim_ground_state():
    n = 6
    perm = W.chain_translations(n)
    op = W.ising(n, W.chain_bonds(n), h=1.0)
    e0 = hamiltonian.tfim_chain_ground(n, 1.0, 1.0)
    ps = W.init_symm_params(n, 2, False, sigma=0.01, seed=1234)
    xs = hamiltonian.configs(hamiltonian.basis(n), n)
    energies = []
    for _ in range(150):
        w, e = _full_sum(ps, perm, op, xs)
        energies.append(float(w @ e.real))
        d = rbm_symm.sr_direction_dense(ps, perm, xs, e, 0.01, weights=w)
        ps = W.RbmSymmParams.from_flat(sr.sgd_update(ps.flat(), d, 0.05), n, 2)
    assert energies[-1] < energies[0]
    assert abs((energies[-1] - e0) / e0) < 2e-3


@pytest.mark.parametrize("case", ["heis_chain12", "j1j2_4x4"])
def test_marshall_rotated_hamiltonians_commute_with_translations(case):
    """The symmetric ansatz suits the bench workloads: the Marshall-rotated
    Heisenberg chain and J1-J2 square lattice commute with every lattice
    translation in the S^z = 0 sector (N/2 even), so the ground state is
    translation invariant."""
    if case == "heis_chain12":
        n = 12
        op = W.heisenberg(n, W.chain_bonds(n), 1.0, True, W.sublattice(n))
        perm = W.chain_translations(n)
    else:
        n = 16
        op = W.j1j2(4, 1.0, 0.5, True)
        perm = W.square_translations(4)
    xs = hamiltonian.basis(n, True)
    cf = hamiltonian.configs(xs, n)
    h = hamiltonian.sparse_h(op, xs)
    rng = np.random.default_rng(0)
    v = rng.normal(size=len(xs)) + 1j * rng.normal(size=len(xs))
    for g in perm[1:3]:
        # (T v)(sigma) = v(sigma o g): configurations permuted by the translation
        moved = cf[:, g]
        ints = ((1 - moved.astype(np.int64)) // 2) @ (1 << np.arange(n))
        at = np.searchsorted(xs, ints)
        tv = v[at]
        htv = h @ tv
        th_v = (h @ v)[at]
        assert np.allclose(htv, th_v, atol=1e-10)
