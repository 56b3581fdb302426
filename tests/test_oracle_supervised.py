"""Pins of the supervised-learning oracle (Sec. 2.2.3, Eq. 1; AdaMax of the
optimiser list): the loss vanishes exactly on a target proportional to psi and
is otherwise positive (Cauchy-Schwarz); the weighted-sample form with exact
weights equals the summed overlaps; the gradient matches central finite
differences; AdaMax takes steps of exactly lr sign(g) under a constant gradient
(its closed form); and full-sum training reaches the TFIM ground state."""
import numpy as np
import pytest

from oracle import hamiltonian, rbm, supervised
from paper_1904_00031_gb300 import workloads as W


def _basis(n):
    return hamiltonian.configs(hamiltonian.basis(n), n)


def _full(p, cf, tar):
    w = np.abs(tar) ** 2
    return supervised.overlap_loss_and_grad(p, cf, tar, weights=w)


@pytest.mark.parametrize("cplx", [False, True])
def test_loss_is_zero_on_a_proportional_target_and_positive_otherwise(cplx):
    n = 6
    cf = _basis(n)
    p = W.perturb_params(W.init_params(n, 6, cplx, 0.01, 3), 0.3, 4)
    tar = (0.7 - 0.4j) * np.exp(rbm.logpsi(p, cf))
    assert abs(supervised.overlap_loss_full(p, cf, tar)) < 1e-12
    lw, g = _full(p, cf, tar)
    assert abs(lw) < 1e-12 and np.abs(g).max() < 1e-10
    other = W.perturb_params(p, 0.3, 9)
    assert supervised.overlap_loss_full(other, cf, tar) > 1e-3
    # sampled form on any samples: still exactly 0 for a proportional target
    s = W.random_configs(50, n, 5)
    ls, _ = supervised.overlap_loss_and_grad(p, s, (0.7 - 0.4j) * np.exp(rbm.logpsi(p, s)))
    assert abs(ls) < 1e-12


@pytest.mark.parametrize("cplx", [False, True])
def test_weighted_samples_equal_the_summed_overlaps_and_finite_differences(cplx):
    n = 5
    cf = _basis(n)
    rng = np.random.default_rng(2)
    tar = rng.normal(size=len(cf)) + 1j * rng.normal(size=len(cf))
    p = W.perturb_params(W.init_params(n, 4, cplx, 0.01, 7), 0.4, 8)
    loss, g = _full(p, cf, tar)
    assert abs(loss - supervised.overlap_loss_full(p, cf, tar)) < 1e-12
    x0 = p.flat()
    h = 1e-6
    for k in range(p.n_params):
        for step, part in ((1.0, "re"), (1j, "im")):
            if part == "im" and not cplx:
                continue
            e = np.zeros_like(x0)
            e[k] = h * step
            up = supervised.overlap_loss_full(W.RbmParams.from_flat(x0 + e, n, 4), cf, tar)
            dn = supervised.overlap_loss_full(W.RbmParams.from_flat(x0 - e, n, 4), cf, tar)
            fd = (up - dn) / (2 * h)
            want = g[k].real if part == "re" else g[k].imag
            assert abs(fd - want) < 1e-6 * max(1.0, abs(want)), (k, part, fd, want)


def test_adamax_closed_form_steps():
    opt = supervised.AdaMax(lr=0.01)
    theta = np.array([1.0, -2.0, 0.5])
    g = np.array([3.0, -0.2, 0.0])
    for t in range(5):
        new = opt.step(theta, g)
        assert np.allclose(new - theta, [-0.01, 0.01, 0.0], atol=1e-15)
        theta = new
    # complex parameters: real and imaginary parts move independently
    opt = supervised.AdaMax(lr=0.1)
    z = opt.step(np.array([1.0 + 1.0j]), np.array([2.0 - 5.0j]))
    assert np.allclose(z, [0.9 + 1.1j], atol=1e-15)
    # a sign change: m and u follow Algorithm 2
    opt = supervised.AdaMax(lr=1.0, beta1=0.5, beta2=0.5)
    th = opt.step(np.array([0.0]), np.array([4.0]))       # m=2, u=4, step 1/(1-.5)*2/4 = 1
    th = opt.step(th, np.array([-1.0]))                     # m=0.5, u=2, step 1/(1-.25)*.5/2
    assert np.allclose(th, [-1.0 - 1.0 / 3.0], atol=1e-15)


def test_full_sum_training_reaches_the_tfim_ground_state():
    n = 6
    op = W.ising(n, W.chain_bonds(n), h=1.0)
    _, vec, xs = hamiltonian.exact_ground(op)
    cf = hamiltonian.configs(xs, n)
    tar = np.asarray(vec, dtype=np.complex128)
    p = W.init_params(n, n, False, 0.01, 1234)
    opt = supervised.AdaMax(lr=0.02)
    losses = []
    for _ in range(400):
        loss, g = _full(p, cf, tar)
        losses.append(loss)
        p = W.RbmParams.from_flat(opt.step(p.flat(), g), n, n)
    assert losses[-1] < 0.25 * losses[0]
    assert losses[-1] < 1e-2  # overlap above 0.99
