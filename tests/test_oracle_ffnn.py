"""Pins of the multi-layer ln cosh FFNN oracle (Sec. 2.2.2): the one-layer
network is the RBM without visible bias (the paper's statement, checked against
the separately pinned RBM oracle); with zero first-layer biases psi is even
under sigma -> -sigma at any depth (ln cosh is even); zero weights in the last
layer make ln psi constant; and the analytic log-derivatives and the backward
match central finite differences of ln psi, for real and complex parameters."""
import numpy as np
import pytest

from oracle import ffnn, rbm
from paper_1904_00031_gb300 import workloads as W


@pytest.mark.parametrize("cplx", [False, True])
def test_one_layer_is_the_rbm_without_visible_bias(cplx):
    n, m = 9, 14
    widths = [n, m]
    x = W.init_ffnn_params(widths, cplx, 0.3, 4)
    (Wm, b), = ffnn.unpack(x, widths)
    s = W.random_configs(50, n, 5)
    p = W.RbmParams(np.zeros(n, dtype=Wm.dtype), b, Wm)
    assert np.allclose(ffnn.logpsi(x, widths, s), rbm.logpsi(p, s), atol=1e-13, rtol=1e-13)


@pytest.mark.parametrize("cplx", [False, True])
def test_spin_flip_symmetry_without_first_biases(cplx):
    widths = [8, 12, 6, 5]
    x = W.init_ffnn_params(widths, cplx, 0.4, 6)
    o = widths[1] * widths[0]
    x[o:o + widths[1]] = 0.0       # b_1 = 0
    s = W.random_configs(40, 8, 7)
    assert np.allclose(ffnn.logpsi(x, widths, s), ffnn.logpsi(x, widths, -s), atol=1e-12)
    y = x.copy()
    y[o] = 0.3                     # a nonzero first-layer bias breaks it
    assert not np.allclose(ffnn.logpsi(y, widths, s), ffnn.logpsi(y, widths, -s), atol=1e-6)


def test_zero_last_weights_make_psi_constant():
    widths = [6, 10, 4]
    x = W.init_ffnn_params(widths, True, 0.5, 8)
    o = widths[1] * (widths[0] + 1)
    x[o:o + widths[2] * widths[1]] = 0.0    # W_2 = 0
    s = W.random_configs(30, 6, 9)
    lp = ffnn.logpsi(x, widths, s)
    b2 = x[o + widths[2] * widths[1]:]
    assert np.allclose(lp, np.sum(rbm.lncosh(b2)), atol=1e-13)


@pytest.mark.parametrize("cplx", [False, True])
def test_log_derivatives_match_finite_differences(cplx):
    widths = [6, 8, 5, 3]
    x = W.init_ffnn_params(widths, cplx, 0.4, 10)
    s = W.random_configs(7, 6, 11)
    o = ffnn.logderiv_dense(x, widths, s)
    assert o.shape == (7, ffnn.n_params(widths))
    h = 1e-6
    for k in range(len(x)):
        e = np.zeros_like(x)
        e[k] = h
        fd = (ffnn.logpsi(x + e, widths, s) - ffnn.logpsi(x - e, widths, s)) / (2 * h)
        assert np.allclose(fd, o[:, k], atol=1e-7, rtol=1e-7), k
        if cplx:  # holomorphic: the derivative along i h is i times the same
            fdi = (ffnn.logpsi(x + 1j * e, widths, s) - ffnn.logpsi(x - 1j * e, widths, s)) / (2 * h)
            assert np.allclose(fdi, 1j * o[:, k], atol=1e-7, rtol=1e-7), k


@pytest.mark.parametrize("cplx", [False, True])
def test_backward_is_the_gradient_of_a_real_loss(cplx):
    """For L = Re sum_s c_s ln psi_s, PyTorch's upstream gradient is g = conj(c)
    and the backward then returns dL/dRe(alpha_k) + i dL/dIm(alpha_k)."""
    widths = [5, 7, 4]
    x = W.init_ffnn_params(widths, cplx, 0.4, 12)
    s = W.random_configs(9, 5, 13)
    rng = np.random.default_rng(14)
    c = rng.normal(size=9) + (1j * rng.normal(size=9) if cplx else 0)
    b = ffnn.backward(x, widths, s, np.conj(c))

    def loss(y):
        return float(np.real(np.sum(c * ffnn.logpsi(y, widths, s))))

    h = 1e-6
    for k in range(len(x)):
        e = np.zeros_like(x)
        e[k] = h
        assert abs((loss(x + e) - loss(x - e)) / (2 * h) - np.real(b[k])) < 1e-7
        if cplx:
            assert abs((loss(x + 1j * e) - loss(x - 1j * e)) / (2 * h) - np.imag(b[k])) < 1e-7
