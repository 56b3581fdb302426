"""Multi-layer ln cosh networks on the GPU (nk_ffnn_logpsi / nk_ffnn_backward and
the autograd wrapper) against the FP64 oracle (oracle/ffnn.py), with ragged
tiles (widths and sample counts not multiples of 64) and several weight-gradient
splits.  Tolerances: ln psi |d| <= 1e-5 max(1, |ref|) (the FP32 path's target,
Im compared mod 2 pi); gradients rel 1e-4 norm-wise (the gradient target)."""
import numpy as np
import pytest
import torch

from oracle import ffnn as off
from paper_1904_00031_gb300 import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def mods():
    from paper_1904_00031_gb300 import autograd as ag
    from paper_1904_00031_gb300 import build, nk
    build.build()
    nk.load_library()
    return nk, ag


def wrap(d):
    return np.angle(np.exp(1j * d))


NETS = [([10, 20, 10], False), ([10, 20, 10], True), ([40, 80, 40, 20], True),
        ([100, 64], False), ([37, 75, 3], True), ([16, 130, 70, 33, 9], False)]


def net_of(nk, widths, cplx, x):
    f = nk.Ffnn(widths, cplx)
    f.load(x)
    return f


@pytest.mark.parametrize("widths,cplx", NETS)
def test_logpsi(mods, widths, cplx):
    nk, _ = mods
    x = W.init_ffnn_params(widths, cplx, 0.3 / np.sqrt(widths[0]), 50 + len(widths))
    s = W.random_configs(333, widths[0], 51)
    f = net_of(nk, widths, cplx, x)
    got = nk.nk_ffnn_logpsi(f, torch.from_numpy(s).cuda()).cpu().numpy()
    ref = off.logpsi(x, widths, s)
    scale = np.maximum(1.0, np.abs(ref))
    assert np.all(np.abs(got.real - ref.real) <= 1e-5 * scale), np.abs(got.real - ref.real).max()
    assert np.all(np.abs(wrap(got.imag - np.imag(ref))) <= 1e-5 * scale)


@pytest.mark.parametrize("cplx", [False, True])
def test_one_layer_equals_the_rbm_without_visible_bias(mods, cplx):
    nk, _ = mods
    n, m = 24, 48
    x = W.init_ffnn_params([n, m], cplx, 0.1, 60)
    (Wm, b), = off.unpack(x, [n, m])
    f = net_of(nk, [n, m], cplx, x)
    r = nk.Rbm(n, m, cplx)
    r.load(np.zeros(n), b, Wm)
    s = torch.from_numpy(W.random_configs(500, n, 61)).cuda()
    a = nk.nk_ffnn_logpsi(f, s).cpu().numpy()
    c = nk.nk_rbm_logpsi(r, s).cpu().numpy()
    assert np.abs(a - c).max() <= 1e-5 * max(1.0, np.abs(c).max())


@pytest.mark.parametrize("widths,cplx", NETS)
@pytest.mark.parametrize("ns", [333, 5000])
def test_backward(mods, widths, cplx, ns):
    nk, _ = mods
    x = W.init_ffnn_params(widths, cplx, 0.3 / np.sqrt(widths[0]), 70 + len(widths))
    s = W.random_configs(ns, widths[0], 71)
    rng = np.random.default_rng(72)
    g = (rng.normal(size=ns) + 1j * rng.normal(size=ns)) / ns
    f = net_of(nk, widths, cplx, x)
    got = nk.nk_ffnn_backward(f, torch.from_numpy(s).cuda(), torch.from_numpy(g).cuda())
    got = got.cpu().numpy()
    ref = off.backward(x, widths, s, g)
    assert np.linalg.norm(got - ref) <= 1e-4 * np.linalg.norm(ref), \
        np.linalg.norm(got - ref) / np.linalg.norm(ref)


@pytest.mark.parametrize("cplx", [False, True])
def test_autograd_gradient_and_finite_differences(mods, cplx):
    nk, ag = mods
    widths = [14, 28, 12]
    x0 = W.init_ffnn_params(widths, cplx, 0.1, 80)
    s = W.random_configs(600, 14, 81)
    f = nk.Ffnn(widths, cplx)
    dt = torch.complex128 if cplx else torch.float64
    x = torch.tensor(x0, dtype=dt, device="cuda", requires_grad=True)
    sg = torch.from_numpy(s).cuda()
    rng = np.random.default_rng(82)
    c = rng.normal(size=600) + (1j * rng.normal(size=600) if cplx else 0)
    ct = torch.tensor(c, dtype=dt, device="cuda")
    lp = ag.ffnn_logpsi(x, f, sg)
    loss = (ct * lp).real.sum() if cplx else (ct * lp).sum()
    (grad,) = torch.autograd.grad(loss, x)
    grad = grad.cpu().numpy()
    # PyTorch's gradient of the real loss: conj(sum_s c_s O_sk) (conjugate Wirtinger)
    o = off.logderiv_dense(x0, widths, s)
    ref = np.conj(c @ o) if cplx else c @ o
    assert np.linalg.norm(grad - ref) <= 1e-4 * np.linalg.norm(ref)
    h = 1e-3
    for k in [0, widths[1] * widths[0] + 3, off.n_params(widths) - 1]:
        for d in ([1.0, 1j] if cplx else [1.0]):
            e = np.zeros(len(x0), dtype=np.complex128 if cplx else np.float64)
            e[k] = h * d
            with torch.no_grad():
                lpp = ag.ffnn_logpsi(torch.tensor(x0 + e, dtype=dt, device="cuda"), f, sg)
                lpm = ag.ffnn_logpsi(torch.tensor(x0 - e, dtype=dt, device="cuda"), f, sg)
                fd = (((ct * (lpp - lpm)).real.sum() if cplx else (ct * (lpp - lpm)).sum()) /
                      (2 * h)).item()
            an = (np.conj(grad[k]) * d).real if cplx else grad[k]
            assert abs(fd - an) <= 1e-2 * max(1.0, abs(an))
