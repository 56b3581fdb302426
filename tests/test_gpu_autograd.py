"""The autograd wrapper around nk_rbm_logpsi / nk_rbm_logpsi_backward against the
FP64 oracle gradient and against central finite differences of the GPU forward."""
import numpy as np
import pytest
import torch

from oracle import rbm as orbm
from paper_1904_00031_gb300 import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def nkmods():
    from paper_1904_00031_gb300 import build, nk
    from paper_1904_00031_gb300 import autograd as ag
    build.build()
    nk.load_library()
    return nk, ag


@pytest.mark.parametrize("cplx", [False, True])
@pytest.mark.parametrize("prec", [0, 1])
def test_autograd_gradient(nkmods, cplx, prec):
    nk, ag = nkmods
    n, m, ns = 14, 28, 600
    p = W.perturb_params(W.init_params(n, m, cplx, 0.01, 21), 0.1, 22)
    s = W.random_configs(ns, n, 23)
    r = nk.Rbm(n, m, cplx)
    dt = torch.complex128 if cplx else torch.float64
    x = torch.tensor(p.flat(), dtype=dt, device="cuda", requires_grad=True)
    sg = torch.from_numpy(s).cuda()
    rng = np.random.default_rng(24)
    c = rng.normal(size=ns) + (1j * rng.normal(size=ns) if cplx else 0)
    ct = torch.tensor(c, dtype=dt, device="cuda")
    lp = ag.logpsi(x, r, sg, prec)
    loss = (ct * lp).real.sum() if cplx else (ct * lp).sum()
    (grad,) = torch.autograd.grad(loss, x)
    grad = grad.cpu().numpy()
    # oracle: dL/d alpha for L = Re sum c_s lnpsi_s; PyTorch returns the conjugate
    # Wirtinger gradient 2 dL/d conj(alpha) = conj(sum_s c_s O_sk) for holomorphic lnpsi
    o = orbm.logderiv_dense(p, s)
    ref = np.conj(c @ o) if cplx else c @ o
    tol = 1e-5 if prec == 0 else 1e-4
    assert np.linalg.norm(grad - ref) <= tol * np.linalg.norm(ref)
    # central finite differences of the GPU forward along a few coordinates
    h = 1e-3
    for k in [0, n + 3, n + m + 7, len(p.flat()) - 1]:
        for d in ([1.0, 1j] if cplx else [1.0]):
            e = np.zeros(len(p.flat()), dtype=np.complex128 if cplx else np.float64)
            e[k] = h * d
            with torch.no_grad():
                lpp = ag.logpsi(torch.tensor(p.flat() + e, dtype=dt, device="cuda"), r, sg, prec)
                lpm = ag.logpsi(torch.tensor(p.flat() - e, dtype=dt, device="cuda"), r, sg, prec)
                fd = (((ct * (lpp - lpm)).real.sum() if cplx else (ct * (lpp - lpm)).sum()) /
                      (2 * h)).item()
            an = (np.conj(grad[k]) * d).real if cplx else grad[k]
            assert abs(fd - an) <= 1e-2 * max(1.0, abs(an))
