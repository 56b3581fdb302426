"""The backward of ln psi with theta recomputed per chunk of samples
(nk_rbm_logpsi_backward): several chunks with a ragged last one against the
oracle's analytic gradient, and the 20x20 J1-J2 shape at its full sample count
(65,536 configurations, four chunks) on sampled hidden units, whose gradient
rows the oracle computes one by one.  Tolerances: rel 1e-5 (FP32), 1e-4 (BF16
hi + lo), norm-wise over the compared entries; at the 20x20 shape rel 1e-4 for
both (the gradient target), since there complex theta of FP32 accuracy near
zeros of cosh give tanh(theta) errors that move the gradient by ~1e-5 (measured
1.1e-5 with FP32 contractions; the same effect as in the SR force)."""
import numpy as np
import pytest
import torch

from oracle import rbm as orbm
from paper_1904_00031_gb300 import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def nk():
    from paper_1904_00031_gb300 import build, nk as nkmod
    build.build()
    nkmod.load_library()
    return nkmod


def _g(ns, cplx, seed):
    rng = np.random.default_rng(seed)
    g = rng.normal(size=ns)
    if cplx:
        g = g + 1j * rng.normal(size=ns)
    return g.astype(np.complex128)


@pytest.mark.parametrize("cplx", [False, True])
@pytest.mark.parametrize("prec", [0, 1])
def test_backward_several_chunks(nk, cplx, prec):
    n, m = 21, 45
    ns = 2 * 16384 + 777
    p = W.perturb_params(W.init_params(n, m, cplx, 0.01, 12), 0.1, 13)
    s = W.random_configs(ns, n, 14)
    g = _g(ns, cplx, 15)
    r = nk.Rbm(n, m, cplx)
    r.load(p.a, p.b, p.w)
    got = nk.nk_rbm_logpsi_backward(r, torch.from_numpy(s).cuda(), torch.from_numpy(g).cuda(),
                                    prec=prec).cpu().numpy()
    # sum_s conj(O_sk) g_s
    ref = np.conj(orbm.logpsi_backward(p, s, np.conj(g)))
    if not cplx:
        ref = ref.real
    tol = 1e-5 if prec == 0 else 1e-4
    assert np.linalg.norm(got - ref) <= tol * np.linalg.norm(ref)


@pytest.mark.parametrize("prec", [0, 1])
def test_backward_full_size_sampled_rows(nk, prec):
    w = W.workload("c5")
    n, m, ns = w.n, w.m, w.n_samples
    lib = nk.load_library()
    assert lib.nk_backward_scratch_bytes(n, m, 1, ns) == lib.nk_backward_scratch_bytes(n, m, 1,
                                                                                        16384)
    p = W.perturb_params(W.init_params(n, m, True, 0.01, w.seed), 0.02, 5)
    s = W.random_configs(ns, n, 31, True)
    g = _g(ns, True, 32) / ns
    r = nk.Rbm(n, m, True)
    r.load(p.a, p.b, p.w)
    got = nk.nk_rbm_logpsi_backward(r, torch.from_numpy(s).cuda(), torch.from_numpy(g).cuda(),
                                    prec=prec).cpu().numpy()
    sig = s.astype(np.float64)
    rows = np.random.default_rng(33).choice(m, 6, replace=False)
    ga = sig.T @ g                                     # visible biases: O_a = sigma
    sub = W.RbmParams(p.a, p.b[rows], p.w[rows])       # the sampled hidden units alone
    t = np.tanh(orbm.theta(sub, s))                    # [ns, 6]
    gb = t.conj().T @ g
    gw = (t.conj() * g[:, None]).T @ sig               # [6, n]
    ref = np.concatenate([ga, gb, gw.reshape(-1)])
    got_rows = np.concatenate([got[:n], got[n + rows],
                               got[n + m:].reshape(m, n)[rows].reshape(-1)])
    tol = 1e-4
    assert np.linalg.norm(got_rows - ref) <= tol * np.linalg.norm(ref), \
        np.linalg.norm(got_rows - ref) / np.linalg.norm(ref)
