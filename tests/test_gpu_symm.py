"""Symmetric RBM (RbmSpinSymm) through the C ABI against the oracle: the
expansion of the tied parameters (exact: a copy), amplitudes of the expanded
RBM, and the SR step in the tied space at both precisions (direction, ||F_t||,
a fixed number of CG iterations, the degenerate one-permutation group), plus a
full-size 20x20 step checked on the tied direction after a few CG iterations.

Tolerances: the tied direction within 1e-3 (FP32 contractions) or 5e-3 (BF16
hi + lo contractions) relative, the same bounds as the untied SR step; ||F_t||
within 1e-5 relative."""
import numpy as np
import pytest
import torch

from oracle import rbm_symm as osym
from oracle import sr as osr
from paper_1904_00031_gb300 import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def nk():
    from paper_1904_00031_gb300 import build, nk as nkmod
    build.build()
    lib = nkmod.load_library()
    assert lib.nk_device_supported() == 1
    return nkmod


def dev(x):
    return torch.from_numpy(np.ascontiguousarray(x)).cuda()


GROUPS = {
    "chain12": (12, lambda: W.chain_translations(12)),
    "square4": (16, lambda: W.square_translations(4)),
    "identity": (12, lambda: np.arange(12, dtype=np.int32)[None, :]),
}


def _setup(nk, name, alpha, cplx, ns, seed=3, scale=0.3):
    n, mk = GROUPS[name]
    perm = mk()
    ps = W.init_symm_params(n, alpha, cplx, sigma=scale / np.sqrt(n), seed=seed)
    sy = nk.RbmSymm(perm, alpha, cplx)
    sy.load(ps.a, ps.b, ps.w)
    s = W.random_configs(ns, n, seed + 1)
    rng = np.random.default_rng(seed + 2)
    e = rng.normal(-0.5 * n, 1.0, ns) + (1j * rng.normal(0, 0.3, ns) if cplx else 0.0)
    return perm, ps, sy, s, np.asarray(e, np.complex128)


def _t(nk, sy, sg):
    r = sy.rbm
    th = torch.empty(sg.shape[0], r.m, dtype=r.f32_dtype(), device="cuda")
    nk.nk_rbm_logpsi(r, sg, theta_out=th)
    return nk.nk_logderiv(r, sg, th)


@pytest.mark.parametrize("name", list(GROUPS))
@pytest.mark.parametrize("cplx", [False, True])
def test_expand_and_amplitudes(nk, name, cplx):
    perm, ps, sy, s, _ = _setup(nk, name, 3, cplx, 200)
    a, b, w = sy.rbm.params_numpy()
    ref = osym.expand(ps, perm)
    assert np.array_equal(a, ref.a) and np.array_equal(b, ref.b) and np.array_equal(w, ref.w)
    lp = nk.nk_rbm_logpsi(sy.rbm, dev(s)).cpu().numpy()
    lref = osym.logpsi(ps, perm, s)
    scale = np.maximum(1.0, np.abs(lref))
    assert np.all(np.abs(lp.real - lref.real) <= 1e-5 * scale)
    # invariance of the GPU amplitudes under a lattice translation
    lp2 = nk.nk_rbm_logpsi(sy.rbm, dev(s[:, perm[-1]])).cpu().numpy()
    assert np.all(np.abs(lp2.real - lp.real) <= 1e-5 * scale)


def _tied_after(sy):
    a, b, w = sy.params_numpy()
    return np.concatenate([a, b, w.reshape(-1)])


@pytest.mark.parametrize("name", list(GROUPS))
@pytest.mark.parametrize("cplx", [False, True])
@pytest.mark.parametrize("prec", ["fp32", "bf16x2"])
def test_sr_step_symm_matches_oracle(nk, name, cplx, prec):
    alpha, ns, nc, lr, eps = 2, 2048, 64, 0.05, 0.01
    perm, ps, sy, s, e = _setup(nk, name, alpha, cplx, ns)
    sg = dev(s)
    t = _t(nk, sy, sg)
    delta = osym.sr_direction_dense(ps, perm, s, e, eps)
    o = osym.logderiv_dense(ps, perm, s)
    _, f = osr.sr_matrices(o, e, None, not cplx)
    pr = nk.NK_PREC_FP32 if prec == "fp32" else nk.NK_PREC_BF16X2
    info = nk.info_dict(nk.nk_sr_step_symm(sy, sg, t, dev(e), nc, eps, lr, n_cg=4 * ps.n_params,
                                           cg_rtol=1e-10, prec=pr))
    assert abs(info["f_norm"] - np.linalg.norm(f)) <= 1e-5 * np.linalg.norm(f)
    assert info["cg_resid"] <= 1e-6
    d_gpu = (ps.flat() - _tied_after(sy)) / lr
    tol = 1e-3 if prec == "fp32" else 5e-3
    assert np.linalg.norm(d_gpu - delta) <= tol * np.linalg.norm(delta)
    # the untied RBM was rewritten from the updated tied parameters (a copy)
    new = W.RbmSymmParams.from_flat(_tied_after(sy), ps.n, alpha)
    ref = osym.expand(new, perm)
    a, b, w = sy.rbm.params_numpy()
    assert np.array_equal(a, ref.a) and np.array_equal(b, ref.b) and np.array_equal(w, ref.w)


@pytest.mark.parametrize("prec", ["fp32", "bf16x2"])
def test_sr_symm_fixed_iterations(nk, prec):
    alpha, ns, lr = 2, 1024, 0.1
    perm, ps, sy, s, e = _setup(nk, "square4", alpha, True, ns, seed=9)
    sg = dev(s)
    t = _t(nk, sy, sg)
    x, _, res = osym.sr_direction_cg(ps, perm, s, e, 0.01, 5, 1e-12)
    pr = nk.NK_PREC_FP32 if prec == "fp32" else nk.NK_PREC_BF16X2
    info = nk.info_dict(nk.nk_sr_step_symm(sy, sg, t, dev(e), 16, 0.01, lr, n_cg=5,
                                           cg_rtol=1e-12, prec=pr))
    assert info["cg_iters"] == 5 and int(info["flags"]) & (1 << 4)
    d_gpu = (ps.flat() - _tied_after(sy)) / lr
    tol = 1e-3 if prec == "fp32" else 5e-3
    assert np.linalg.norm(d_gpu - x) <= tol * np.linalg.norm(x)
    assert abs(info["cg_resid"] - res) <= 1e-2 * res


def test_sr_symm_full_size_20x20(nk):
    # 20x20 lattice, 400 translations, alpha = 4 (m = 1600, complex): the SR step
    # of the symmetric 20x20 workload on 2048 samples, 8 CG iterations against the
    # oracle's CG on its dense tied S (the same Krylov iterates)
    L, alpha, ns, lr, eps, k = 20, 4, 2048, 0.01, 0.01, 8
    n = L * L
    perm = W.square_translations(L)
    ps = W.init_symm_params(n, alpha, True, sigma=0.02, seed=17)
    sy = nk.RbmSymm(perm, alpha, True)
    sy.load(ps.a, ps.b, ps.w)
    s = W.random_configs(ns, n, 18, True)
    rng = np.random.default_rng(19)
    e = (rng.normal(-450.0, 5.0, ns) + 1j * rng.normal(0, 1.0, ns)).astype(np.complex128)
    sg = dev(s)
    t = _t(nk, sy, sg)
    info = nk.info_dict(nk.nk_sr_step_symm(sy, sg, t, dev(e), 64, eps, lr, n_cg=k, cg_rtol=0.0,
                                           prec=nk.NK_PREC_BF16X2))
    o = osym.logderiv_dense(ps, perm, s)
    smat, f = osr.sr_matrices(o, e, None, False)
    x, it, _ = osr.cg(lambda v: smat @ v, f, eps, k, 0.0)
    assert it == k and info["cg_iters"] == k
    assert abs(info["f_norm"] - np.linalg.norm(f)) <= 1e-5 * np.linalg.norm(f)
    d_gpu = (ps.flat() - _tied_after(sy)) / lr
    assert np.linalg.norm(d_gpu - x) <= 5e-3 * np.linalg.norm(x)
