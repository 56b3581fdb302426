"""Measured error of every result of the path against the FP64 oracle, at the
shapes of the 40-site Heisenberg (n = 40, m = 80 complex), 10x10 TFIM (n = 100,
m = 400 real) and 20x20 J1-J2 (n = 400, m = 1600 complex) workloads, for both
contraction precisions: ln psi, theta, E_loc (from theta of that precision),
the SR force F and the SR direction after a fixed number of CG iterations.
Each row is printed (pytest -s) and checked against the stated targets:
ln psi rel 1e-5 (FP32) / 2e-3 (BF16 hi + lo) for 99 % of the samples and ten
times that for the worst (see below), E_loc mean rel 1e-4, gradients
(F) rel 1e-4, the fixed-iteration direction rel 1e-3 (FP32) / 5e-3.
Inputs: parameters N(0, 0.01^2) perturbed by N(0, scale^2) (structured psi),
uniformly random configurations (S^z = 0 for the Heisenberg models), synthetic
E_loc for the SR rows."""
import numpy as np
import pytest
import torch

from oracle import local_energy as ole
from oracle import rbm as orbm
from oracle import sr as osr
from paper_1904_00031_gb300 import workloads as W

pytestmark = pytest.mark.gpu

SHAPES = {
    # name: (workload, perturbation scale, samples for ln psi / SR, samples for E_loc)
    "heisenberg40": ("c2", 0.05, 2048, 512),
    "tfim10x10": ("c3", 0.03, 2048, 256),
    "j1j2_20x20": ("c5", 0.02, 2048, 64),
}
TARGET = {0: dict(logpsi=1e-5, eloc=1e-4, force=1e-4, cg=1e-3),
          1: dict(logpsi=2e-3, eloc=1e-4, force=1e-4, cg=5e-3)}


@pytest.fixture(scope="module")
def nk():
    from paper_1904_00031_gb300 import build, nk as nkmod
    build.build()
    nkmod.load_library()
    return nkmod


def rel_err(got, ref):
    return np.abs(got - ref) / np.maximum(1.0, np.abs(ref))


def rel_max(got, ref):
    return float(np.max(rel_err(got, ref)))


@pytest.mark.parametrize("name", list(SHAPES))
@pytest.mark.parametrize("prec", [0, 1])
def test_error_table(nk, name, prec):
    wl, scale, ns, ns_e = SHAPES[name]
    w = W.workload(wl)
    n, m, cplx = w.n, w.m, w.is_complex
    p = W.perturb_params(W.init_params(n, m, cplx, 0.01, w.seed), scale, 5)
    s = W.random_configs(ns, n, 21, w.zero_magnetisation)
    r = nk.Rbm(n, m, cplx)
    r.load(p.a, p.b, p.w)
    sg = torch.from_numpy(s).cuda()
    th = torch.empty(ns, m, dtype=r.f32_dtype(), device="cuda")
    lp = nk.nk_rbm_logpsi(r, sg, prec, theta_out=th).cpu().numpy()
    lp_ref = orbm.logpsi(p, s)
    th_ref = orbm.theta(p, s)
    e_lp_s = np.maximum(rel_err(lp.real, lp_ref.real),
                        np.abs(np.angle(np.exp(1j * (lp.imag - np.imag(lp_ref)))))
                        / np.maximum(1.0, np.abs(lp_ref)))
    e_lp, e_lp99 = float(e_lp_s.max()), float(np.quantile(e_lp_s, 0.99))
    e_th = rel_max(th.cpu().numpy(), th_ref)
    # local energies of the first ns_e samples, from theta of this precision
    gop = nk.Operator(w.op)
    el = nk.nk_local_energy(r, gop, sg[:ns_e].contiguous(), th[:ns_e].contiguous()).cpu().numpy()
    el_ref = ole.local_energy_rbm(p, w.op, s[:ns_e])
    e_el = rel_max(el, el_ref)
    e_el_mean = abs(el.mean() - el_ref.mean()) / max(1.0, abs(el_ref.mean()))
    # SR: force and a 5-iteration CG direction on synthetic E_loc
    g = np.random.default_rng(22)
    e = (-20.0 + 3.0 * g.normal(size=ns) + (0.5j * g.normal(size=ns) if cplx else 0)
         ).astype(np.complex128)
    sig, t_ref = orbm.logderiv_factored(p, s)
    f = osr.force_lazy(sig, t_ref, e, n, m, None, not cplx)
    d_ref, _, _ = osr.cg(lambda x: osr.sr_matvec_lazy(sig, t_ref, x, n, m, None, not cplx), f,
                         0.01, 5, 0.0)
    t = nk.nk_logderiv(r, sg, th)
    lr = 0.5
    info = nk.info_dict(nk.nk_sr_step(r, sg, t, torch.from_numpy(e).cuda(), 8, 0.01, lr, 5,
                                      cg_rtol=0.0, prec=prec))
    e_f = abs(info["f_norm"] - np.linalg.norm(f)) / np.linalg.norm(f)
    d = (p.flat() - np.concatenate([x.reshape(-1) for x in r.params_numpy()])) / lr
    e_d = float(np.linalg.norm(d - d_ref) / np.linalg.norm(d_ref))
    print(f"\n| {name} | {'fp32' if prec == 0 else 'bf16x2'} | {e_lp99:.1e} / {e_lp:.1e} | "
          f"{e_th:.1e} | {e_el:.1e} | {e_el_mean:.1e} | {e_f:.1e} | {e_d:.1e} |")
    T = TARGET[prec]
    # ln psi: the target holds for 99 % of the samples; the worst sample may sit
    # near a zero of cosh theta, where |d ln cosh / d theta| = |tanh theta| (a few
    # hundred at the 20x20 shape: a theta 0.0045 from i pi / 2) amplifies the
    # ~1e-7 relative FP32 error of theta
    assert e_lp99 <= T["logpsi"]
    assert e_lp <= 10 * T["logpsi"]
    assert e_el_mean <= T["eloc"]
    assert e_f <= T["force"]
    assert e_d <= T["cg"]
