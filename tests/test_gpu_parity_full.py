"""Parity with the FP64 oracle at the benchmarked launch configurations, and
element by element where other tests compare norms.

* Metropolis in the template the 20x20 J1-J2 workload runs (complex RBM,
  m = 1600: two warps per chain, 26 hidden units per lane; exchange moves, and
  flips), trajectories bit for bit for every chain whose oracle accept
  decisions never came within EPS_TIE of a tie (|ln U - 2 Re Delta|).
* The SR force element by element: with one CG iteration from x0 = 0 the
  direction is alpha F with alpha = F.F / F.(S + eps)F, so the update
  delta = (alpha_before - alpha_after) / lr is compared with the oracle's
  alpha F entry by entry (|d| <= tol max |alpha F|).
* The untied SR step at the 20x20 J1-J2 shape (n = 400, m = 1600 complex:
  26 parameter tiles, the SR forward's hidden tiles split over two CTAs, the
  separate centring kernel) against the oracle's lazy CG with the same fixed
  number of iterations.
* The batched first iteration of uneven instances: every chain's samples
  away from ties, and each instance's energy statistics and force whenever all
  its chains are away from ties, for at least four instances, at both
  precisions.

Tolerances (TOL_* below): ||F|| rel 1e-4 (the gradient target); force entries
5e-4 (FP32) / 1e-3 (BF16 hi + lo) of max |alpha F|; fixed-iteration CG direction
rel 1e-3 (FP32) / 5e-3 (BF16 hi + lo), norm-wise.  The measured errors are
printed (pytest -s)."""
import numpy as np
import pytest
import torch

from oracle import local_energy as ole
from oracle import rbm as orbm
from oracle import sampler as osam
from oracle import sr as osr
from paper_1904_00031_gb300 import workloads as W

pytestmark = pytest.mark.gpu

# Accept decisions of the kernel take 2 Re Delta from FP32 arithmetic (the
# per-unit factors, t = tanh theta kept by the addition formula within a sweep,
# the log of the running products); decisions whose oracle margin is at least
# this are compared exactly.
EPS_TIE = 1e-4

# Stated targets: gradients (the force) rel 1e-4; force entries relative to the
# largest entry; the fixed-iteration CG direction norm-wise.  At the 20x20 shape
# (complex W of scale 0.02 over 400 sites) some theta lie close to zeros of
# cosh, where tanh amplifies the ~1e-6 error of an FP32 theta: a numpy emulation
# of theta accumulated in FP32 alone moves ||F|| by 1.3e-5 and its entries by
# 5.6e-5 of the largest, and both contraction precisions measure the same
# 1.4e-5 / 1.8e-4, so the entry bound of the FP32 path is 5e-4.
TOL_F = 1e-4
TOL_ENTRY = {0: 5e-4, 1: 1e-3}
TOL_CG = {0: 1e-3, 1: 5e-3}


@pytest.fixture(scope="module")
def nk():
    from paper_1904_00031_gb300 import build, nk as nkmod
    build.build()
    lib = nkmod.load_library()
    assert lib.nk_device_supported() == 1
    return nkmod


def dev(x):
    return torch.from_numpy(np.ascontiguousarray(x)).cuda()


def make_rbm(nk, p):
    r = nk.Rbm(p.n, p.m, p.is_complex)
    r.load(p.a, p.b, p.w)
    return r


# ---------------------------------------------------------------- Metropolis, bench template

# sampler 1: two warps per chain; 3 (the built-in choice here) and 4: one CTA per
# proposal group with 2 and 3 hidden-unit pairs per thread
@pytest.mark.parametrize("sampler", [1, 3, 4])
@pytest.mark.parametrize("move", ["exchange", "flip"])
def test_metropolis_trajectories_m1600(nk, move, sampler):
    L, m = 8, 1600
    n = L * L
    p = W.perturb_params(W.init_params(n, m, True, 0.01, 1237), 0.03, 5)
    nc, group = 48, 8
    sz = move == "exchange"
    s0 = W.init_chains(nc, n, sz, 8)
    bonds = W.square_bonds(L)
    seed, counter, nd, nsamp = 1237, 3 * n, 1, 4
    samp, fin, cnt, nacc, marg = osam.metropolis(p, s0, move, bonds, group, seed, counter, nd,
                                                 nsamp, return_margin=True)
    r = make_rbm(nk, p)
    r._s.sampler = sampler
    ch = nk.Chains(s0, group, seed)
    ch.counter = counter
    acc = torch.zeros(nc, dtype=torch.int64, device="cuda")
    mv = nk.NK_MOVE_FLIP if move == "flip" else nk.NK_MOVE_EXCHANGE
    out = nk.nk_metropolis_sweep(r, ch, mv, dev(bonds[:, 0].copy()), dev(bonds[:, 1].copy()), nd,
                                 nsamp, n_accept_out=acc)
    assert ch.counter == cnt
    got = out.cpu().numpy().reshape(nc, nsamp, n)
    ref = samp.reshape(nc, nsamp, n)
    ok = marg > EPS_TIE
    print(f"\nMetropolis m=1600 {move} sampler {sampler}: {ok.sum()} of {nc} chains away from "
          f"ties, acceptance "
          f"{nacc.sum() / (nc * (nd + nsamp) * n):.3f}")
    assert ok.sum() >= (3 * nc) // 4, ok.sum()
    assert 0 < nacc.sum() < nc * (nd + nsamp) * n  # neither frozen nor trivially accepting
    bad = [c for c in np.flatnonzero(ok) if not np.array_equal(got[c], ref[c])]
    assert not bad, (bad, marg[bad])
    assert np.array_equal(ch.sigma.cpu().numpy()[ok], fin[ok])
    assert np.array_equal(acc.cpu().numpy()[ok], nacc[ok])


@pytest.mark.parametrize("sampler", [1, 3])
def test_metropolis_low_acceptance_reports_no_timeout(nk, sampler):
    """Chains of a 400-site, 1600-unit complex RBM (parameters perturbed by 0.05)
    that have settled where almost every exchange is rejected: some proposals
    then have |r_j|^2 that rounds to zero or below in the expanded FP32 form
    (theta near a zero of cosh).  Such a move is rejected; it must not read as a
    timed-out warp (which once stopped a CTA's copies until its bounded waits ran
    out, and marked its chains).  Two calls of 1 + 4 sweeps of 16384 chains."""
    n, m, nc, group = 400, 1600, 16384, 8
    p = W.perturb_params(W.init_params(n, m, True, 0.01, 7), 0.05, 5)
    r = make_rbm(nk, p)
    r._s.sampler = sampler
    bonds = W.chain_bonds(n)
    bi, bk = dev(bonds[:, 0].copy()), dev(bonds[:, 1].copy())
    ch = nk.Chains(W.init_chains(nc, n, True, 3), group, 11)
    acc = torch.zeros(nc, dtype=torch.int64, device="cuda")
    flags = nk.nk_query_status()  # clears earlier bits
    out = None
    for _ in range(2):
        out = nk.nk_metropolis_sweep(r, ch, nk.NK_MOVE_EXCHANGE, bi, bk, 1, 4, samples_out=out,
                                     n_accept_out=acc)
    nk.nk_query_status(flags)
    torch.cuda.synchronize()
    a = acc.cpu().numpy()
    assert int(flags.item()) == 0
    assert np.all(a >= 0)  # no chain marked (UINT64_MAX reads as -1)
    rate = a.sum() / (nc * 5 * n)
    print(f"\nlow-acceptance sampling, sampler {sampler}: acceptance {rate:.4f}")
    assert 0 < rate < 0.05
    assert np.all(out.cpu().numpy().astype(int).sum(axis=1) == 0)  # S^z = 0 kept


# ---------------------------------------------------------------- SR force entry by entry

def _t_on_gpu(nk, r, sg, m):
    th = torch.empty(sg.shape[0], m, dtype=r.f32_dtype(), device="cuda")
    nk.nk_rbm_logpsi(r, sg, theta_out=th)
    return nk.nk_logderiv(r, sg, th)


def _synthetic_eloc(ns, cplx, seed):
    g = np.random.default_rng(seed)
    e = -20.0 + 3.0 * g.normal(size=ns)
    if cplx:
        e = e + 0.5j * g.normal(size=ns)
    return e.astype(np.complex128)


def _one_cg_direction(p, s, e, eps, real):
    sig, t = orbm.logderiv_factored(p, s)
    f = osr.force_lazy(sig, t, e, p.n, p.m, None, real)
    sf = osr.sr_matvec_lazy(sig, t, f, p.n, p.m, None, real) + eps * f
    alpha = np.vdot(f, f).real / np.vdot(f, sf).real
    return alpha * f, sig, t, f


@pytest.mark.parametrize("n,m,cplx", [(12, 24, False), (12, 24, True), (40, 80, True),
                                      (100, 400, False)])
@pytest.mark.parametrize("prec", [0, 1])
def test_sr_force_entry_by_entry(nk, n, m, cplx, prec):
    ns, eps, lr = 2048 + 64, 0.01, 0.5
    p = W.perturb_params(W.init_params(n, m, cplx, 0.01, 40 + n), 0.2 / np.sqrt(n), 41)
    s = W.random_configs(ns, n, 42, cplx)
    e = _synthetic_eloc(ns, cplx, 43)
    ref, _, _, f = _one_cg_direction(p, s, e, eps, not cplx)
    r = make_rbm(nk, p)
    sg = dev(s)
    t = _t_on_gpu(nk, r, sg, m)
    info = nk.info_dict(nk.nk_sr_step(r, sg, t, dev(e), 8, eps, lr, n_cg=1, cg_rtol=0.0,
                                      prec=prec))
    assert info["cg_iters"] == 1
    fe = abs(info["f_norm"] - np.linalg.norm(f)) / np.linalg.norm(f)
    d = (p.flat() - np.concatenate([x.reshape(-1) for x in r.params_numpy()])) / lr
    err = np.abs(d - ref).max() / np.abs(ref).max()
    print(f"\nforce n={n} m={m} cplx={cplx} prec={prec}: |F| rel {fe:.2e}, entries {err:.2e}")
    assert fe <= TOL_F
    assert err <= TOL_ENTRY[prec]


# ---------------------------------------------------------------- untied SR at 20x20 J1-J2 size

@pytest.mark.parametrize("prec", [0, 1])
def test_sr_step_m1600_fixed_iterations(nk, prec):
    w = W.workload("c5")
    n, m = w.n, w.m
    ns, eps, lr, n_cg = 2048, 0.01, 0.5, 5
    p = W.perturb_params(W.init_params(n, m, True, 0.01, w.seed), 0.02, 5)
    s = W.random_configs(ns, n, 77, True)
    e = _synthetic_eloc(ns, True, 78)
    sig, tref = orbm.logderiv_factored(p, s)
    f = osr.force_lazy(sig, tref, e, n, m, None, False)
    ref, it, _ = osr.cg(lambda x: osr.sr_matvec_lazy(sig, tref, x, n, m, None, False), f, eps,
                        n_cg, 0.0)
    assert it == n_cg
    r = make_rbm(nk, p)
    sg = dev(s)
    t = _t_on_gpu(nk, r, sg, m)
    info = nk.info_dict(nk.nk_sr_step(r, sg, t, dev(e), 256, eps, lr, n_cg=n_cg, cg_rtol=0.0,
                                      prec=prec))
    assert info["cg_iters"] == n_cg and int(info["flags"]) & (1 << 6) == 0
    fe = abs(info["f_norm"] - np.linalg.norm(f)) / np.linalg.norm(f)
    d = (p.flat() - np.concatenate([x.reshape(-1) for x in r.params_numpy()])) / lr
    de = np.linalg.norm(d - ref) / np.linalg.norm(ref)
    # the one-iteration direction entry by entry at this size as well
    r1 = make_rbm(nk, p)
    nk.nk_sr_step(r1, sg, t, dev(e), 256, eps, lr, n_cg=1, cg_rtol=0.0, prec=prec)
    d1 = (p.flat() - np.concatenate([x.reshape(-1) for x in r1.params_numpy()])) / lr
    ref1, _, _, _ = _one_cg_direction(p, s, e, eps, False)
    e1 = np.abs(d1 - ref1).max() / np.abs(ref1).max()
    print(f"\nSR 20x20 prec={prec}: |F| rel {fe:.2e}, {n_cg}-iteration direction rel {de:.2e}, "
          f"one-iteration entries {e1:.2e}")
    assert fe <= TOL_F
    assert de <= TOL_CG[prec]
    assert e1 <= TOL_ENTRY[prec]


# ---------------------------------------------------------------- batched first iteration

@pytest.mark.parametrize("prec", [0, 1])
def test_batched_first_iteration_checks_instances(nk, prec):
    from paper_1904_00031_gb300.batch import BatchedVmc
    insts = W.batched_instances(n_inst=12, seed=4242, n_chains=16)
    for w in insts:
        w.n_cg = 10
    b = BatchedVmc(insts, prec=prec, graph=False)
    b.step()
    torch.cuda.synchronize()
    full = 0
    chains_checked = 0
    for v, w in zip(b.items, insts):
        p = W.init_params(w.n, w.m, w.is_complex, 0.01, w.seed)
        s0 = W.init_chains(w.n_chains, w.n, w.zero_magnetisation, w.seed)
        samp, fin, cnt, nacc, marg = osam.metropolis(
            p, s0, w.move, w.sampler_bonds, w.group_size, w.seed, 0, w.n_discard,
            w.samples_per_chain, return_margin=True)
        got = v.samples.cpu().numpy().reshape(w.n_chains, -1, w.n)
        ref = samp.reshape(w.n_chains, -1, w.n)
        ok = marg > EPS_TIE
        chains_checked += int(ok.sum())
        assert np.array_equal(got[ok], ref[ok]), w.name
        if not ok.all():
            continue
        e = ole.local_energy_rbm(p, w.op, samp)
        mean, var, err = osr.stats(e, w.n_chains // w.group_size)
        info = v.info()
        assert abs(info["energy"] - mean.real) <= 1e-6 * abs(mean.real), w.name
        assert abs(info["variance"] - var) <= 1e-4 * var, w.name
        assert abs(info["error"] - err) <= 1e-4 * err, w.name
        sig, t = orbm.logderiv_factored(p, samp)
        f = osr.force_lazy(sig, t, e, w.n, w.m, None, not w.is_complex)
        tol = 1e-5 if prec == 0 else 1e-4
        assert abs(info["f_norm"] - np.linalg.norm(f)) <= tol * np.linalg.norm(f), w.name
        full += 1
    print(f"\nbatched prec={prec}: {full} instances checked in full, {chains_checked} chains")
    assert full >= 4, full
    assert chains_checked >= 0.75 * sum(w.n_chains for w in insts)
