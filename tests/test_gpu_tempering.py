"""Parallel tempering on the GPU (nk_pt_sweep) against the oracle
(oracle/tempering.py): one replica is the plain sampler bit for bit; ladders of
several replicas follow the oracle's trajectories (samples of the beta = 1
replicas, final states of every replica, accepted moves and exchanges) for
every ladder whose decisions never came within EPS_TIE of a tie, including the
20x20 J1-J2 kernel template (m = 1600, two warps per chain); and every replica
samples |psi|^(2 beta_r) (chi-square against the exact tempered distribution)."""
import numpy as np
import pytest
import torch

from oracle import hamiltonian, rbm, sampler, tempering
from paper_1904_00031_gb300 import workloads as W

pytestmark = pytest.mark.gpu

EPS_TIE = 1e-4  # as the Metropolis trajectory tests


@pytest.fixture(scope="module")
def nk():
    from paper_1904_00031_gb300 import build, nk as nkmod
    build.build()
    nkmod.load_library()
    return nkmod


def dev(x):
    return torch.from_numpy(np.ascontiguousarray(x)).cuda()


def rbm_of(nk, p):
    r = nk.Rbm(p.n, p.m, p.is_complex)
    r.load(p.a, p.b, p.w)
    return r


@pytest.mark.parametrize("move", ["flip", "exchange"])
def test_one_replica_is_the_plain_sampler(nk, move):
    n, m = 12, 24
    p = W.perturb_params(W.init_params(n, m, True, 0.01, 3), 0.4 / np.sqrt(n), 4)
    s0 = W.init_chains(64, n, move == "exchange", 5)
    b = W.chain_bonds(n)
    mv = nk.NK_MOVE_FLIP if move == "flip" else nk.NK_MOVE_EXCHANGE
    r = rbm_of(nk, p)
    outs = []
    for pt in (False, True):
        ch = nk.Chains(s0, 8, 77)
        ch.counter = 3 * n
        acc = torch.zeros(64, dtype=torch.int64, device="cuda")
        if pt:
            smp = nk.nk_pt_sweep(r, ch, 1, mv, dev(b[:, 0].copy()), dev(b[:, 1].copy()), 2, 3,
                                 n_accept_out=acc)
        else:
            smp = nk.nk_metropolis_sweep(r, ch, mv, dev(b[:, 0].copy()), dev(b[:, 1].copy()), 2,
                                         3, n_accept_out=acc)
        outs.append((smp.cpu().numpy(), ch.sigma.cpu().numpy(), acc.cpu().numpy(), ch.counter))
    (a_s, a_f, a_acc, a_c), (b_s, b_f, b_acc, b_c) = outs
    assert np.array_equal(a_s, b_s) and np.array_equal(a_f, b_f)
    assert np.array_equal(a_acc, b_acc) and a_c == b_c


CASES = [
    # move, n, m, complex, lattice L (square) or 0 (chain), ladders, replicas
    ("exchange", 12, 24, True, 0, 32, 4),
    ("flip", 10, 20, False, 0, 32, 3),
    ("flip", 16, 48, True, 0, 16, 5),
    ("exchange", 64, 1600, True, 8, 8, 2),
]


@pytest.mark.parametrize("move,n,m,cplx,L,nlad,R", CASES)
def test_ladders_follow_the_oracle(nk, move, n, m, cplx, L, nlad, R):
    scale = 0.03 if m >= 512 else 0.5 / np.sqrt(n)
    p = W.perturb_params(W.init_params(n, m, cplx, 0.01, 100 + n), scale, 7)
    sz = move == "exchange"
    s0 = W.init_chains(nlad * R, n, sz, 9)
    bonds = W.square_bonds(L) if L else W.chain_bonds(n)
    seed, counter, nd, ns = 4321, 5 * n, 2, 3
    samp, fin, cnt, nacc, nswap, marg = tempering.parallel_tempering(
        p, s0, R, move, bonds, 8, seed, counter, counter // n, nd, ns, return_margin=True)
    r = rbm_of(nk, p)
    ch = nk.Chains(s0, 8, seed)
    ch.counter = counter
    acc = torch.zeros(nlad * R, dtype=torch.int64, device="cuda")
    sw = torch.zeros(nlad * max(R - 1, 1), dtype=torch.int64, device="cuda")
    mv = nk.NK_MOVE_FLIP if move == "flip" else nk.NK_MOVE_EXCHANGE
    out = nk.nk_pt_sweep(r, ch, R, mv, dev(bonds[:, 0].copy()), dev(bonds[:, 1].copy()), nd, ns,
                         n_accept_out=acc, n_swap_out=sw)
    assert ch.counter == cnt
    ok = marg > EPS_TIE
    print(f"\nPT {move} n={n} m={m} R={R}: {ok.sum()} of {nlad} ladders away from ties, "
          f"{nswap.sum()} exchanges")
    assert ok.sum() >= nlad // 2
    assert nswap.sum() > 0
    got = out.cpu().numpy().reshape(nlad, ns, n)
    assert np.array_equal(got[ok], samp.reshape(nlad, ns, n)[ok])
    rok = np.repeat(ok, R)
    assert np.array_equal(ch.sigma.cpu().numpy()[rok], fin[rok])
    assert np.array_equal(acc.cpu().numpy()[rok], nacc[rok])
    if R > 1:
        assert np.array_equal(sw.cpu().numpy().reshape(nlad, R - 1)[ok], nswap[ok])


@pytest.mark.parametrize("move", ["flip", "exchange"])
def test_every_replica_samples_its_tempered_distribution(nk, move):
    n, m, R, nlad = 8, 8, 3, 4096
    sz = move == "exchange"
    p = W.init_params(n, m, True, 0.35, 31)
    xs = hamiltonian.basis(n, sz)
    cf = hamiltonian.configs(xs, n)
    lv = 2.0 * np.real(rbm.logpsi(p, cf))
    r = rbm_of(nk, p)
    ch = nk.Chains(W.init_chains(nlad * R, n, sz, 12), 8, 2024)
    b = W.chain_bonds(n)
    sw = torch.zeros(nlad * (R - 1), dtype=torch.int64, device="cuda")
    mv = nk.NK_MOVE_FLIP if move == "flip" else nk.NK_MOVE_EXCHANGE
    nk.nk_pt_sweep(r, ch, R, mv, dev(b[:, 0].copy()), dev(b[:, 1].copy()), 200, 0, n_swap_out=sw)
    assert sw.sum().item() > 0
    fin = ch.sigma.cpu().numpy().astype(np.int64)
    betas = tempering.ladder(R)
    for k in range(R):
        target = np.exp(betas[k] * (lv - lv.max()))
        target /= target.sum()
        ints = ((1 - fin[k::R]) // 2) @ (1 << np.arange(n))
        c = np.bincount(np.searchsorted(xs, ints), minlength=len(xs)).astype(np.float64)
        exp = target * nlad
        keep = exp >= 5
        chi2 = np.sum((c[keep] - exp[keep]) ** 2 / exp[keep])
        dof = keep.sum() - 1
        assert chi2 < dof + 5 * np.sqrt(2 * dof), (k, chi2, dof)
