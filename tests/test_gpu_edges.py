"""Edge sizes of the CUDA path against the FP64 oracle: the largest visible
count the tensor-core path takes (n + 1 = 448), the largest hidden count the
Metropolis kernel keeps in registers and tensor memory (m = 2048), ragged
sample tiles, and calls with nothing to do (no samples, no chains, no sweeps),
which must leave every output and the chain counter untouched."""
import numpy as np
import pytest
import torch

from oracle import local_energy as ole
from oracle import rbm as orbm
from oracle import sampler as osam
from paper_1904_00031_gb300 import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def nk():
    from paper_1904_00031_gb300 import build, nk as nkmod
    build.build()
    nkmod.load_library()
    return nkmod


def make_rbm(nk, p):
    r = nk.Rbm(p.n, p.m, p.is_complex)
    r.load(p.a, p.b, p.w)
    return r


def dev(x):
    return torch.from_numpy(np.ascontiguousarray(x)).cuda()


@pytest.mark.parametrize("cplx", [False, True])
def test_logpsi_bf16x2_widest_visible_layer(nk, cplx):
    """n = 447 (n + 1 = 448 = 7 K-chunks of 64), 131 samples (two tiles, ragged)."""
    n, m, ns = 447, 70, 131
    p = W.perturb_params(W.init_params(n, m, cplx, 0.01, 12), 0.5 / np.sqrt(n), 13)
    s = W.random_configs(ns, n, 14)
    r = make_rbm(nk, p)
    got = nk.nk_rbm_logpsi(r, dev(s), prec=nk.NK_PREC_BF16X2).cpu().numpy()
    ref = orbm.logpsi(p, s)
    scale = np.maximum(1.0, np.abs(ref))
    assert np.all(np.abs(got.real - ref.real) <= 1e-4 * scale)
    assert np.all(np.abs(np.angle(np.exp(1j * (got.imag - ref.imag)))) <= 1e-4 * scale)


def test_logpsi_bf16x2_rejects_too_wide(nk):
    p = W.init_params(448, 16, False, 0.01, 1)
    r = make_rbm(nk, p)
    with pytest.raises(nk.NkError):
        nk.nk_rbm_logpsi(r, dev(W.random_configs(4, 448, 1)), prec=nk.NK_PREC_BF16X2)


@pytest.mark.parametrize("cplx,sampler,m", [(False, 0, 2048), (True, 1, 2048), (True, 0, 2048),
                                             (True, 4, 2304)])
def test_metropolis_widest_hidden_layer(nk, cplx, sampler, m):
    """The largest hidden layers the samplers hold on chip: m = 2048 with warps
    per chain, 2048 and 2304 with one CTA per proposal group."""
    n, nc, G = 8, 16, 4
    p = W.perturb_params(W.init_params(n, m, cplx, 0.01, 21), 0.05, 22)
    s0 = W.init_chains(nc, n, False, 23)
    bonds = W.chain_bonds(n)
    seed, counter, nd, nsamp = 99, 0, 1, 2
    samp, fin, cnt, nacc, marg = osam.metropolis(p, s0, "flip", bonds, G, seed, counter, nd, nsamp,
                                                 return_margin=True)
    r = make_rbm(nk, p)
    r._s.sampler = sampler
    ch = nk.Chains(s0, G, seed)
    acc = torch.zeros(nc, dtype=torch.int64, device="cuda")
    out = nk.nk_metropolis_sweep(r, ch, nk.NK_MOVE_FLIP, None, None, nd, nsamp, n_accept_out=acc)
    assert ch.counter == cnt
    ok = marg > 1e-3
    assert ok.sum() >= nc // 2
    got = out.cpu().numpy().reshape(nc, nsamp, n)
    assert np.array_equal(got[ok], samp.reshape(nc, nsamp, n)[ok])
    assert np.array_equal(acc.cpu().numpy()[ok], nacc[ok])


@pytest.mark.parametrize("cplx,m,G,sampler", [(True, 2049, 4, 1), (False, 2049, 4, 0),
                                              (True, 2049, 16, 0), (True, 2305, 4, 0),
                                              (True, 1025, 4, 2), (True, 2049, 4, 3),
                                              (True, 40, 16, 3), (False, 40, 4, 3),
                                              (True, 40, 4, 5)])
def test_metropolis_rejects_shapes_out_of_range(nk, cplx, m, G, sampler):
    """Hidden layers beyond what a sampler holds on chip, the group kernel on a
    real RBM or with more than 8 chains per group, an unknown sampler."""
    p = W.init_params(8, m, cplx, 0.01, 2)
    r = make_rbm(nk, p)
    r._s.sampler = sampler
    ch = nk.Chains(W.init_chains(G, 8, False, 3), G, 5)
    with pytest.raises(nk.NkError):
        nk.nk_metropolis_sweep(r, ch, nk.NK_MOVE_FLIP, None, None, 1, 1)
    assert ch.counter == 0


def test_calls_with_nothing_to_do(nk):
    n, m = 12, 24
    p = W.init_params(n, m, True, 0.01, 4)
    r = make_rbm(nk, p)
    op = nk.Operator(W.heisenberg(n, W.chain_bonds(n), 1.0, True, W.sublattice(n)))
    # no samples: the local energy call enqueues nothing and touches no output
    sentinel = torch.full((3,), 7.0, dtype=torch.complex128, device="cuda")
    empty_s = torch.empty(0, n, dtype=torch.int8, device="cuda")
    empty_t = torch.empty(0, m, dtype=torch.complex64, device="cuda")
    nk.nk_local_energy(r, op, empty_s, empty_t, eloc_out=sentinel)
    assert torch.all(sentinel == 7.0)
    # no sweeps: chains, counter and samples unchanged
    s0 = W.init_chains(8, n, True, 6)
    ch = nk.Chains(s0, 4, 9)
    out = torch.full((0, n), 3, dtype=torch.int8, device="cuda")
    nk.nk_metropolis_sweep(r, ch, nk.NK_MOVE_EXCHANGE, dev(W.chain_bonds(n)[:, 0].copy()),
                           dev(W.chain_bonds(n)[:, 1].copy()), 0, 0, samples_out=out)
    assert ch.counter == 0
    assert np.array_equal(ch.sigma.cpu().numpy(), s0)
    # the batch calls with no items
    nk.nk_batch_logpsi([])
    nk.nk_batch_sweep([])
    nk.nk_batch_local_energy([])
    torch.cuda.synchronize()
