"""Uneven independent instances advanced together (per-instance streams captured
into one CUDA graph): each instance's first iteration must reproduce the oracle's
energy statistics and force on the same seeded chains (the first sweep's
trajectories coincide except at near-ties, which the margin filter rules out)."""
import numpy as np
import pytest
import torch

from oracle import local_energy as ole
from oracle import rbm as orbm
from oracle import sampler as osam
from oracle import sr as osr
from paper_1904_00031_gb300 import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def mods():
    from paper_1904_00031_gb300 import build, nk
    from paper_1904_00031_gb300.batch import BatchedVmc
    build.build()
    nk.load_library()
    return nk, BatchedVmc


def test_batched_first_iteration_per_instance(mods):
    nk, BatchedVmc = mods
    insts = W.batched_instances(n_inst=6, seed=4242, n_chains=64)
    for w in insts:
        w.n_cg = 10
    b = BatchedVmc(insts, prec=nk.NK_PREC_FP32, graph=True)
    b.step()                     # eager first iteration (then captured)
    torch.cuda.synchronize()
    for v, w in zip(b.items, insts):
        p = W.init_params(w.n, w.m, w.is_complex, 0.01, w.seed)
        s0 = W.init_chains(w.n_chains, w.n, w.zero_magnetisation, w.seed)
        samp, fin, cnt, nacc, marg = osam.metropolis(
            p, s0, w.move, w.sampler_bonds, w.group_size, w.seed, 0, w.n_discard,
            w.samples_per_chain, return_margin=True)
        if marg.min() < 1e-3:
            continue  # a near-tie: trajectories may legitimately differ
        got = v.samples.cpu().numpy()
        assert np.array_equal(got, samp), w.name
        e = ole.local_energy_rbm(p, w.op, samp)
        mean, var, err = osr.stats(e, w.n_chains)
        info = v.info()
        assert abs(info["energy"] - mean.real) <= 1e-6 * abs(mean.real), w.name
        sig, t = orbm.logderiv_factored(p, samp)
        f = osr.force_lazy(sig, t, e, w.n, w.m, None, not w.is_complex)
        assert abs(info["f_norm"] - np.linalg.norm(f)) <= 1e-5 * np.linalg.norm(f), w.name
    for _ in range(3):
        b.step()                 # graph replays
    torch.cuda.synchronize()
    for v in b.items:
        assert np.isfinite(v.info()["energy"])


def test_batched_sr_step_equals_per_instance_steps(mods):
    """nk_sr_step_batch (one launch per kernel for all instances of a field) runs
    each instance's arithmetic in the order nk_sr_step does: with the same split
    count, one iteration of the batch reproduces the per-instance SR steps bit
    for bit (parameters and info vectors), for mixed real / complex, uneven
    instances."""
    nk, BatchedVmc = mods
    insts = W.batched_instances(n_inst=7, seed=77, n_chains=96)
    for w in insts:
        w.n_cg = 12
    a = BatchedVmc(insts, prec=nk.NK_PREC_BF16X2, graph=False, batch_sr=True, sr_splits=2)
    b = BatchedVmc(insts, prec=nk.NK_PREC_BF16X2, graph=False, batch_sr=False, sr_splits=2)
    assert a.srb is not None and b.srb is None
    for _ in range(2):
        a.step()
        b.step()
    torch.cuda.synchronize()
    for va, vb in zip(a.items, b.items):
        assert np.array_equal(va.samples.cpu().numpy(), vb.samples.cpu().numpy())
        for xa, xb in zip(va.rbm.params_numpy(), vb.rbm.params_numpy()):
            assert np.array_equal(xa, xb), va.w.name
        assert np.array_equal(va.info_buf.cpu().numpy(), vb.info_buf.cpu().numpy()), va.w.name
        assert va.info()["cg_iters"] == 12


def test_batched_sr_graph_replays(mods):
    """The batched SR step inside the captured multi-instance iteration: replays
    keep every instance finite and the batch's energies decreasing on average."""
    nk, BatchedVmc = mods
    insts = W.batched_instances(n_inst=10, seed=5, n_chains=128)
    b = BatchedVmc(insts, prec=nk.NK_PREC_BF16X2, graph=True)
    assert b.srb is not None
    b.step()
    torch.cuda.synchronize()
    e0 = np.array([v.info()["energy"] for v in b.items])
    for _ in range(20):
        b.step()
    torch.cuda.synchronize()
    e1 = np.array([v.info()["energy"] for v in b.items])
    assert np.all(np.isfinite(e1))
    assert np.mean(e1 / np.abs(e0)) < np.mean(e0 / np.abs(e0))


def _batch_jobs(nk, vs, streams=None):
    sweep, amp, eloc = [], [], []
    for k, v in enumerate(vs):
        st = None if streams is None else streams[k]
        sweep.append(dict(rbm=v.rbm, chains=v.chains, move=v.move, bond_i=v.bond_i,
                          bond_k=v.bond_k, n_discard=v.w.n_discard,
                          n_samples_per_chain=v.w.samples_per_chain, samples_out=v.samples,
                          n_accept_out=v.n_acc, scratch=v.metro_scratch, stream=st))
        amp.append(dict(rbm=v.rbm, sigma=v.samples, logpsi_out=v.logpsi, theta_out=v.theta,
                        stream=st))
        eloc.append(dict(rbm=v.rbm, op=v.op, sigma=v.samples, theta=v.theta, eloc_out=v.eloc,
                         t_out=v.t, scratch=v.eloc_scratch, stream=st))
    return sweep, amp, eloc


@pytest.mark.parametrize("prec_name", ["fp32", "bf16x2"])
@pytest.mark.parametrize("own_streams", [False, True])
def test_batch_entry_points_equal_single_calls(mods, prec_name, own_streams):
    """nk_batch_sweep / nk_batch_logpsi / nk_batch_local_energy over uneven
    instances give bit for bit the results of the single calls (chains,
    accept counts, ln psi, theta, E_loc, tanh theta), also with one stream per
    item."""
    nk, _ = mods
    from paper_1904_00031_gb300.vmc import VmcSr
    prec = nk.NK_PREC_FP32 if prec_name == "fp32" else nk.NK_PREC_BF16X2
    insts = W.batched_instances(n_inst=5, seed=321, n_chains=64)
    mk = lambda w: VmcSr(w, W.init_params(w.n, w.m, w.is_complex, 0.05, w.seed), prec=prec)
    single = [mk(w) for w in insts]
    batch = [mk(w) for w in insts]
    for v in single:
        v.sample()
        nk.nk_rbm_logpsi(v.rbm, v.samples, prec, v.logpsi, v.theta)
        v.energies()
    streams = [torch.cuda.Stream() for _ in insts] if own_streams else None
    sweep, amp, eloc = _batch_jobs(nk, batch, streams)
    cur = torch.cuda.current_stream()
    if streams:
        for s in streams:
            s.wait_stream(cur)
    nk.nk_batch_sweep(sweep)
    nk.nk_batch_logpsi(amp, prec=prec)
    nk.nk_batch_local_energy(eloc)
    torch.cuda.synchronize()
    for a, b in zip(single, batch):
        for x, y in ((a.samples, b.samples), (a.n_acc, b.n_acc), (a.chains.sigma, b.chains.sigma),
                     (a.logpsi, b.logpsi), (a.theta, b.theta), (a.eloc, b.eloc), (a.t, b.t)):
            assert torch.equal(x, y), a.w.name
        assert a.chains.counter == b.chains.counter


def test_batch_entry_point_rejects_bad_item_before_enqueueing(mods):
    nk, _ = mods
    from paper_1904_00031_gb300.vmc import VmcSr
    insts = W.batched_instances(n_inst=3, seed=5, n_chains=32)
    vs = [VmcSr(w, W.init_params(w.n, w.m, w.is_complex, 0.05, w.seed)) for w in insts]
    sweep, amp, eloc = _batch_jobs(nk, vs)
    before = [v.samples.clone() for v in vs]
    counters = [v.chains.counter for v in vs]
    sweep[2]["scratch"] = None if sweep[2]["scratch"] is None else sweep[2]["scratch"][:256]
    sweep[2]["n_samples_per_chain"] = -1
    with pytest.raises(nk.NkError, match="item 2"):
        nk.nk_batch_sweep(sweep)
    torch.cuda.synchronize()
    for v, s0, c0 in zip(vs, before, counters):
        assert torch.equal(v.samples, s0)      # nothing ran, item 0 included
        assert v.chains.counter == c0
