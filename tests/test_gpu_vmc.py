"""End-to-end VMC + SR runs through the C ABI, compared with the FP64 oracle's
runs on the same workloads and seeds (traces in tests/golden/vmc_*.json, written
by tests/golden/make_vmc_golden.py) and with exact ground energies.

Criterion (the two trajectories differ: FP32 vs FP64 arithmetic and near-tie
accept decisions): mean energy of the last 50 iterations, error bar from blocks
of 10 iterations; |E_gpu - E_oracle| <= 3 sqrt(err_gpu^2 + err_oracle^2), and
neither lies below the exact ground energy by more than 3 error bars."""
import json
import os

import numpy as np
import pytest
import torch

from paper_1904_00031_gb300 import workloads as W

pytestmark = pytest.mark.gpu
GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


@pytest.fixture(scope="module")
def mods():
    from paper_1904_00031_gb300 import build, nk
    from paper_1904_00031_gb300.vmc import VmcSr
    build.build()
    nk.load_library()
    return nk, VmcSr


def blocked(e, block=10):
    e = np.asarray(e[-50:])
    means = e.reshape(-1, block).mean(axis=1)
    return float(e.mean()), float(means.std(ddof=1) / np.sqrt(len(means)))


def workload_of(name):
    if name == "tfim10":
        return W.workload("c1")
    n = 12
    return W.Workload("heisenberg1d_n12_alpha2", n, 2 * n, True,
                      W.heisenberg(n, W.chain_bonds(n), 1.0, True, W.sublattice(n)), "exchange",
                      W.chain_bonds(n), True, 256, 4, 1, 0.01, 0.02, 50, 77)


@pytest.mark.parametrize("name", ["tfim10", "heis12"])
@pytest.mark.parametrize("prec", [0, 1])
def test_vmc_energy_matches_oracle(mods, name, prec):
    nk, VmcSr = mods
    path = os.path.join(GOLDEN, f"vmc_{name}.json")
    g = json.load(open(path))
    w = workload_of(name)
    w.lr = g["lr"]
    p = W.init_params(w.n, w.m, w.is_complex, 0.01, w.seed)
    v = VmcSr(w, p, prec=prec)
    energies = []
    for _ in range(len(g["energies"])):
        v.step()
        energies.append(v.info()["energy"])
    e_gpu, s_gpu = blocked(energies)
    e_or, s_or = g["last50_mean"], g["last50_err"]
    comb = np.sqrt(s_gpu ** 2 + s_or ** 2)
    assert abs(e_gpu - e_or) <= 3 * comb, (e_gpu, s_gpu, e_or, s_or)
    assert e_gpu >= g["e_exact"] - 3 * s_gpu
    assert e_or >= g["e_exact"] - 3 * s_or


def _criterion(g, energies):
    e_gpu, s_gpu = blocked(energies)
    e_or, s_or = g["last50_mean"], g["last50_err"]
    comb = np.sqrt(s_gpu ** 2 + s_or ** 2)
    assert abs(e_gpu - e_or) <= 3 * comb, (g["name"], e_gpu, s_gpu, e_or, s_or)
    if g["e_exact"] is not None:
        assert e_gpu >= g["e_exact"] - 3 * s_gpu
        assert e_or >= g["e_exact"] - 3 * s_or
    return e_gpu, s_gpu, e_or, s_or


@pytest.mark.parametrize("prec", [0, 1])
def test_vmc_energy_matches_oracle_heisenberg40(mods, prec):
    """The 40-site Heisenberg workload (complex RBM alpha = 2, 4096 chains x 4
    samples, exchange moves, SR with 50 CG iterations), 150 iterations from the
    same seeds as the oracle's run (tests/golden/vmc_c2.json)."""
    nk, VmcSr = mods
    g = json.load(open(os.path.join(GOLDEN, "vmc_c2.json")))
    w = W.workload("c2")
    p = W.init_params(w.n, w.m, w.is_complex, 0.01, w.seed)
    v = VmcSr(w, p, prec=prec, graph=True)
    energies = []
    for _ in range(len(g["energies"])):
        v.step()
        energies.append(v.info()["energy"])
    e_gpu, s_gpu, e_or, s_or = _criterion(g, energies)
    print(f"\nHeisenberg N=40 prec={prec}: GPU {e_gpu:.4f} +- {s_gpu:.4f}, "
          f"oracle {e_or:.4f} +- {s_or:.4f}")


@pytest.mark.parametrize("prec", [0, 1])
def test_batched_instances_match_oracle_runs(mods, prec):
    """All 64 uneven 1D instances advanced together (one graph per iteration,
    batched SR at BF16 hi + lo) for 100 iterations; the energy traces of
    instances 0, 2, 3 and 8 (TFIM n = 82 alpha 4, Heisenberg n = 32 alpha 4,
    TFIM n = 18 alpha 1, Heisenberg n = 64 alpha 2) against the oracle's runs of
    those instances alone (tests/golden/vmc_c4_*.json)."""
    nk, _ = mods
    from paper_1904_00031_gb300.batch import BatchedVmc
    insts = W.batched_instances(64, 4242, 1024)
    b = BatchedVmc(insts, prec=prec, graph=True)
    keys = [0, 2, 3, 8]
    goldens = {k: json.load(open(os.path.join(GOLDEN, f"vmc_c4_{k}.json"))) for k in keys}
    traces = {k: [] for k in keys}
    for _ in range(len(goldens[0]["energies"])):
        b.step()
        for k in keys:
            traces[k].append(b.items[k].info()["energy"])
    for k in keys:
        e_gpu, s_gpu, e_or, s_or = _criterion(goldens[k], traces[k])
        print(f"\ninstance {k} prec={prec}: GPU {e_gpu:.4f} +- {s_gpu:.4f}, "
              f"oracle {e_or:.4f} +- {s_or:.4f}")


def test_heisenberg20_listing_run(mods):
    """The VMC listing of Sec. 3.1 (1D Heisenberg N=20, S^z=0, RBM alpha=1, init
    sigma 0.01 seed 1234, exchange moves, 1000 samples per iteration, SR with an
    iterative solver, lr 0.01), 200 iterations; the paper reports a relative error
    of 4.16e-5 (Fig. 2), with SR settings it does not state.  With this build's
    reading (absolute diagonal shift 0.01, learning rate 0.01) the run is still
    converging at 200 iterations (relative error ~3e-3).  Checked: the variational
    bound, and a relative error below 1e-2 for the last 50 iterations."""
    nk, VmcSr = mods
    n = 20
    op = W.heisenberg(n, W.chain_bonds(n), 1.0, True, W.sublattice(n))
    w = W.Workload("heisenberg1d_n20_alpha1", n, n, True, op, "exchange", W.chain_bonds(n), True,
                   16, 63, 7, 0.01, 0.01, 200, 1234)
    from oracle import hamiltonian
    e_exact = hamiltonian.lanczos_ground(op, True)[0]  # S^z = 0 sector, Pauli units
    p = W.init_params(w.n, w.m, True, 0.01, 1234)
    v = VmcSr(w, p, prec=nk.NK_PREC_FP32)
    energies = []
    for _ in range(200):
        v.step()
        energies.append(v.info()["energy"])
    e, s = blocked(energies)
    assert e >= e_exact - 3 * s
    rel = abs((e - e_exact) / e_exact)
    print(f"heisenberg N=20 listing run: E = {e:.5f} +- {s:.5f}, exact {e_exact:.5f}, rel {rel:.2e}")
    assert rel < 1e-2, (e, s)


def test_listing_run_readings(mods):
    """The Sec. 3.1 listing run (Fig. 2 reports a relative error of 4.16e-5) under
    readings of its unstated settings, 200 iterations each: the Marshall-rotated
    Hamiltonian (this build's reading) or the unrotated one, 1,008 or 4,032
    samples per iteration, diagonal shift 0.01 or 0.001.  Relative errors of the
    mean energy over iterations 91-100 and 191-200 are printed (pytest -s); every
    run must respect the variational bound."""
    nk, VmcSr = mods
    from oracle import hamiltonian
    n = 20
    rows = []
    for marshall, spc, eps in [(True, 63, 0.01), (False, 63, 0.01), (True, 252, 0.01),
                               (True, 63, 0.001)]:
        op = W.heisenberg(n, W.chain_bonds(n), 1.0, marshall, W.sublattice(n))
        e_exact = hamiltonian.lanczos_ground(op, True)[0]
        w = W.Workload("heisenberg1d_n20_alpha1", n, n, True, op, "exchange", W.chain_bonds(n),
                       True, 16, spc, max(1, -(-spc // 10)), eps, 0.01, 200, 1234)
        v = VmcSr(w, W.init_params(n, n, True, 0.01, 1234), prec=nk.NK_PREC_FP32, graph=True)
        energies = []
        for _ in range(200):
            v.step()
            energies.append(v.info()["energy"])
        e100 = float(np.mean(energies[90:100]))
        e200 = float(np.mean(energies[190:200]))
        _, s200 = blocked(energies)
        rows.append((marshall, 16 * spc, eps, abs((e100 - e_exact) / e_exact),
                     abs((e200 - e_exact) / e_exact)))
        assert float(np.mean(energies[150:])) >= e_exact - 3 * s200
    print("\n| Marshall rotation | samples | diag shift | rel. error at 100 | rel. error at 200 |")
    for r in rows:
        print(f"| {r[0]} | {r[1]} | {r[2]} | {r[3]:.2e} | {r[4]:.2e} |")


@pytest.mark.parametrize("prec", [0, 1])
def test_graph_replay_equals_eager(mods, prec):
    """A captured iteration replays the same arithmetic: with the Philox counter on
    the device, K graph replays give bit-identical parameters to K eager steps."""
    nk, VmcSr = mods
    w = workload_of("heis12")
    p = W.init_params(w.n, w.m, w.is_complex, 0.01, w.seed)
    a = VmcSr(w, p, prec=prec, graph=False)
    b = VmcSr(w, p, prec=prec, graph=True)
    a.chains.counter_dev = None
    for _ in range(4):
        a.step()
        b.step()
    torch.cuda.synchronize()
    for xa, xb in zip(a.rbm.params_numpy(), b.rbm.params_numpy()):
        assert np.array_equal(xa, xb)
    assert np.array_equal(a.chains.sigma.cpu().numpy(), b.chains.sigma.cpu().numpy())
    assert b.chains.counter == a.chains.counter


@pytest.mark.parametrize("prec", [0, 1])
def test_tempering_iteration_matches_oracle_heis12(mods, prec):
    """The VMC iteration with the parallel-tempering sampler (ladders of 3
    replicas, only the beta = 1 replica recorded) samples the same |psi|^2 as the
    plain sampler, so its energies meet the criterion against the oracle's run of
    the plain sampler on the same workload."""
    nk, VmcSr = mods
    g = json.load(open(os.path.join(GOLDEN, "vmc_heis12.json")))
    w = workload_of("heis12")
    w.lr = g["lr"]
    p = W.init_params(w.n, w.m, w.is_complex, 0.01, w.seed)
    v = VmcSr(w, p, prec=prec, replicas=3)
    energies = []
    for _ in range(len(g["energies"])):
        v.step()
        energies.append(v.info()["energy"])
    _criterion(dict(g, name="heis12, tempering sampler"), energies)
    inf = v.info()
    assert 0.0 < inf["acceptance"] < 1.0
    assert 0.0 < inf["exchange_rate"] <= 1.0


def test_tempering_graph_replay_equals_eager(mods):
    """With the tempering sampler a captured iteration also replays the eager
    arithmetic bit for bit (the device counter advances once per sweep)."""
    nk, VmcSr = mods
    w = workload_of("heis12")
    p = W.init_params(w.n, w.m, w.is_complex, 0.01, w.seed)
    a = VmcSr(w, p, prec=nk.NK_PREC_BF16X2, graph=False, replicas=2)
    b = VmcSr(w, p, prec=nk.NK_PREC_BF16X2, graph=True, replicas=2)
    a.chains.counter_dev = None
    for _ in range(4):
        a.step()
        b.step()
    torch.cuda.synchronize()
    for xa, xb in zip(a.rbm.params_numpy(), b.rbm.params_numpy()):
        assert np.array_equal(xa, xb)
    assert np.array_equal(a.chains.sigma.cpu().numpy(), b.chains.sigma.cpu().numpy())
    assert np.array_equal(a.n_swap.cpu().numpy(), b.n_swap.cpu().numpy())
    assert b.chains.counter == a.chains.counter


def test_symmetric_rbm_heisenberg20(mods):
    """The same listing run with the translation-symmetric RBM (alpha = 1: one
    filter of 20 weights, 22 parameters instead of 440), SR in the tied space:
    the variational bound and a relative error below 1e-2 for the last 50 of 200
    iterations, and the untied RBM stays the expansion of the tied parameters."""
    nk, _ = mods
    from oracle import hamiltonian, rbm_symm
    from paper_1904_00031_gb300.vmc import VmcSrSymm
    n = 20
    op = W.heisenberg(n, W.chain_bonds(n), 1.0, True, W.sublattice(n))
    w = W.Workload("heisenberg1d_n20_symm_alpha1", n, n, True, op, "exchange", W.chain_bonds(n),
                   True, 16, 63, 7, 0.01, 0.01, 200, 1234)
    e_exact = hamiltonian.lanczos_ground(op, True)[0]
    perm = W.chain_translations(n)
    v = VmcSrSymm(w, W.init_symm_params(n, 1, True, 0.01, 1234), perm,
                  prec=nk.NK_PREC_BF16X2)
    energies = []
    for _ in range(200):
        v.step()
        energies.append(v.info()["energy"])
    e, s = blocked(energies)
    assert e >= e_exact - 3 * s
    assert abs((e - e_exact) / e_exact) < 1e-2, (e, e_exact)
    a, b, wt = v.sy.params_numpy()
    ref = rbm_symm.expand(W.RbmSymmParams(a, b, wt), perm)
    ua, ub, uw = v.rbm.params_numpy()
    assert np.array_equal(ua, ref.a) and np.array_equal(ub, ref.b) and np.array_equal(uw, ref.w)


def test_symmetric_graph_replay_equals_eager(mods):
    nk, _ = mods
    from paper_1904_00031_gb300.vmc import VmcSrSymm
    w = workload_of("heis12")
    perm = W.translations(w)
    p = W.init_symm_params(w.n, w.m // w.n, w.is_complex, 0.01, w.seed)
    a = VmcSrSymm(w, p, perm, prec=nk.NK_PREC_BF16X2, graph=False)
    b = VmcSrSymm(w, p, perm, prec=nk.NK_PREC_BF16X2, graph=True)
    a.chains.counter_dev = None
    for _ in range(4):
        a.step()
        b.step()
    torch.cuda.synchronize()
    for xa, xb in zip(a.sy.params_numpy(), b.sy.params_numpy()):
        assert np.array_equal(xa, xb)
