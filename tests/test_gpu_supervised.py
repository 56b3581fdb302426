"""Supervised learning on the GPU (nk_supervised_step: the overlap loss of Eq. 1,
its gradient, AdaMax) against the oracle (oracle/supervised.py) on the
workload of the paper's supervised example: the ground state of the 10-site
periodic TFIM chain (h = 1) from exact diagonalisation as the target, an RBM
with 20 hidden units initialised N(0, 0.01^2) from seed 1234, batches of 400
samples drawn from |target|^2, AdaMax with its default settings.

Tolerances: loss abs 1e-6 (FP32) / 1e-5 (BF16 hi + lo); gradient rel 1e-5 /
1e-4 norm-wise (the gradient target is rel 1e-4); parameters along a 40-step
AdaMax trajectory abs 1e-6 / 1e-5 (AdaMax steps are lr m / u, bounded by lr)."""
import numpy as np
import pytest
import torch

from oracle import hamiltonian, supervised
from paper_1904_00031_gb300 import workloads as W

pytestmark = pytest.mark.gpu

N, M, NS = 10, 20, 400
TOL = {0: dict(loss=1e-6, grad=1e-5, par=1e-6), 1: dict(loss=1e-5, grad=1e-4, par=1e-5)}


@pytest.fixture(scope="module")
def nk():
    from paper_1904_00031_gb300 import build, nk as nkmod
    build.build()
    nkmod.load_library()
    return nkmod


@pytest.fixture(scope="module")
def target():
    op = W.ising(N, W.chain_bonds(N), h=1.0)
    _, vec, xs = hamiltonian.exact_ground(op)
    cf = hamiltonian.configs(xs, N)
    tar = np.asarray(vec, dtype=np.complex128)
    tar = tar * np.sign(tar.real.sum())          # the ground state is positive up to a sign
    prob = np.abs(tar) ** 2
    return cf, tar, prob / prob.sum()


def batch(target, seed):
    cf, tar, prob = target
    idx = np.random.default_rng(seed).choice(len(cf), NS, p=prob)
    return cf[idx], tar[idx]


def rbm_of(nk, p):
    r = nk.Rbm(p.n, p.m, p.is_complex)
    r.load(p.a, p.b, p.w)
    return r


@pytest.mark.parametrize("cplx", [False, True])
@pytest.mark.parametrize("prec", [0, 1])
def test_loss_and_gradient(nk, target, cplx, prec):
    p = W.perturb_params(W.init_params(N, M, cplx, 0.01, 1234), 0.1, 5)
    s, t = batch(target, 11)
    loss, g = supervised.overlap_loss_and_grad(p, s, t)
    r = rbm_of(nk, p)
    dt = torch.complex128 if cplx else torch.float64
    grad = torch.empty(p.n_params, dtype=dt, device="cuda")
    info = nk.nk_supervised_step(r, torch.from_numpy(s).cuda(), torch.from_numpy(np.log(t)).cuda(),
                                 prec=prec, grad_out=grad).cpu().numpy()
    gg = grad.cpu().numpy()
    assert abs(info[0] - loss) <= TOL[prec]["loss"], (info[0], loss)
    assert abs(info[1] - np.exp(-loss)) <= TOL[prec]["loss"]
    assert info[3] == 0.0
    assert np.linalg.norm(gg - g) <= TOL[prec]["grad"] * np.linalg.norm(g), \
        np.linalg.norm(gg - g) / np.linalg.norm(g)


@pytest.mark.parametrize("cplx", [False, True])
def test_weighted_full_sum_equals_the_overlap(nk, target, cplx):
    """Every basis state as a sample with weight |tar|^2: the loss is the exact
    negative log overlap of Eq. 1 (summed, not sampled)."""
    cf, tar, prob = target
    p = W.perturb_params(W.init_params(N, M, cplx, 0.01, 1234), 0.2, 6)
    ref = supervised.overlap_loss_full(p, cf, tar)
    r = rbm_of(nk, p)
    info = nk.nk_supervised_step(r, torch.from_numpy(cf).cuda(),
                                 torch.from_numpy(np.log(tar)).cuda(),
                                 weights=torch.from_numpy(prob * 7.0).cuda()).cpu().numpy()
    assert abs(info[0] - ref) <= 1e-6, (info[0], ref)


@pytest.mark.parametrize("cplx", [False, True])
@pytest.mark.parametrize("prec", [0, 1])
def test_adamax_trajectory(nk, target, cplx, prec):
    """40 AdaMax steps on the same batches: parameters and losses follow the
    oracle's (oracle gradient + oracle AdaMax) step by step."""
    p = W.init_params(N, M, cplx, 0.01, 1234)
    r = rbm_of(nk, p)
    opt = supervised.AdaMax()
    pr = p.n_params * (2 if cplx else 1)
    mom = torch.zeros(2 * pr, dtype=torch.float64, device="cuda")
    info = torch.zeros(4, dtype=torch.float64, device="cuda")
    scratch = nk.supervised_scratch(r, NS)
    for step in range(1, 41):
        s, t = batch(target, 1000 + step)
        loss, g = supervised.overlap_loss_and_grad(p, s, t)
        p = W.RbmParams.from_flat(opt.step(p.flat(), g), N, M)
        nk.nk_supervised_step(r, torch.from_numpy(s).cuda(), torch.from_numpy(np.log(t)).cuda(),
                              prec=prec, lr=opt.lr, beta1=opt.b1, beta2=opt.b2, step=step,
                              moments=mom, scratch=scratch, info_out=info)
        got = info.cpu().numpy()
        assert abs(got[0] - loss) <= max(TOL[prec]["loss"], 1e-4 * loss), (step, got[0], loss)
    a, b, w = r.params_numpy()
    gp = np.concatenate([a, b, w.reshape(-1)])
    assert np.abs(gp - p.flat()).max() <= TOL[prec]["par"], np.abs(gp - p.flat()).max()


def test_training_raises_the_overlap_like_the_oracle(nk, target):
    """The listing's setting (real RBM, 20 hidden units, batches of 400, AdaMax
    defaults) for 600 steps on both sides: the GPU's exact overlap (its own
    weighted full-sum evaluation) follows the oracle's run and rises well above
    the initial one."""
    cf, tar, prob = target
    p = W.init_params(N, M, False, 0.01, 1234)
    opt = supervised.AdaMax()
    r = rbm_of(nk, p)
    mom = torch.zeros(2 * p.n_params, dtype=torch.float64, device="cuda")
    scratch = nk.supervised_scratch(r, NS)
    full_s = torch.from_numpy(cf).cuda()
    full_lt = torch.from_numpy(np.log(tar)).cuda()
    full_w = torch.from_numpy(prob).cuda()
    ov0 = float(np.exp(-supervised.overlap_loss_full(p, cf, tar)))
    for step in range(1, 601):
        s, t = batch(target, 5000 + step)
        _, g = supervised.overlap_loss_and_grad(p, s, t)
        p = W.RbmParams.from_flat(opt.step(p.flat(), g), N, M)
        nk.nk_supervised_step(r, torch.from_numpy(s).cuda(), torch.from_numpy(np.log(t)).cuda(),
                              step=step, moments=mom, scratch=scratch)
    ov_or = float(np.exp(-supervised.overlap_loss_full(p, cf, tar)))
    ov_gpu = float(nk.nk_supervised_step(r, full_s, full_lt, weights=full_w)[1].item())
    print(f"\nsupervised TFIM N=10: overlap {ov0:.4f} -> GPU {ov_gpu:.5f}, oracle {ov_or:.5f}")
    assert abs(ov_gpu - ov_or) <= 1e-4
    assert ov_or > ov0 + 0.5 * (1.0 - ov0)
