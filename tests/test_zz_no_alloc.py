"""The allocation-free SR step (nk_sr_step_noalloc) for callers that cannot
allocate device memory, e.g. code inside a framework that owns the device
allocator, or a plugin that is given only a stream and its tensors.  It must
give the same result as nk_sr_step with caller-provided scratch, on two calls
in a row (the built-in scratch array keeps the previous call's contents), and
reject problems whose scratch exceeds the built-in size.

This file is named so that pytest collects it last."""
import numpy as np
import pytest
import torch

from paper_1904_00031_gb300 import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def nk():
    from paper_1904_00031_gb300 import build, nk as nkmod
    build.build()
    nkmod.load_library()
    return nkmod


def _setup(nk, n, m, cplx, ns, seed):
    p = W.perturb_params(W.init_params(n, m, cplx, 0.01, seed), 0.2 / np.sqrt(n), seed + 1)
    op = W.heisenberg(n, W.chain_bonds(n), 1.0, True, W.sublattice(n)) if cplx else \
        W.ising(n, W.chain_bonds(n), h=1.0)
    s = torch.from_numpy(W.random_configs(ns, n, seed + 2, cplx)).cuda()
    gop = nk.Operator(op)
    rbms = []
    for _ in range(2):
        r = nk.Rbm(n, m, cplx)
        r.load(p.a, p.b, p.w)
        rbms.append(r)
    th = torch.empty(ns, m, dtype=rbms[0].f32_dtype(), device="cuda")
    nk.nk_rbm_logpsi(rbms[0], s, theta_out=th)
    t = torch.empty_like(th)
    e = nk.nk_local_energy(rbms[0], gop, s, th, t_out=t)
    return rbms, s, t, e


@pytest.mark.parametrize("cplx", [False, True])
@pytest.mark.parametrize("prec", [0, 1])
def test_noalloc_matches_caller_scratch_twice(nk, cplx, prec):
    """Both precisions: the BF16 hi + lo path also places its sigma' planes, the
    split direction and its tensor maps inside the built-in array."""
    n, m, ns, nc = 16, 32, 2048, 64
    (ra, rb), s, t, e = _setup(nk, n, m, cplx, ns, 5)
    scratch = nk.sr_scratch(ra, ns)
    for call in range(2):
        ia = nk.info_dict(nk.nk_sr_step(ra, s, t, e, nc, 0.01, 0.05, 30, prec=prec,
                                        scratch=scratch))
        ib = nk.info_dict(nk.nk_sr_step_noalloc(rb, s, t, e, nc, 0.01, 0.05, 30, prec=prec))
        torch.cuda.synchronize()
        for k in ("energy", "variance", "error", "cg_iters", "f_norm", "cg_resid"):
            assert ia[k] == pytest.approx(ib[k], rel=1e-12, abs=1e-300), (call, k)
        for xa, xb in zip(ra.params_numpy(), rb.params_numpy()):
            assert np.allclose(xa, xb, rtol=1e-12, atol=1e-15), call


def test_noalloc_rejects_oversized_problems(nk):
    n, m = 400, 1600
    r = nk.Rbm(n, m, True)
    need = nk.load_library().nk_sr_scratch_bytes(n, m, 1, 65536)
    assert need > nk.NK_SR_NOALLOC_MAX_BYTES
    s = torch.zeros(65536, n, dtype=torch.int8, device="cuda")
    t = torch.zeros(1, dtype=torch.complex64, device="cuda")
    e = torch.zeros(1, dtype=torch.complex128, device="cuda")
    with pytest.raises(nk.NkError, match="built-in"):
        nk.nk_sr_step_noalloc(r, s, t, e, 16384, 0.01, 0.01, 5)
