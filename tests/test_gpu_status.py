"""Device-side failure reporting: a bounded wait that gives up sets a status bit
that nk_query_status returns (and clears), without hanging or faulting the GPU,
and the context stays usable afterwards.  The timeout is made by a probe that
waits for an mbarrier phase nothing completes; no kernel is broken."""
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


def _status(nk):
    f = nk.nk_query_status()
    torch.cuda.synchronize()
    return int(f.item())


def _logpsi_ok(nk):
    p = W.init_params(20, 40, True, 0.05, 11)
    r = nk.Rbm(p.n, p.m, p.is_complex)
    r.load(p.a, p.b, p.w)
    s = W.init_chains(64, p.n, False, 3)
    got = nk.nk_rbm_logpsi(r, torch.from_numpy(s).cuda(), prec=nk.NK_PREC_BF16X2).cpu().numpy()
    ref = orbm.logpsi(p, s)
    assert np.allclose(got.real, ref.real, rtol=1e-5, atol=1e-5)


def test_clean_runs_report_no_status(nk):
    _status(nk)  # clear whatever earlier tests left
    _logpsi_ok(nk)
    assert _status(nk) == 0


def test_timed_out_wait_is_reported_and_cleared(nk):
    _status(nk)
    nk.nk_debug_bounded_wait(4096)
    assert _status(nk) == 1 << nk.NK_ERR_TIMEOUT
    assert _status(nk) == 0          # the query cleared it
    _logpsi_ok(nk)                   # the context is still usable
    assert _status(nk) == 0


def test_status_host_argument_checks(nk):
    lib = nk.load_library()
    assert lib.nk_query_status(None, None) == nk.NK_ERR_INVALID_ARG
    assert lib.nk_debug_bounded_wait(0, None) == nk.NK_ERR_INVALID_ARG
    assert lib.nk_debug_bounded_wait((1 << 20) + 1, None) == nk.NK_ERR_INVALID_ARG


def test_measured_alu_peaks_are_plausible(nk):
    """The FP32 FMA rate lies between half and 1.2 times the unit-count figure
    (152 SMs x 128 lanes x 2 flop x the maximum clock); the MUFU rates are
    positive and below the FMA instruction rate."""
    pk = nk.nk_measure_alu_peaks()
    nominal = 152 * 128 * 2 * 2.07e9
    assert 0.5 * nominal < pk["fp32_fma_flops"] < 1.2 * nominal, pk
    for k in ("mufu_ex2_ops", "mufu_lg2_ops", "mufu_sin_ops"):
        assert 0 < pk[k] < pk["fp32_fma_flops"] / 2, pk
