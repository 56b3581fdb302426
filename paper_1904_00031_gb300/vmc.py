"""One VMC + SR iteration (Sec. 2.2.5) driven through the C ABI:

    nk_metropolis_sweep -> nk_rbm_logpsi (theta only) -> nk_local_energy
    (E_loc and T = tanh theta) -> nk_sr_step (statistics, force, lazy CG, update)

All buffers are allocated once; a step launches only library kernels and does
not synchronise the host (``info()`` reads the small FP64 status block).
"""
from __future__ import annotations

import numpy as np
import torch

from . import nk
from . import workloads as W


def centring_fused(ns: int, m: int, is_complex: bool) -> bool:
    """Whether the tensor-core SR forward writes the centring partials itself:
    one per CTA (sample tiles x hidden-tile halves) must fit 1024 slots.  The
    halves rule is the library's: two when the hidden tiles are at least two
    and twice the CTAs fill their last wave of 152 better."""
    tiles = (ns + 127) // 128
    mt = (m + 1 + (63 if is_complex else 127)) // (64 if is_complex else 128)

    def eff(b):
        return b / (((b + 151) // 152) * 152)

    nseg = 2 if mt >= 2 and eff(2 * tiles) > eff(tiles) else 1
    return tiles * nseg <= 1024


def error_blocks(n_chains: int, group_size: int) -> int:
    """Independent units of the energy error bar: the chains of one proposal
    group share their proposal sequence, so whole groups are the blocks (one
    block, i.e. no error bar, when the chains do not split into whole groups)."""
    return n_chains // group_size if n_chains % group_size == 0 else 1


def adj_centres(m: int, is_complex: bool) -> bool:
    """Whether the SR adjoint centres the forward's output itself (at most four
    parameter tiles of 64 complex or 128 real hidden units)."""
    per = 64 if is_complex else 128
    return (m + 1 + per - 1) // per <= 4


class VmcSr:
    def __init__(self, w: W.Workload, params: W.RbmParams | None, sigma0=None,
                 prec: int = nk.NK_PREC_FP32, device="cuda", graph: bool = False,
                 autotune: bool = False, rbm: nk.Rbm | None = None, replicas: int = 1):
        """``params`` are loaded into a new RBM, or ``rbm`` (already loaded and
        prepared, params None) is used as it is.  ``replicas`` > 1 samples by
        parallel tempering: every chain becomes a ladder of that many replicas
        (``sigma0``, if given, holds all n_chains * replicas states, ladder-major)
        and only the beta = 1 replicas are recorded."""
        self.w = w
        self.prec = prec
        self.replicas = int(replicas)
        if rbm is None:
            rbm = nk.Rbm(w.n, w.m, w.is_complex, device)
            rbm.load(params.a, params.b, params.w)
        self.rbm = rbm
        n_rep = w.n_chains * self.replicas
        if sigma0 is None:
            sigma0 = W.init_chains(n_rep, w.n, w.zero_magnetisation, w.seed)
        self.chains = nk.Chains(sigma0, w.group_size, w.seed, device, device_counter=graph)
        self.blocks = error_blocks(w.n_chains, w.group_size)
        self.use_graph = graph
        self.graph = None
        self.autotune = autotune
        self.tuned = False
        self.op = nk.Operator(w.op, device)
        b = np.ascontiguousarray(w.sampler_bonds, dtype=np.int32)
        self.bond_i = torch.from_numpy(b[:, 0].copy()).to(device)
        self.bond_k = torch.from_numpy(b[:, 1].copy()).to(device)
        ns = w.n_samples
        self.ns = ns
        self.samples = torch.empty(ns, w.n, dtype=torch.int8, device=device)
        f32 = self.rbm.f32_dtype()
        self.theta = torch.empty(ns, w.m, dtype=f32, device=device)
        self.t = torch.empty(ns, w.m, dtype=f32, device=device)
        self.logpsi = torch.empty(ns, dtype=torch.complex128, device=device)
        self.eloc = torch.empty(ns, dtype=torch.complex128, device=device)
        self.n_acc = torch.zeros(n_rep, dtype=torch.int64, device=device)
        self.n_swap = (torch.zeros(w.n_chains * (self.replicas - 1), dtype=torch.int64,
                                   device=device) if self.replicas > 1 else None)
        self.scratch = self._sr_scratch(device)
        self.info_buf = torch.zeros(nk.NK_INFO_LEN, dtype=torch.float64, device=device)
        self.move = nk.NK_MOVE_FLIP if w.move == "flip" else nk.NK_MOVE_EXCHANGE
        self.metro_scratch = (nk.metropolis_scratch(self.rbm, self.move, len(b), device)
                              if self.replicas == 1 else
                              nk.pt_scratch(self.rbm, self.move, len(b), n_rep, device))
        self.eloc_scratch = nk.local_energy_scratch(self.rbm, self.op, device)

    def _sr_scratch(self, device):
        return nk.sr_scratch(self.rbm, self.ns, device)

    # stages ---------------------------------------------------------------
    def sample(self):
        if self.replicas > 1:
            nk.nk_pt_sweep(self.rbm, self.chains, self.replicas, self.move, self.bond_i,
                           self.bond_k, self.w.n_discard, self.w.samples_per_chain, self.samples,
                           self.n_acc, self.n_swap, self.metro_scratch)
            return
        nk.nk_metropolis_sweep(self.rbm, self.chains, self.move, self.bond_i, self.bond_k,
                               self.w.n_discard, self.w.samples_per_chain, self.samples,
                               self.n_acc, self.metro_scratch)

    def amplitudes(self):
        """theta = W sigma + b of the samples (the local energies and T need theta;
        the iteration consumes no ln psi, so the ln cosh epilogue is skipped)."""
        nk.nk_rbm_theta(self.rbm, self.samples, self.theta, self.prec)

    def energies(self):
        nk.nk_local_energy(self.rbm, self.op, self.samples, self.theta, self.eloc, self.t,
                           self.eloc_scratch)

    def sr(self):
        nk.nk_sr_step(self.rbm, self.samples, self.t, self.eloc, self.blocks,
                      self.w.diag_shift, self.w.lr, self.w.n_cg, 1e-12, self.prec,
                      scratch=self.scratch, info_out=self.info_buf)

    def _eager_step(self):
        self.sample()
        self.amplitudes()
        self.energies()
        self.sr()

    def capture(self):
        """Capture one whole iteration in a CUDA graph (nothing runs during the
        capture; the Philox counter lives on the device, so every replay draws
        fresh random numbers).  Call after at least one eager step."""
        torch.cuda.synchronize()
        self.graph = torch.cuda.CUDAGraph()
        with torch.cuda.graph(self.graph):
            self._eager_step()

    def tune(self):
        """Autotune the tile shapes on the current samples (synchronises): the SR
        adjoint's split-K count, and the CTAs per tile of the theta contraction
        (tensor-core path) and of the local energies."""
        self.split_k = nk.nk_sr_tune(self.rbm, self.samples, self.t, self.prec, self.scratch)
        if self.prec == nk.NK_PREC_BF16X2:
            self.shapes = nk.nk_tune_shapes(self.rbm, self.op, self.samples, self.theta,
                                            self.eloc, self.eloc_scratch, self.t)
            # the tuner overwrote theta and E_loc: recompute them for the SR inputs
            self.amplitudes()
            self.energies()
        self.tuned = True

    def step(self):
        """One iteration.  The first call also autotunes (if asked) and, in graph
        mode, captures the graph; later graph-mode calls replay it."""
        if self.use_graph and self.graph is not None:
            self.graph.replay()
            return
        self._eager_step()
        if self.autotune and not self.tuned:
            self.tune()
        if self.use_graph:
            self.capture()

    def info(self) -> dict:
        d = nk.info_dict(self.info_buf)
        sweeps = self.w.n_discard + self.w.samples_per_chain
        d["acceptance"] = float(self.n_acc.sum().item()) / (self.w.n_chains * self.replicas *
                                                           sweeps * self.w.n)
        if self.n_swap is not None:
            d["exchange_rate"] = float(self.n_swap.sum().item()) / (
                self.w.n_chains * sweeps * (self.replicas - 1) / 2)
        return d

    def sr_launches(self) -> int:
        """Kernel launches of one SR step: statistics (3), force and CG start, the
        CG iterations, the update and the refreshed planes (2)."""
        if self.prec == nk.NK_PREC_BF16X2:
            # sigma'^T, sigma' rows, adjoint, reduction, CG start (2); per CG
            # iteration 7, or 5 when the forward writes the centring partials and
            # the adjoint centres its input itself (the first iteration also
            # builds the planes of p)
            fused = centring_fused(self.ns, self.w.m, self.w.is_complex)
            per = (5 if adj_centres(self.w.m, self.w.is_complex) else 6) if fused else 7
            return 3 + 6 + per * self.w.n_cg + 1 + 3
        # adjoint, reduction, CG start (2); 8 per CG iteration
        return 3 + 4 + 8 * self.w.n_cg + 3

    def param_tensors(self):
        """The FP64 master parameters a caller uploads (device tensors)."""
        return [self.rbm.a, self.rbm.b, self.rbm.w]

    def refresh(self):
        """Derive the kernels' planes after new master parameters were uploaded."""
        nk.nk_rbm_prepare(self.rbm)

    # kernel launches per step (for reporting)
    def launches_per_step(self) -> int:
        # move rows, sweep; with tempering a sweep launch and an exchange launch
        # per sweep (the rows once)
        n = 2
        sweeps = self.w.n_discard + self.w.samples_per_chain
        if self.replicas > 1:
            n += 2 * sweeps - 1
        if self.use_graph:  # the device counter is advanced by a kernel after each sweep launch
            n += sweeps if self.replicas > 1 else 1
        n += 1                                                  # ln psi / theta
        n += 2                                                  # move tables, local energy
        n += self.sr_launches()                                 # SR step
        return n


class VmcSrSymm(VmcSr):
    """The same iteration for a symmetric RBM (RbmSpinSymm, Sec. 2.2.2): sampling,
    amplitudes and local energies run on the untied RBM it stands for; SR runs in
    the tied parameters (nk_sr_step_symm), which also rewrites the untied RBM."""

    def __init__(self, w: W.Workload, params: W.RbmSymmParams, perm, sigma0=None,
                 prec: int = nk.NK_PREC_FP32, device="cuda", graph: bool = False,
                 autotune: bool = False):
        self.sy = nk.RbmSymm(perm, params.alpha, params.is_complex, device)
        self.sy.load(params.a, params.b, params.w)
        super().__init__(w, None, sigma0, prec, device, graph, autotune, rbm=self.sy.rbm)

    def _sr_scratch(self, device):
        return nk.sr_symm_scratch(self.sy, self.ns, device)

    def sr(self):
        nk.nk_sr_step_symm(self.sy, self.samples, self.t, self.eloc, self.blocks,
                           self.w.diag_shift, self.w.lr, self.w.n_cg, 1e-12, self.prec,
                           scratch=self.scratch, info_out=self.info_buf)

    def param_tensors(self):
        return [self.sy.a, self.sy.b, self.sy.w]

    def refresh(self):
        nk.nk_symm_expand(self.sy)

    def sr_launches(self) -> int:
        """As the untied step, plus per CG iteration the expansion of p, its planes
        and the fold of S p (tensor cores; expansion and fold on the FP32 path),
        the fold of F, and the expansion of the updated parameters."""
        if self.prec == nk.NK_PREC_BF16X2:
            return super().sr_launches() + 3 * self.w.n_cg + 1
        return super().sr_launches() + 2 * self.w.n_cg + 2
