"""Many independent, unevenly sized VMC + SR problems advanced together.

By default (fused) the instances' sweeps run as one launch per Metropolis
kernel template, each template's call on a stream of its own (forked from and
joined back into the caller's stream, so that the templates overlap), then
ln psi / theta and the local energies as one launch per field; otherwise every
instance samples, evaluates ln psi and its local energies on a stream of its
own.  The SR steps of all instances then run as one batch (nk_sr_step_batch:
one launch of each kernel per group of up to 64 instances, instead of one per
instance), on the tensor-core path when every instance shares the SR settings.
The whole multi-instance iteration is captured once into a single CUDA graph,
so each later iteration is one graph launch.
"""
from __future__ import annotations

import torch

from . import nk
from . import workloads as W
from .vmc import VmcSr, adj_centres, centring_fused


def _metro_template(w) -> tuple:
    """The Metropolis kernel template an instance runs: the library's built-in
    rule, for counting the fused launches.  One CTA per proposal group (complex
    RBMs, group size <= 8, m <= 256 or > 2048): (unit pairs per thread, block
    size); else warps per chain: (field, hidden units per lane, warps per chain,
    group size)."""
    if w.is_complex and w.group_size <= 8 and (w.m <= 256 or w.m > 2048):
        pp = 1 if w.m <= 256 else 3
        pairs = (w.m + 1) // 2
        return ("group", pp, (pairs + pp - 1) // pp + (-((pairs + pp - 1) // pp)) % 32)
    mp = (w.m + 31) // 32 * 32
    wpc = 2 if (mp >= 512 and w.group_size * 64 <= 512) else 1
    e = (mp + 32 * wpc - 1) // (32 * wpc)
    lists = {(True, 1): [2, 4, 8, 16, 32, 64], (True, 2): [8, 14, 16, 26, 32],
             (False, 1): [1, 2, 4, 8, 16, 32, 64], (False, 2): [8, 13, 16, 25, 32]}
    nu = next(x for x in lists[(w.is_complex, wpc)] if x >= e)
    return (w.is_complex, nu, wpc, w.group_size)


class BatchedVmc:
    def __init__(self, instances, prec: int = nk.NK_PREC_FP32, device="cuda",
                 graph: bool = True, param_scale: float = 0.01, batch_sr: bool = True,
                 sr_splits: int = 0, fused: bool = True, autotune: bool = False):
        """``fused``: sampling, theta and local energies of all instances run as
        fused launches (nk_batch_sweep / nk_batch_logpsi / nk_batch_local_energy
        on one stream); else every instance launches its own kernels on a stream
        of its own."""
        self.fused = fused
        self.prec = prec
        self.autotune = autotune
        self.items = []
        for w in instances:
            p = W.init_params(w.n, w.m, w.is_complex, param_scale, w.seed)
            v = VmcSr(w, p, prec=prec, device=device, graph=graph)
            v.rbm._s.sr_splits = int(sr_splits)  # 0: built-in (per call, or batch-wide) default
            self.items.append(v)
        self.streams = [torch.cuda.Stream(device=device) for _ in instances]
        self.sweep_jobs = [dict(rbm=v.rbm, chains=v.chains, move=v.move, bond_i=v.bond_i,
                                bond_k=v.bond_k, n_discard=v.w.n_discard,
                                n_samples_per_chain=v.w.samples_per_chain, samples_out=v.samples,
                                n_accept_out=v.n_acc, scratch=v.metro_scratch)
                           for v in self.items]
        # one fused sweep call per kernel template, each on a stream of its own, so
        # that the templates' launches (each covering only its own instances)
        # overlap on the GPU instead of running one after another
        groups = {}
        for v, job in zip(self.items, self.sweep_jobs):
            groups.setdefault(_metro_template(v.w), []).append(job)
        self.sweep_groups = list(groups.values())
        self.group_streams = [torch.cuda.Stream(device=device) for _ in self.sweep_groups]
        self.theta_jobs = [dict(rbm=v.rbm, sigma=v.samples, logpsi_out=None, theta_out=v.theta)
                           for v in self.items]
        self.eloc_jobs = [dict(rbm=v.rbm, op=v.op, sigma=v.samples, theta=v.theta,
                               eloc_out=v.eloc, t_out=v.t, scratch=v.eloc_scratch)
                          for v in self.items]
        self.use_graph = graph
        self.graph = None
        ws = list(instances)
        same = all((w.diag_shift, w.lr, w.n_cg) == (ws[0].diag_shift, ws[0].lr, ws[0].n_cg)
                   for w in ws)
        self.srb = None
        if batch_sr and same and prec == nk.NK_PREC_BF16X2:
            self.sr_args = (ws[0].diag_shift, ws[0].lr, ws[0].n_cg)
            self.srb = nk.SrBatch([
                {"rbm": v.rbm, "sigma": v.samples, "t": v.t, "eloc": v.eloc,
                 "scratch": v.scratch, "info": v.info_buf, "n_chains": v.blocks}
                for v in self.items], prec=prec, device=device)

    @property
    def n_samples(self) -> int:
        return sum(v.ns for v in self.items)

    def _fork(self, fn, groups):
        """fn(jobs, stream) for every group of jobs, each group on a stream of its
        own forked from (and joined back into) the current stream."""
        if len(groups) == 1:
            fn(groups[0], None)
            return
        cur = torch.cuda.current_stream()
        for jobs, st in zip(groups, self.group_streams):
            st.wait_stream(cur)
            fn(jobs, st)
        for st in self.group_streams[:len(groups)]:
            cur.wait_stream(st)

    def _eager_step(self):
        if self.fused:
            self._fork(lambda j, st: nk.nk_batch_sweep(j, stream=st), self.sweep_groups)
            nk.nk_batch_logpsi(self.theta_jobs, prec=self.prec)
            nk.nk_batch_local_energy(self.eloc_jobs)
            if self.srb is not None:
                d, lr, n_cg = self.sr_args
                self.srb.step(d, lr, n_cg)
            else:
                for v in self.items:
                    v.sr()
            return
        cur = torch.cuda.current_stream()
        for v, st in zip(self.items, self.streams):
            st.wait_stream(cur)
            with torch.cuda.stream(st):
                v.sample()
                v.amplitudes()
                v.energies()
                if self.srb is None:
                    v.sr()
        for st in self.streams:
            cur.wait_stream(st)
        if self.srb is not None:
            d, lr, n_cg = self.sr_args
            self.srb.step(d, lr, n_cg)

    def capture(self):
        torch.cuda.synchronize()
        self.graph = torch.cuda.CUDAGraph()
        with torch.cuda.graph(self.graph):
            self._eager_step()

    def tune_shapes(self):
        """Autotune every instance's theta and local-energy tile shapes on its
        current samples (tensor-core path; synchronises), then recompute theta and
        the local energies the tuner overwrote."""
        if self.prec != nk.NK_PREC_BF16X2:
            return
        for v in self.items:
            nk.nk_tune_shapes(v.rbm, v.op, v.samples, v.theta, v.eloc, v.eloc_scratch, v.t)
            v.amplitudes()
            v.energies()

    def step(self):
        """One iteration of every instance.  In graph mode the first call runs
        eagerly (and autotunes, if asked) and captures the graph; later calls
        replay it."""
        if self.use_graph:
            if self.graph is None:
                self._eager_step()
                if self.autotune:
                    self.tune_shapes()
                self.capture()
            else:
                self.graph.replay()
        else:
            self._eager_step()

    def infos(self):
        return [v.info() for v in self.items]

    def launches_per_step(self) -> int:
        if self.fused:
            fields = len({v.w.is_complex for v in self.items})
            # sampling, per kernel template (one call each, on its own stream): the
            # move rows, the sweep launch, the device counters (graph mode); up to
            # 64 items per launch
            n = len(self.sweep_groups) * (2 + (1 if self.use_graph else 0))
            n += fields            # theta
            n += 1 + fields        # move tables, local energies
        elif self.srb is None:
            return sum(v.launches_per_step() for v in self.items)
        else:
            n = sum(v.launches_per_step() - v.sr_launches() for v in self.items)
        if self.srb is None:
            return n + sum(v.sr_launches() for v in self.items)
        groups = (len(self.items) + 63) // 64   # up to 64 instances per launch
        # per group: statistics (3), flags, sigma' planes (2), force, CG start (2),
        # 7 per CG iteration (6 when every forward writes its centring partials, 5
        # when every adjoint also centres its input)
        # plus the first iteration's planes, update, prepare (2)
        fused = all(centring_fused(v.ns, v.w.m, v.w.is_complex) for v in self.items)
        adj = fused and all(adj_centres(v.w.m, v.w.is_complex) for v in self.items)
        per = 5 if adj else (6 if fused else 7)
        return n + groups * (3 + 1 + 2 + 2 + 2 + per * self.sr_args[2] + 1 + 3)
