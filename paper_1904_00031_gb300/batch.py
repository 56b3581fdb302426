"""Many independent, unevenly sized VMC + SR problems advanced together.

Every instance samples, evaluates ln psi and its local energies on a stream of
its own (the streams fork from and join the caller's stream); the SR steps of
all instances then run as one batch (nk_sr_step_batch: one launch of each
kernel per group of up to 64 instances, instead of one per instance), on the tensor-core path when every instance shares the SR settings.
The whole multi-instance iteration is captured once into a single CUDA graph,
so each later iteration is one graph launch.
"""
from __future__ import annotations

import torch

from . import nk
from . import workloads as W
from .vmc import VmcSr, adj_centres, centring_fused


class BatchedVmc:
    def __init__(self, instances, prec: int = nk.NK_PREC_FP32, device="cuda",
                 graph: bool = True, param_scale: float = 0.01, batch_sr: bool = True,
                 sr_splits: int = 0):
        self.items = []
        for w in instances:
            p = W.init_params(w.n, w.m, w.is_complex, param_scale, w.seed)
            v = VmcSr(w, p, prec=prec, device=device, graph=graph)
            v.rbm._s.sr_splits = int(sr_splits)  # 0: built-in (per call, or batch-wide) default
            self.items.append(v)
        self.streams = [torch.cuda.Stream(device=device) for _ in instances]
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

    def _eager_step(self):
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

    def step(self):
        """One iteration of every instance.  In graph mode the first call runs
        eagerly and captures the graph; later calls replay it."""
        if self.use_graph:
            if self.graph is None:
                self._eager_step()
                self.capture()
            else:
                self.graph.replay()
        else:
            self._eager_step()

    def infos(self):
        return [v.info() for v in self.items]

    def launches_per_step(self) -> int:
        if self.srb is None:
            return sum(v.launches_per_step() for v in self.items)
        n = sum(v.launches_per_step() - v.sr_launches() for v in self.items)
        groups = (len(self.items) + 63) // 64   # up to 64 instances per launch
        # per group: statistics (3), flags, sigma' planes (2), force, CG start (2),
        # 7 per CG iteration (6 when every forward writes its centring partials, 5
        # when every adjoint also centres its input)
        # plus the first iteration's planes, update, prepare (2)
        fused = all(centring_fused(v.ns, v.w.m, v.w.is_complex) for v in self.items)
        adj = fused and all(adj_centres(v.w.m, v.w.is_complex) for v in self.items)
        per = 5 if adj else (6 if fused else 7)
        return n + groups * (3 + 1 + 2 + 2 + 2 + per * self.sr_args[2] + 1 + 3)
