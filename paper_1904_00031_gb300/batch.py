"""Many independent, unevenly sized VMC + SR problems advanced together.

Every instance runs the ordinary iteration (``vmc.VmcSr``: sweep -> ln psi ->
local energies -> SR step) on a stream of its own; the streams fork from and
join the caller's stream, and the whole multi-instance iteration is captured
once into a single CUDA graph, so each later iteration is one graph launch in
which the instances' kernels run concurrently and fill the GPU.
"""
from __future__ import annotations

import torch

from . import nk
from . import workloads as W
from .vmc import VmcSr


class BatchedVmc:
    def __init__(self, instances, prec: int = nk.NK_PREC_FP32, device="cuda",
                 graph: bool = True, param_scale: float = 0.01):
        self.items = []
        for w in instances:
            p = W.init_params(w.n, w.m, w.is_complex, param_scale, w.seed)
            self.items.append(VmcSr(w, p, prec=prec, device=device, graph=graph))
        self.streams = [torch.cuda.Stream(device=device) for _ in instances]
        self.use_graph = graph
        self.graph = None

    @property
    def n_samples(self) -> int:
        return sum(v.ns for v in self.items)

    def _eager_step(self):
        cur = torch.cuda.current_stream()
        for v, st in zip(self.items, self.streams):
            st.wait_stream(cur)
            with torch.cuda.stream(st):
                v._eager_step()
        for st in self.streams:
            cur.wait_stream(st)

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
        return sum(v.launches_per_step() for v in self.items)
