"""The multi-GPU path is independent replicas (chains are independent; no
data-path collective): per-rank chain seeds, barriers, the maximum of the ranks'
times and the whole-job rate.  Checked here with two CPU processes over gloo."""
import os
import socket

import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

from paper_1904_00031_gb300 import replicas as R
from paper_1904_00031_gb300 import workloads as W


def _free_port() -> int:
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), WORLD_SIZE=str(world),
                      RANK=str(rank), LOCAL_RANK=str(rank))
    wsize, r, local = R.env_world()
    assert (wsize, r, local) == (world, rank, rank)
    R.init(wsize, "gloo")
    w = W.workload("c2", n_chains=8, samples_per_chain=2)
    seed = R.replica_seed(w.seed, r)
    chains = W.init_chains(w.n_chains, w.n, w.zero_magnetisation, seed)
    R.barrier(wsize)
    local_ms = 10.0 * (1 + r)                      # rank r "took" 10 (r + 1) ms
    slowest = R.max_over_ranks(local_ms, wsize)
    rate = R.aggregate_rate(w.n_samples, wsize, slowest / 1e3)
    gathered = [None] * wsize
    dist.all_gather_object(gathered, (seed, chains.tobytes()))
    out[r] = (slowest, rate, gathered, w.n_samples)
    dist.destroy_process_group()


def test_two_gloo_ranks_replica_bookkeeping():
    world = 2
    mgr = mp.get_context("spawn").Manager()
    out = mgr.dict()
    mp.start_processes(_rank_main, args=(world, _free_port(), out), nprocs=world,
                       start_method="spawn", join=True)
    res = [out[r] for r in range(world)]
    for slowest, rate, gathered, ns in res:
        assert slowest == 20.0                     # the maximum over both ranks, on each rank
        assert rate == pytest.approx(world * ns / 0.020)
        (s0, c0), (s1, c1) = gathered
        assert s0 != s1 and c0 != c1               # each rank samples its own chains
    assert res[0][2] == res[1][2]                  # both ranks saw the same gathered state


def test_single_process_defaults():
    assert R.replica_seed(1237, 0) == 1237
    assert R.max_over_ranks(3.5, 1) == 3.5
    assert R.aggregate_rate(100, 1, 0.5) == 200
