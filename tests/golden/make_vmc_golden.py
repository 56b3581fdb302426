"""Write the oracle's VMC + SR energy traces used by the GPU end-to-end tests.

Calls only the FP64 oracle (oracle/) and the seeded input generators.  Output:
tests/golden/vmc_<name>.json with the per-iteration energies and the mean and
blocked error bar (blocks of 10) of the last 50 iterations.

    python tests/golden/make_vmc_golden.py [tfim10|heis12|c2|c4_0|c4_2|c4_3|c4_8] ...

Runs: tfim10 (the 10-site TFIM workload), heis12 (a 12-site Heisenberg ring),
c2 (the 40-site Heisenberg workload: complex RBM alpha = 2, 4096 chains x 4
samples, 50 CG iterations), c4_<k> (instance k of the 64 uneven 1D instances,
1024 chains x 4 samples, 50 CG iterations).
"""
import json
import os
import sys

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

from oracle import hamiltonian, vmc  # noqa: E402
from paper_1904_00031_gb300 import workloads as W  # noqa: E402

RUNS = {
    # 1D TFIM N=10, h=1, real RBM alpha=1, 16 chains x 63 samples, SR dense solve,
    # diag shift 0.01, lr 0.01 (the 10-site TFIM workload); 300 iterations
    "tfim10": dict(workload="c1", n_iter=300, lr=0.01),
    # 1D Heisenberg N=12 (Marshall-rotated), complex RBM alpha=2, exchange moves,
    # 256 chains x 4 samples, CG 50 iterations; 150 iterations
    "heis12": dict(workload=None, n_iter=150, lr=0.02),
    # 1D Heisenberg N=40 (Marshall-rotated, S^z = 0), complex RBM alpha=2 (M=80),
    # exchange moves, 4096 chains x 4 samples, CG 50 iterations; 150 iterations
    "c2": dict(workload="c2", n_iter=150, lr=0.01),
    # instances of the 64 uneven 1D problems (seed 4242): TFIM n=82 alpha=4,
    # Heisenberg n=32 alpha=4, TFIM n=18 alpha=1, Heisenberg n=64 alpha=2; 100 iterations
    "c4_0": dict(workload="c4", instance=0, n_iter=100, lr=0.01),
    "c4_2": dict(workload="c4", instance=2, n_iter=100, lr=0.01),
    "c4_3": dict(workload="c4", instance=3, n_iter=100, lr=0.01),
    "c4_8": dict(workload="c4", instance=8, n_iter=100, lr=0.01),
}


def blocked(e, block=10):
    e = np.asarray(e[-50:])
    means = e.reshape(-1, block).mean(axis=1)
    return float(e.mean()), float(means.std(ddof=1) / np.sqrt(len(means)))


def run(name):
    spec = RUNS[name]
    if spec["workload"] == "c1":
        w = W.workload("c1")
        e_exact = hamiltonian.tfim_chain_ground(w.n, 1.0, 1.0)
        n_cg = None
    elif spec["workload"] in ("c2", "c4"):
        w = (W.workload("c2") if spec["workload"] == "c2"
             else W.batched_instances(64, 4242, 1024)[spec["instance"]])
        # exact ground energy where a closed form exists (TFIM chains of even length)
        e_exact = (hamiltonian.tfim_chain_ground(w.n, 1.0, 1.0)
                   if w.move == "flip" and w.n % 2 == 0 else None)
        n_cg = w.n_cg
    else:
        n = 12
        w = W.Workload("heisenberg1d_n12_alpha2", n, 2 * n, True,
                       W.heisenberg(n, W.chain_bonds(n), 1.0, True, W.sublattice(n)), "exchange",
                       W.chain_bonds(n), True, 256, 4, 1, 0.01, spec["lr"], 50, 77)
        e_exact = hamiltonian.exact_ground(w.op, True)[0]
        n_cg = 50
    p = W.init_params(w.n, w.m, w.is_complex, 0.01, w.seed)
    ch = vmc.ChainState(W.init_chains(w.n_chains, w.n, w.zero_magnetisation, w.seed), 0)
    energies = []
    for it in range(spec["n_iter"]):
        p, ch, info = vmc.vmc_sr_iteration(
            p, w.op, ch, move=w.move, bonds=w.sampler_bonds, group_size=w.group_size, seed=w.seed,
            n_discard=w.n_discard, samples_per_chain=w.samples_per_chain,
            diag_shift=w.diag_shift, lr=spec["lr"], n_cg=n_cg)
        energies.append(info["energy"])
        if it % 25 == 0:
            print(name, it, info["energy"], flush=True)
    mean, err = blocked(energies)
    out = {"name": name, "workload": w.name, "e_exact": e_exact, "energies": energies,
           "last50_mean": mean, "last50_err": err, "lr": spec["lr"],
           "n_chains": w.n_chains, "samples_per_chain": w.samples_per_chain}
    path = os.path.join(os.path.dirname(os.path.abspath(__file__)), f"vmc_{name}.json")
    with open(path, "w") as f:
        json.dump(out, f)
    print(name, "mean", mean, "+-", err, "exact", e_exact)


if __name__ == "__main__":
    for nm in (sys.argv[1:] or list(RUNS)):
        run(nm)
