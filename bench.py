"""Throughput of one RBM-VMC + SR iteration on the 20x20 J1-J2 workload
(N = 400 sites, complex RBM alpha = 4: M = 1600, 642,000 complex parameters,
16384 chains x 4 samples = 65,536 samples per iteration, exchange moves,
SR by lazy CG with 50 iterations), on synthetic seeded inputs.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
                  [--prec fp32|bf16x2] [--workload c5|c3|c2|c1]

One JSON line on rank 0.  `value` = samples per second of whole iterations
(Metropolis sweeps incl. burn-in, ln psi, local energies, SR step), device
timed with CUDA events, max over ranks; several GPUs run independent replicas
(weak scaling).  `--impl reference` times the FP64 CPU oracle on a bounded
sample of the same workload instead.
"""
from __future__ import annotations

import argparse
import json
import os
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "RBM-VMC samples/s and SR steps/s at N=400 vs plain FP32 GPU path; % roofline"


T_START = time.perf_counter()


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--prec", default="auto", choices=["auto", "fp32", "bf16x2"])
    ap.add_argument("--workload", default="c5", choices=["c1", "c2", "c3", "c4", "c5"])
    ap.add_argument("--model", default="rbm", choices=["rbm", "symm", "supervised", "ffnn"],
                    help="symm: the translation-symmetric RBM (alpha = m / n families) on the "
                         "workload's lattice, SR in its tied parameters; supervised: overlap "
                         "learning steps (c1: the paper's example shape, c5); ffnn: a two-layer "
                         "ln cosh network's ln psi and gradient (c2, c5)")
    ap.add_argument("--graph", type=int, default=1, help="replay iterations as CUDA graphs")
    ap.add_argument("--profile-kernels", action="store_true",
                    help="small 20x20 J1-J2 case for ncu captures: one CTA per SM per kernel")
    ap.add_argument("--oracle-sample", default=None, help=argparse.SUPPRESS)
    ap.add_argument("--no-baseline", action="store_true", help="skip the CPU oracle baseline")
    ap.add_argument("--no-fp32-arm", action="store_true", help="skip the plain FP32 comparison")
    ap.add_argument("--phase-times", action="store_true",
                    help="print the wall time of each bench phase to stderr")
    ap.add_argument("--replicas", type=int, default=1,
                    help="sample by parallel tempering with this many replicas per chain")
    ap.add_argument("--checkpoint-iters", type=int, default=50,
                    help="also time the iteration after this many more SR iterations "
                         "(structured psi, realistic acceptance); 0 skips it")
    return ap.parse_args()


# ---------------------------------------------------------------------- CPU oracle sample

def oracle_setup(workload: str, n_chains: int, offset: int = 0):
    """Inputs of a bounded oracle sample: the workload, its initial parameters
    and n_chains chain states from chain ``offset`` on."""
    from paper_1904_00031_gb300 import workloads as W
    w = W.workload(workload) if workload != "c4" else W.batched_instances(64, 4242, 1024)[0]
    p = W.init_params(w.n, w.m, w.is_complex, 0.01, w.seed)
    s0 = W.init_chains(max(w.n_chains, offset + n_chains), w.n, w.zero_magnetisation,
                       w.seed)[offset:offset + n_chains]
    return w, p, s0


def oracle_iteration(w, p, s0, spc: int, n_cg: int) -> dict:
    """One oracle VMC + SR iteration on the given chains (spc samples per chain,
    1 burn-in sweep); returns seconds and samples."""
    from oracle import local_energy, rbm, sampler, sr
    n_chains = len(s0)
    t0 = time.perf_counter()
    samples, fin, cnt, nacc = sampler.metropolis(p, s0, w.move, w.sampler_bonds, w.group_size,
                                                 w.seed, 0, 1, spc)
    e = local_energy.local_energy_rbm(p, w.op, samples)
    blocks = n_chains // w.group_size if n_chains % w.group_size == 0 else 1
    mean, var, err = sr.stats(e, blocks)
    sig, t = rbm.logderiv_factored(p, samples)
    real = not p.is_complex
    f = sr.force_lazy(sig, t, e, p.n, p.m, None, real)
    delta, it, res = sr.cg(lambda x: sr.sr_matvec_lazy(sig, t, x, p.n, p.m, None, real), f,
                           w.diag_shift, n_cg, 1e-12)
    sr.sgd_update(p.flat(), delta, w.lr)
    dt = time.perf_counter() - t0
    return {"seconds": dt, "samples": int(len(samples)), "energy": float(mean.real)}


def oracle_sample(workload: str, n_chains: int, spc: int, n_cg: int, offset: int = 0) -> dict:
    """One oracle VMC + SR iteration on a bounded sample (n_chains chains from
    chain ``offset`` on, spc samples per chain, 1 burn-in sweep)."""
    w, p, s0 = oracle_setup(workload, n_chains, offset)
    return oracle_iteration(w, p, s0, spc, n_cg)


def _oracle_env():
    env = dict(os.environ)
    for k in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS"):
        env[k] = "1"
    return env


def run_oracle_subprocess(workload: str, n_chains: int, spc: int, n_cg: int) -> dict:
    spec = json.dumps({"workload": workload, "n_chains": n_chains, "spc": spc, "n_cg": n_cg})
    r = subprocess.run([sys.executable, os.path.abspath(__file__), "--oracle-sample", spec],
                       capture_output=True, text=True, env=_oracle_env(), cwd=ROOT)
    if r.returncode != 0:
        raise RuntimeError("oracle sample failed: " + r.stderr[-2000:])
    return json.loads(r.stdout.strip().splitlines()[-1])


def _oracle_worker(workload, n_chains, spc, n_cg, offset, n_iter, barrier, out):
    for k in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS"):
        os.environ[k] = "1"
    sys.path.insert(0, ROOT)
    w, p, s0 = oracle_setup(workload, n_chains, offset)
    for _ in range(n_iter):
        barrier.wait()
        r = oracle_iteration(w, p, s0, spc, n_cg)
        barrier.wait()
    out.put(r["samples"])


def run_oracle_all_cores(workload: str, n_chains: int, spc: int, n_cg: int,
                         n_iter: int = 1) -> dict:
    """The oracle on every host core at once: one single-threaded worker process
    per core (started with spawn, before any CUDA call), each on its own
    n_chains chains; every iteration starts and ends on a barrier of all
    workers, and its rate is all samples / the wall time between the two."""
    import multiprocessing as mp
    cores = os.cpu_count() or 1
    ctx = mp.get_context("spawn")
    barrier = ctx.Barrier(cores + 1)
    out = ctx.Queue()
    procs = [ctx.Process(target=_oracle_worker, args=(workload, n_chains, spc, n_cg,
                                                      k * n_chains, n_iter, barrier, out))
             for k in range(cores)]
    for pr in procs:
        pr.start()
    secs = []
    for _ in range(n_iter):
        barrier.wait()
        t0 = time.perf_counter()
        barrier.wait()
        secs.append(time.perf_counter() - t0)
    per = sum(out.get() for _ in procs)
    for pr in procs:
        pr.join()
    return {"seconds": secs, "samples": per, "cores": cores}


# DRAM bytes (read + write) per launch of a stage's dominant kernel, from one
# single-pass ncu capture (dram__bytes_read.sum + dram__bytes_write.sum) of the
# workload at full size; a kernel that changed since its capture has no entry.
NCU_TRAFFIC = {
    ("j1j2_20x20_alpha4", "bf16x2", "local_energy_tiled"): 9.327e9 + 0.864e9,
}

ORACLE_SAMPLE = {"c5": (24, 2, 50), "c3": (64, 1, 50), "c2": (128, 4, 50), "c1": (16, 63, 120),
                 "c4": (64, 4, 50)}
# per process of the all-core oracle runs (one single-threaded process per core)
ORACLE_SAMPLE_CORE = {"c5": (8, 2, 50), "c3": (24, 1, 50), "c2": (48, 4, 50), "c1": (16, 63, 120),
                      "c4": (24, 4, 50)}


# ---------------------------------------------------------------------- clocks

class ClockSampler:
    def __init__(self, index: int):
        self.f = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)
        q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
        try:
            self.p = subprocess.Popen(["nvidia-smi", f"--id={index}", f"--query-gpu={q}",
                                       "--format=csv,noheader,nounits", "-lms", "200"],
                                      stdout=self.f, stderr=subprocess.DEVNULL)
        except OSError:
            self.p = None

    def stop(self) -> dict:
        if self.p is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.p.terminate()
        self.p.wait()
        self.f.flush()
        self.f.seek(0)
        rows = [ln.strip().split(", ") for ln in self.f.read().splitlines() if ln.strip()]
        os.unlink(self.f.name)
        sm, mx, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for r in rows:
            try:
                sm.append(float(r[1]))
                mx = float(r[2])
                for nm, v in zip(names, r[5:9]):
                    if v.strip().lower() == "active":
                        reasons.add(nm)
            except (ValueError, IndexError):
                continue
        sm.sort()
        return {"sm_mhz": sm[len(sm) // 2] if sm else None, "sm_max_mhz": mx,
                "reasons": sorted(reasons), "samples": len(sm)}


# ---------------------------------------------------------------------- GPU arm

def peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            d = json.load(f)
        return d, "measured"
    except OSError:
        return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "sm_max_mhz": 2070.0}, "fallback"


def fp32_peak_tflops(sm_mhz: float) -> float:
    # 152 SMs x 128 FP32 lanes x 2 flop per FMA x clock
    return 152 * 128 * 2 * sm_mhz * 1e6 / 1e12


# Algorithmic FLOPs per stage (counted from the formulas, not from the kernels'
# instruction streams; FMA = 2 flop; complex multiply = 6, complex add = 2):
#  sampling, per hidden unit: a non-null proposal evaluates r = C - s t D and
#    accumulates |r|^2 (complex 12, real 4); an accepted one also updates
#    t' = (t C - s D) / r and theta (complex 32, real 8).
#  local energy, per (configuration, move, hidden unit): r = C - s t D and the
#    running product (complex 14, real 4).
#  ln psi: theta = W sigma' (complex W: 4 n m per configuration).
#  SR: per CG iteration the forward and adjoint contractions, 4 n m each per
#    sample (complex), 2 n m (real); plus the force (one adjoint).
def connected_per_config(op, sm) -> float:
    """Mean number of connected configurations sigma' != sigma (nonzero
    <sigma'|H|sigma>) of the configurations sm (int8 [S][n]): the local-energy
    terms the method evaluates.  Terms producing the same sigma' count once."""
    import numpy as np
    idx = (sm < 0).astype(np.int64)
    active = {}

    def add(key, mask):
        active[key] = active[key] | mask if key in active else mask.copy()

    for t in range(op.n_site_terms):
        i, M = int(op.site_idx[t]), op.site_mat[t]
        add((i,), np.array([M[1, 0] != 0, M[0, 1] != 0])[idx[:, i]])
    for t in range(op.n_bond_terms):
        i, k, M = int(op.bond_i[t]), int(op.bond_k[t]), op.bond_mat[t]
        x = 2 * idx[:, i] + idx[:, k]
        for flip, key in ((2, (i,)), (1, (k,)), (3, (min(i, k), max(i, k)))):
            add(key, np.array([M[xx ^ flip, xx] != 0 for xx in range(4)])[x])
    return float(sum(v.mean() for v in active.values()))


def stage_flops(w, n_nonnull: float, n_accept: float, n_connected: float) -> dict:
    """Algorithmic FLOPs per stage; n_connected = mean connected configurations
    per sample (the local-energy terms)."""
    c = w.is_complex
    m, n, ns = w.m, w.n, w.n_samples
    return {
        "sample": m * ((12 if c else 4) * n_nonnull + (32 if c else 8) * n_accept),
        "energies": float(ns) * n_connected * m * (14 if c else 4),
        "amplitudes": float(ns) * (4 if c else 2) * n * m,
        "sr": float(ns) * (4 if c else 2) * n * m * (2 * w.n_cg + 1),
    }


def run_gpu(args):
    import numpy as np
    import torch

    from paper_1904_00031_gb300 import nk
    from paper_1904_00031_gb300 import workloads as W
    from paper_1904_00031_gb300 import replicas as R
    from paper_1904_00031_gb300.vmc import VmcSr, VmcSrSymm

    world, rank, local = R.env_world()
    R.init(world, "nccl")
    torch.cuda.set_device(local)
    nk.load_library()
    w = W.workload(args.workload)
    params = W.init_params(w.n, w.m, w.is_complex, 0.01, w.seed)
    prec_name = args.prec if args.prec != "auto" else "bf16x2"
    prec = nk.NK_PREC_FP32 if prec_name == "fp32" else nk.NK_PREC_BF16X2
    # each rank samples its own chains (independent replicas)
    sigma0 = W.init_chains(w.n_chains, w.n, w.zero_magnetisation, R.replica_seed(w.seed, rank))
    symm = args.model == "symm"
    if symm:
        perm = W.translations(w)
        sparams = W.init_symm_params(w.n, w.m // w.n, w.is_complex, 0.01, w.seed)

        def make(pr, **kw):
            return VmcSrSymm(w, sparams, perm, sigma0, pr, **kw)
    else:
        if args.replicas > 1:
            sigma0 = W.init_chains(w.n_chains * args.replicas, w.n, w.zero_magnetisation,
                                   R.replica_seed(w.seed, rank))

        def make(pr, **kw):
            return VmcSr(w, params, sigma0, pr, replicas=args.replicas, **kw)

    t_phase = [T_START]

    def phase(name):
        if args.phase_times:
            torch.cuda.synchronize()
            now = time.perf_counter()
            print(f"[bench] {name}: {now - t_phase[0]:.2f} s", file=sys.stderr, flush=True)
            t_phase[0] = now

    phase("setup (imports, CUDA context, workload)")
    v = make(prec, graph=bool(args.graph), autotune=True)
    phase("driver construction")
    wname = w.name + ("_symm" if symm else "")
    stream = torch.cuda.current_stream()

    def barrier():
        R.barrier(world)
        torch.cuda.synchronize()

    for _ in range(args.warmup):
        v.step()
    barrier()
    phase("warm-up (first step autotunes and captures)")
    # timed region: K whole iterations (CUDA-graph replays unless --graph 0)
    clocks = ClockSampler(local)
    barrier()
    small = w.n_samples * w.m * (8 if w.is_complex else 4) <= 129e6
    flush = torch.empty(256 << 20, dtype=torch.uint8, device="cuda") if small else None
    ev_it = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
             for _ in range(args.steps)]
    for k in range(args.steps):
        if flush is not None:
            flush.zero_()  # evict the working set from the 129 MB L2 (outside the timing)
        ev_it[k][0].record(stream)
        v.step()
        ev_it[k][1].record(stream)
    barrier()
    clk = clocks.stop()
    total_ms = sum(a.elapsed_time(b) for a, b in ev_it)
    phase("timed steps and clock sampling")
    # per-stage breakdown (eager launches, CUDA events between the stages)
    stages = ["sample", "amplitudes", "energies", "sr"]
    ev = [[torch.cuda.Event(enable_timing=True) for _ in range(5)] for _ in range(args.steps)]
    for k in range(args.steps):
        ev[k][0].record(stream)
        for si, name in enumerate(stages):
            getattr(v, name)()
            ev[k][si + 1].record(stream)
    barrier()
    stage_ms = {name: float(np.mean([ev[k][si].elapsed_time(ev[k][si + 1])
                                     for k in range(args.steps)]))
                for si, name in enumerate(stages)}
    info = v.info()
    total_ms = R.max_over_ranks(total_ms, world, "cuda")
    ms_per_step = total_ms / args.steps
    value = R.aggregate_rate(w.n_samples, world, ms_per_step / 1e3)

    phase("stage breakdown")
    # end to end through the public API: parameters H2D from pinned memory,
    # one iteration, the FP64 status block D2H, every step
    dev_params = v.param_tensors()
    host_params = [x.cpu().pin_memory() for x in dev_params]
    host_info = torch.empty(nk.NK_INFO_LEN, dtype=torch.float64).pin_memory()
    barrier()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(args.steps):
        for d, h in zip(dev_params, host_params):
            d.copy_(h, non_blocking=True)
        v.refresh()
        v.step()
        host_info.copy_(v.info_buf, non_blocking=True)
    e1.record(stream)
    barrier()
    e2e_ms = R.max_over_ranks(e0.elapsed_time(e1) / args.steps, world, "cuda")
    h2d = sum(h.numel() for h in host_params) * 8

    phase("end to end")
    # the plain FP32 path on the same workload (the mixed-precision ratio) and the
    # same-accuracy evidence: both paths from the same parameters, chains and
    # random streams for warm-up + timed iterations (eager, the energy read after
    # every iteration outside the CUDA-event bracket), energy by energy
    fp32_arm, same_acc, v32 = None, None, None
    if prec != nk.NK_PREC_FP32 and not args.no_fp32_arm:
        n_it = args.warmup + args.steps

        def trace(pr):
            vv = make(pr)
            es, errs, ms = [], [], []
            for _ in range(n_it):
                a0 = torch.cuda.Event(enable_timing=True)
                a1 = torch.cuda.Event(enable_timing=True)
                a0.record(stream)
                vv.step()
                a1.record(stream)
                inf = vv.info()  # synchronises
                es.append(inf["energy"])
                errs.append(inf["error"])
                ms.append(a0.elapsed_time(a1))
            return vv, np.array(es), np.array(errs), np.array(ms)

        v32, e32, s32, ms32 = trace(nk.NK_PREC_FP32)
        _, ebf, sbf, _ = trace(prec)
        barrier()
        fp32_ms = R.max_over_ranks(float(np.mean(ms32[args.warmup:])), world, "cuda")
        fp32_arm = R.aggregate_rate(w.n_samples, world, fp32_ms / 1e3)
        d = np.abs(ebf - e32) / np.sqrt(sbf ** 2 + s32 ** 2)
        half = n_it // 2
        same_acc = {
            "iterations": n_it,
            "energy_bf16x2": [round(float(x), 6) for x in ebf],
            "energy_fp32": [round(float(x), 6) for x in e32],
            "error_bar_bf16x2_last": round(float(sbf[-1]), 6),
            "error_bar_fp32_last": round(float(s32[-1]), 6),
            "mean_last_half_bf16x2": round(float(ebf[half:].mean()), 6),
            "mean_last_half_fp32": round(float(e32[half:].mean()), 6),
            "max_abs_diff_over_error_bar": round(float(d.max()), 4),
            "note": "same seeds, parameters and chains; error bars from proposal-group means "
                    "of each iteration",
        }
        # the FP32 arm's own stage breakdown and SR roofline (one eager iteration)
        e32v = [torch.cuda.Event(enable_timing=True) for _ in range(5)]
        e32v[0].record(stream)
        for si, name in enumerate(stages):
            getattr(v32, name)()
            e32v[si + 1].record(stream)
        barrier()
        stage_ms_fp32 = {name: e32v[si].elapsed_time(e32v[si + 1]) for si, name in enumerate(stages)}

    t_bytes = w.n_samples * w.m * (8 if w.is_complex else 4)
    l2_note = (f"inputs larger than L2 (T = tanh theta is {t_bytes / 1e6:.0f} MB)" if t_bytes > 129e6
               else f"inputs smaller than L2 (T is {t_bytes / 1e6:.1f} MB); L2 flushed before each "
                    "timed iteration")
    phase("FP32 arm")
    pk, pk_kind = peaks()
    sm_max = pk.get("sm_max_mhz", 2070.0)
    # proposals that needed a ratio: every flip; exchanges of two unequal spins
    # (fraction measured on the recorded samples)
    sweeps = w.n_discard + w.samples_per_chain
    n_prop = float(w.n_chains) * sweeps * w.n
    if w.move == "flip":
        nonnull_frac = 1.0
    else:
        sm = v.samples.to(torch.int16)
        bi = v.bond_i.long()
        bk = v.bond_k.long()
        nonnull_frac = float((sm[:, bi] != sm[:, bk]).float().mean().item())
    n_accept = float(v.n_acc.sum().item())
    n_conn = connected_per_config(w.op, v.samples[:4096].cpu().numpy())
    fl = stage_flops(w, n_prop * nonnull_frac, n_accept, n_conn)
    try:
        alu_meas = nk.nk_measure_alu_peaks()
        alu_peak = alu_meas["fp32_fma_flops"] / 1e12
        alu_src = "measured packed FP32 FMA rate (nk_measure_alu_peaks)"
    except Exception as e:  # noqa: BLE001 - report the derived figure instead
        alu_meas = {"error": str(e)[:200]}
        alu_peak = fp32_peak_tflops(sm_max)
        alu_src = f"152 SM x 128 FP32 lanes x 2 x {sm_max:.0f} MHz (derived)"
    tc_peak = pk.get("bf16_tflops_sustained", pk.get("bf16_tflops", 1900.0))
    rl = {}
    for st_name, ms in stage_ms.items():
        tensor = st_name in ("sr", "amplitudes") and prec_name == "bf16x2"
        peak = tc_peak if tensor else alu_peak
        ach = fl[st_name] / (ms / 1e3) / 1e12
        rl[st_name] = {"bound": "tensor" if tensor else "alu", "achieved": round(ach, 3),
                       "peak": round(peak, 1), "unit": "TFLOP/s", "frac": round(ach / peak, 4)}
    dom = max(stage_ms, key=stage_ms.get)
    kern = {"sample": "metropolis_kernel", "energies": "local_energy_tiled",
            "amplitudes": ("fwd_tc_kernel (theta only)" if prec_name == "bf16x2"
                           else "logpsi_fp32_kernel (theta only)"),
            "sr": "SR step (fwd_tc + adj_tc + CG vector kernels)" if prec_name == "bf16x2"
                  else "SR step (forward/adjoint FP32 + CG vector kernels)"}[dom]
    fp32_info = None
    if fp32_arm is not None:
        fl32 = {k: fl[k] for k in stage_ms_fp32}
        fp32_info = {"samples_per_s": round(fp32_arm, 2),
                     "stage_ms": {k: round(x, 3) for k, x in stage_ms_fp32.items()},
                     "stage_roofline": {k: {"bound": "alu", "achieved":
                                            round(fl32[k] / (x / 1e3) / 1e12, 3),
                                            "peak": round(alu_peak, 1), "unit": "TFLOP/s",
                                            "frac": round(fl32[k] / (x / 1e3) / 1e12 / alu_peak, 4)}
                                        for k, x in stage_ms_fp32.items()},
                     "note": "plain FP32 CUDA-core contractions, same algorithm; peak = the "
                             "measured FP32 FMA rate"}
    roof = dict(rl[dom])
    roof.update({"kernel": kern, "traffic": NCU_TRAFFIC.get((wname, prec_name, kern)),
                 "peak_source": (f"{pk_kind} bf16 dense TFLOP/s (sustained)" if roof["bound"] == "tensor"
                                 else alu_src)})
    # the same measurement after more SR iterations: psi has structure and the
    # acceptance is the optimisation's, not the near-uniform initial one
    phase("rooflines and ALU peaks")
    ckpt = None
    if args.checkpoint_iters > 0:
        for _ in range(args.checkpoint_iters):
            v.step()
        barrier()
        ev_ck = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
                 for _ in range(args.steps)]
        for k in range(args.steps):
            if flush is not None:
                flush.zero_()
            ev_ck[k][0].record(stream)
            v.step()
            ev_ck[k][1].record(stream)
        barrier()
        ck_ms = R.max_over_ranks(sum(a.elapsed_time(b) for a, b in ev_ck), world,
                                 "cuda") / args.steps
        info_ck = v.info()
        ckpt = {"sr_iterations_before": args.checkpoint_iters + 3 * args.steps + args.warmup,
                "value": round(R.aggregate_rate(w.n_samples, world, ck_ms / 1e3), 2),
                "unit": "samples/s",
                "ms_per_step": round(ck_ms, 3), "acceptance": round(info_ck["acceptance"], 4),
                "energy": info_ck["energy"]}
    phase("checkpoint iterations")
    out = {
        "metric": METRIC, "value": round(value, 2), "unit": "samples/s", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(ms_per_step, 3),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
        "data": "synthetic (seeded RBM parameters N(0,0.01^2), random S^z=0 chain starts)",
        "config": {"workload": wname, "n": w.n, "m": w.m, "complex": w.is_complex,
                   "chains": w.n_chains, "samples_per_chain": w.samples_per_chain,
                   "burn_in_sweeps": w.n_discard, "samples_per_iter": w.n_samples,
                   "moves": w.move, "n_cg": w.n_cg, "diag_shift": w.diag_shift, "lr": w.lr,
                   "prec": prec_name, "l2": l2_note, "replicas": args.replicas,
                   "parallelism": f"replicas x{world}"},
        "sr_steps_per_s": round(1e3 / ms_per_step, 4),
        "stage_ms": {k: round(x, 3) for k, x in stage_ms.items()},
        "fp32_path_samples_per_s": None if fp32_arm is None else round(fp32_arm, 2),
        "fp32_arm": fp32_info, "same_accuracy": same_acc,
        "cg_iters": int(info["cg_iters"]), "cg_resid": info["cg_resid"],
        "acceptance": round(info["acceptance"], 4),
        "exchange_rate": (round(info["exchange_rate"], 4) if "exchange_rate" in info else None),
        "energy": info["energy"],
        "energy_error_bar": info["error"],
        "nonnull_proposal_fraction": round(nonnull_frac, 4),
        "connected_per_sample": round(n_conn, 2), "moves": v.op.n_moves,
        "roofline": roof, "stage_roofline": rl,
        "alu_peaks_measured": ({"fp32_fma_tflops": round(alu_meas["fp32_fma_flops"] / 1e12, 2),
                                "mufu_ex2_tops": round(alu_meas["mufu_ex2_ops"] / 1e12, 3),
                                "mufu_lg2_tops": round(alu_meas["mufu_lg2_ops"] / 1e12, 3),
                                "mufu_sin_tops": round(alu_meas["mufu_sin_ops"] / 1e12, 3)}
                               if "fp32_fma_flops" in alu_meas else alu_meas),
        "after_sr_iterations": ckpt,
        "e2e": {"value": round(R.aggregate_rate(w.n_samples, world, e2e_ms / 1e3), 2),
                "unit": "samples/s",
                "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": nk.NK_INFO_LEN * 8},
        "gpu_launches": v.launches_per_step() * args.steps,
        "graph": bool(args.graph), "sr_split_k": getattr(v, "split_k", None),
        "tile_shapes": (None if not hasattr(v, "shapes") else
                        {"theta_ctas_per_tile": v.shapes[0], "eloc_ctas_per_tile": v.shapes[1]}),
        "clocks": clk,
    }
    return rank, out


def profile_kernels():
    """Small case of the 20x20 J1-J2 shapes for profiler captures: Metropolis on
    1216 chains (one CTA per SM) for 16 sweeps, ln psi and local energies on their
    19,456 samples, one SR step with 2 CG iterations; every stage runs twice."""
    import torch

    from paper_1904_00031_gb300 import nk
    from paper_1904_00031_gb300 import workloads as W
    from paper_1904_00031_gb300.vmc import VmcSr
    w = W.workload("c5", n_chains=1216, samples_per_chain=16)
    w.n_discard = 0
    w.n_cg = 2
    v = VmcSr(w, W.init_params(w.n, w.m, True, 0.01, w.seed), prec=nk.NK_PREC_BF16X2)
    for _ in range(2):
        for name in ("sample", "amplitudes", "energies", "sr"):
            a = torch.cuda.Event(enable_timing=True)
            b = torch.cuda.Event(enable_timing=True)
            a.record()
            getattr(v, name)()
            b.record()
            torch.cuda.synchronize()
            print(f"{name}: {a.elapsed_time(b):.3f} ms")
    print("acceptance", v.info()["acceptance"])


def run_gpu_batched(args):
    """64 uneven independent instances, one CUDA graph launch per iteration."""
    import torch

    from paper_1904_00031_gb300 import nk
    from paper_1904_00031_gb300 import workloads as W
    from paper_1904_00031_gb300 import replicas as R
    from paper_1904_00031_gb300.batch import BatchedVmc

    world, rank, local = R.env_world()
    R.init(world, "nccl")
    torch.cuda.set_device(local)
    nk.load_library()
    prec_name = args.prec if args.prec != "auto" else "bf16x2"
    prec = nk.NK_PREC_FP32 if prec_name == "fp32" else nk.NK_PREC_BF16X2
    insts = W.batched_instances(64, R.replica_seed(4242, rank), 1024)
    b = BatchedVmc(insts, prec=prec, graph=bool(args.graph), autotune=True)
    stream = torch.cuda.current_stream()

    def barrier():
        R.barrier(world)
        torch.cuda.synchronize()

    for _ in range(max(args.warmup, 2)):
        b.step()
    barrier()
    clocks = ClockSampler(local)
    t_bytes = sum(v.ns * v.w.m * (8 if v.w.is_complex else 4) for v in b.items)
    small = t_bytes <= 129e6
    flush = torch.empty(256 << 20, dtype=torch.uint8, device="cuda") if small else None
    ev_it = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
             for _ in range(args.steps)]
    for k in range(args.steps):
        if flush is not None:
            flush.zero_()  # evict the working set from the 129 MB L2 (outside the timing)
        ev_it[k][0].record(stream)
        b.step()
        ev_it[k][1].record(stream)
    barrier()
    clk = clocks.stop()
    ms = R.max_over_ranks(sum(a.elapsed_time(e) for a, e in ev_it), world, "cuda") / args.steps
    ns = b.n_samples
    return rank, {
        "metric": METRIC, "value": round(R.aggregate_rate(ns, world, ms / 1e3), 2),
        "unit": "samples/s",
        "n_gpus": world, "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(ms, 3),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
        "data": "synthetic (64 seeded uneven 1D TFIM / Heisenberg instances)",
        "config": {"workload": "batched_64_uneven_1d", "instances": len(insts),
                   "n_range": [min(w.n for w in insts), max(w.n for w in insts)],
                   "samples_per_iter": ns, "n_cg": 50, "prec": prec_name,
                   "graph": bool(args.graph), "parallelism": f"replicas x{world}",
                   "l2": (f"inputs larger than L2 (T over all instances is {t_bytes / 1e6:.0f} MB)"
                          if not small else f"inputs smaller than L2 (T over all instances is "
                          f"{t_bytes / 1e6:.1f} MB); L2 flushed before each timed iteration")},
        "sr_steps_per_s": round(1e3 / ms, 4), "roofline": None,
        "gpu_launches": b.launches_per_step() * args.steps, "clocks": clk,
    }


# ---------------------------------------------------------------------- widened rows

def _timed_calls(fn, steps, stream, flush=None) -> float:
    """Mean ms of `steps` calls fn(k) (CUDA events on `stream`; the L2 flushed
    before each call, outside the events, when `flush` is given)."""
    import torch
    evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
           for _ in range(steps)]
    for k in range(steps):
        if flush is not None:
            flush.zero_()
        evs[k][0].record(stream)
        fn(k)
        evs[k][1].record(stream)
    torch.cuda.synchronize()
    return sum(a.elapsed_time(b) for a, b in evs) / steps


# supervised learning shapes: (n, m, complex, target samples per step, the
# target's perturbation: small enough that ln psi - ln target spreads by O(1)
# over the samples, so that the overlap estimate rests on many of them)
SUP_SHAPES = {
    "c1": (10, 20, False, 400, 0.05),      # the paper's example: 10-site TFIM, 20 hidden units
    "c5": (400, 1600, True, 65536, 0.003),  # the 20x20 shapes
}


def run_gpu_supervised(args):
    """Supervised overlap learning (Sec. 2.2.3, Eq. 1): one nk_supervised_step per
    step (ln psi of the target samples, loss, gradient, AdaMax).  The target is a
    second RBM, the model's initial parameters perturbed by N(0, s^2), whose ln psi
    is computed once on the device; the samples are random configurations (the
    step's arithmetic does not depend on how they were drawn).  ln psi and the
    backward are also timed alone."""
    import torch

    from paper_1904_00031_gb300 import nk
    from paper_1904_00031_gb300 import workloads as W
    from paper_1904_00031_gb300 import replicas as R

    if args.workload not in SUP_SHAPES:
        raise SystemExit("--model supervised runs --workload c1 (the paper's example shape) or c5")
    world, rank, local = R.env_world()
    R.init(world, "nccl")
    torch.cuda.set_device(local)
    nk.load_library()
    n, m, cplx, ns, pert = SUP_SHAPES[args.workload]
    prec_name = args.prec if args.prec != "auto" else "bf16x2"
    prec = nk.NK_PREC_FP32 if prec_name == "fp32" else nk.NK_PREC_BF16X2
    seed = R.replica_seed(1238, rank)
    p = W.init_params(n, m, cplx, 0.01, seed)
    rbm = nk.Rbm(n, m, cplx)
    rbm.load(p.a, p.b, p.w)
    pt = W.perturb_params(p, pert, seed + 1)
    tgt = nk.Rbm(n, m, cplx)
    tgt.load(pt.a, pt.b, pt.w)
    sigma = torch.from_numpy(W.random_configs(ns, n, seed)).cuda()
    log_t = nk.nk_rbm_logpsi(tgt, sigma, nk.NK_PREC_FP32)
    pr = p.n_params * (2 if cplx else 1)
    mom = torch.zeros(2 * pr, dtype=torch.float64, device="cuda")
    info = torch.zeros(4, dtype=torch.float64, device="cuda")
    scratch = nk.supervised_scratch(rbm, ns)
    stream = torch.cuda.current_stream()
    step_no = [0]

    def step(_k, s=sigma, lt=log_t):
        step_no[0] += 1
        nk.nk_supervised_step(rbm, s, lt, prec=prec, lr=1e-3, step=step_no[0], moments=mom,
                              scratch=scratch, info_out=info)

    for k in range(args.warmup):
        step(k)
    loss0 = float(info[0].item())
    R.barrier(world)
    torch.cuda.synchronize()
    # working set: sigma, ln psi, the backward's theta / T chunk and the parameters
    small = ns * (n + 16) + min(ns, 16384) * m * (8 if cplx else 4) <= 129e6
    flush = torch.empty(256 << 20, dtype=torch.uint8, device="cuda") if small else None
    clocks = ClockSampler(local)
    ms = _timed_calls(step, args.steps, stream, flush)
    clk = clocks.stop()
    ms = R.max_over_ranks(ms, world, "cuda")
    loss1 = float(info[0].item())
    # the step's two contractions alone: ln psi of the samples, and the backward
    # (theta recomputed per chunk, the adjoint) with an upstream vector g
    lp_buf = torch.empty(ns, dtype=torch.complex128, device="cuda")
    g = torch.full((ns,), 1.0 / ns, dtype=torch.complex128, device="cuda")
    grad = torch.empty(p.n_params, dtype=torch.complex128 if cplx else torch.float64,
                       device="cuda")
    bscr = nk.backward_scratch(rbm, ns)
    lp_ms = _timed_calls(lambda _k: nk.nk_rbm_logpsi(rbm, sigma, prec, logpsi_out=lp_buf),
                         args.steps, stream, flush)
    bk_ms = _timed_calls(lambda _k: nk.nk_rbm_logpsi_backward(rbm, sigma, g, prec, grad, bscr),
                         args.steps, stream, flush)
    # end to end: the batch (samples and ln target) from pinned host memory, the
    # step, the info block back, every step
    h_sig = sigma.cpu().pin_memory()
    h_lt = log_t.cpu().pin_memory()
    h_info = torch.empty(4, dtype=torch.float64).pin_memory()
    d_sig = torch.empty_like(sigma)
    d_lt = torch.empty_like(log_t)

    def e2e(k):
        d_sig.copy_(h_sig, non_blocking=True)
        d_lt.copy_(h_lt, non_blocking=True)
        step(k, d_sig, d_lt)
        h_info.copy_(info, non_blocking=True)

    R.barrier(world)
    e2e_ms = R.max_over_ranks(_timed_calls(e2e, args.steps, stream), world, "cuda")
    # algorithmic FLOPs per step: theta = W sigma' for ln psi and again in the
    # backward, the adjoint contraction sum_s conj(O_s) g_s (complex W: 4 n m per
    # sample each, real: 2 n m)
    flops = 3.0 * ns * (4 if cplx else 2) * n * m
    pk, src = peaks()
    peak = pk.get("bf16_tflops_sustained", pk["bf16_tflops"])
    chunks = (ns + 16383) // 16384
    launches = 1 + 4 + chunks * (5 + (1 if chunks > 1 else 0)) + 1 + 1 + 2
    achieved = flops / (ms / 1e3) / 1e12
    return rank, {
        "metric": "supervised overlap learning (Eq. 1 loss, gradient, AdaMax) target samples/s",
        "value": round(R.aggregate_rate(ns, world, ms / 1e3), 2), "unit": "samples/s",
        "n_gpus": world, "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(ms, 4),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
        "data": "synthetic (random configurations; target = a perturbed RBM, ln psi on the device)",
        "config": {"workload": f"supervised_{args.workload}", "n": n, "m": m, "complex": cplx,
                   "samples_per_step": ns, "target_perturbation": pert, "prec": prec_name,
                   "optimizer": "AdaMax lr 1e-3",
                   "parallelism": f"replicas x{world}",
                   "l2": ("L2 flushed before each timed step" if small else
                          "inputs larger than L2")},
        "steps_per_s": round(1e3 / ms, 3), "loss_first": round(loss0, 6),
        "loss_last": round(loss1, 6),
        "parts_ms": {"logpsi": round(lp_ms, 4), "backward": round(bk_ms, 4)},
        "roofline": {"bound": "tensor" if prec == nk.NK_PREC_BF16X2 else "alu",
                     "achieved": round(achieved, 3),
                     "peak": peak if prec == nk.NK_PREC_BF16X2 else None,
                     "unit": "TFLOP/s",
                     "frac": round(achieved / peak, 4) if prec == nk.NK_PREC_BF16X2 else None,
                     "kernel": "whole step (ln psi, reductions, chunked backward, AdaMax)",
                     "traffic": None,
                     "peak_source": f"{src} bf16 dense TFLOP/s (sustained)"},
        "e2e": {"value": round(R.aggregate_rate(ns, world, e2e_ms / 1e3), 2), "unit": "samples/s",
                "h2d_bytes_per_step": int(h_sig.numel() + h_lt.numel() * 16),
                "d2h_bytes_per_step": 32},
        "gpu_launches": launches * args.steps, "clocks": clk,
    }


# FFNN shapes: (widths, complex, samples)
FFNN_SHAPES = {
    "c2": ([40, 80, 40], True, 16384),
    "c5": ([400, 1600, 400], True, 65536),
}


def run_gpu_ffnn(args):
    """Multi-layer ln cosh FFNN (Sec. 2.2.2): one step = nk_ffnn_logpsi and
    nk_ffnn_backward (grad = sum_s conj(O_s) g_s for an upstream vector g) on a
    batch of random configurations, CUDA-core FP32 contractions."""
    import numpy as np
    import torch

    from paper_1904_00031_gb300 import nk
    from paper_1904_00031_gb300 import workloads as W
    from paper_1904_00031_gb300 import replicas as R

    if args.workload not in FFNN_SHAPES:
        raise SystemExit("--model ffnn runs --workload c2 or c5")
    world, rank, local = R.env_world()
    R.init(world, "nccl")
    torch.cuda.set_device(local)
    nk.load_library()
    widths, cplx, ns = FFNN_SHAPES[args.workload]
    seed = R.replica_seed(1239, rank)
    net = nk.Ffnn(widths, cplx)
    net.load(W.init_ffnn_params(widths, cplx, 0.01, seed))
    sigma = torch.from_numpy(W.random_configs(ns, widths[0], seed)).cuda()
    rng = np.random.default_rng(seed + 1)
    g = torch.from_numpy(rng.normal(size=ns) + 1j * rng.normal(size=ns)).cuda() / ns
    scratch = net.scratch(ns)
    lp = torch.empty(ns, dtype=torch.complex128, device="cuda")
    grad = torch.empty(net.n_params, dtype=torch.complex128 if cplx else torch.float64,
                       device="cuda")
    stream = torch.cuda.current_stream()

    def fwd(_k):
        nk.nk_ffnn_logpsi(net, sigma, lp, scratch)

    def bwd(_k):
        nk.nk_ffnn_backward(net, sigma, g, grad, scratch)

    def step(k):
        fwd(k)
        bwd(k)

    for k in range(args.warmup):
        step(k)
    R.barrier(world)
    torch.cuda.synchronize()
    clocks = ClockSampler(local)
    ms = _timed_calls(step, args.steps, stream)
    ms_f = _timed_calls(fwd, args.steps, stream)
    ms_b = _timed_calls(bwd, args.steps, stream)
    clk = clocks.stop()
    ms = R.max_over_ranks(ms, world, "cuda")
    alu = nk.nk_measure_alu_peaks()
    peak = alu["fp32_fma_flops"] / 1e12
    # algorithmic FLOPs (complex multiply-add 8, complex x real 4): forward
    # h_l = W_l x_(l-1) + b_l; backward e_(l-1) = conj(tanh h) (e_l conj(W_l)) for
    # l > 1 and grad W_l = e_l^T conj(x_(l-1)) (the backward's recomputed forward
    # is not counted)
    L = len(widths) - 1
    per = [(4 if l == 1 else 8) * widths[l] * widths[l - 1] for l in range(1, L + 1)]
    f_fl = float(ns) * sum(per)
    b_fl = float(ns) * (sum(per) + sum(8 * widths[l] * widths[l - 1] for l in range(2, L + 1)))
    ach = (f_fl + b_fl) / (ms / 1e3) / 1e12
    launches = (L + 1) + 4 * L
    big = ns * sum(widths[1:]) * 16 > 129e6
    return rank, {
        "metric": "multi-layer ln cosh FFNN ln psi + gradient, samples/s",
        "value": round(R.aggregate_rate(ns, world, ms / 1e3), 2), "unit": "samples/s",
        "n_gpus": world, "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(ms, 4),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
        "data": "synthetic (random configurations, parameters N(0, 0.01^2), random upstream g)",
        "config": {"workload": f"ffnn_{args.workload}", "widths": widths, "complex": cplx,
                   "samples": ns, "parallelism": f"replicas x{world}",
                   "l2": ("activations larger than L2" if big else
                          "activations smaller than L2, not flushed")},
        "forward_ms": round(ms_f, 4), "backward_ms": round(ms_b, 4),
        "roofline": {"bound": "alu", "achieved": round(ach, 3), "peak": round(peak, 2),
                     "unit": "TFLOP/s", "frac": round(ach / peak, 4),
                     "kernel": "forward + backward (ffnn_fwd / wgrad / bwd kernels)",
                     "traffic": None,
                     "peak_source": "measured packed FP32 FMA rate (nk_measure_alu_peaks)"},
        "gpu_launches": launches * args.steps, "clocks": clk,
    }


def main():
    args = parse()
    if args.oracle_sample:
        spec = json.loads(args.oracle_sample)
        print(json.dumps(oracle_sample(spec["workload"], spec["n_chains"], spec["spc"],
                                       spec["n_cg"], spec.get("offset", 0))))
        return
    if args.profile_kernels:
        profile_kernels()
        return
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    nc, spc, ncg = ORACLE_SAMPLE[args.workload]
    if args.impl == "reference":
        if rank != 0:
            return
        if args.model != "rbm":
            print(json.dumps({"impl": "reference", "unavailable": "the CPU oracle arm times the "
                              "untied RBM only; run it without --model"}))
            return
        from paper_1904_00031_gb300 import workloads as W
        # the 64-instance batch: its first instance stands for the workload
        w = (W.workload(args.workload) if args.workload != "c4"
             else W.batched_instances(64, 4242, 1024)[0])
        tot_s, tot_n = 0.0, 0
        ncc, spcc, ncgc = ORACLE_SAMPLE_CORE[args.workload]
        cores = 1
        r = run_oracle_all_cores(args.workload, ncc, spcc, ncgc, args.warmup + args.steps)
        cores = r["cores"]
        tot_s = sum(r["seconds"][args.warmup:])
        tot_n = r["samples"] * args.steps
        val = tot_n / tot_s
        sample = (f"{cores} single-threaded oracle processes at once (one per host core), each "
                  f"{ncc} chains x ({spcc} samples + 1 burn-in sweep) of the {w.name} workload "
                  f"and a full oracle iteration incl. {ncgc} CG iterations, per step")
        print(json.dumps({
            "impl": "reference", "metric": METRIC, "value": round(val, 4), "unit": "samples/s",
            "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": round(1e3 * tot_s / args.steps, 3), "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": w.name, "n": w.n, "m": w.m, "complex": w.is_complex,
                       "chains": w.n_chains, "samples_per_chain": w.samples_per_chain,
                       "burn_in_sweeps": w.n_discard, "samples_per_iter": w.n_samples,
                       "moves": w.move, "n_cg": w.n_cg, "oracle_sample": sample},
            "cpu_baseline": {"value": round(val, 4), "unit": "samples/s", "cores": cores,
                             "kind": "oracle", "sample": sample},
            "e2e": {"value": round(val, 4), "unit": "samples/s", "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0},
        }))
        return
    base = None
    if rank == 0 and world == 1 and not args.no_baseline and args.model == "rbm":
        # before any CUDA call: the oracle runs in a fresh single-threaded process
        r = run_oracle_subprocess(args.workload, nc, spc, ncg)
        ncc, spcc, ncgc = ORACLE_SAMPLE_CORE[args.workload]
        ra = run_oracle_all_cores(args.workload, ncc, spcc, ncgc)
        ra["seconds"] = ra["seconds"][0]
        base = {"value": round(ra["samples"] / ra["seconds"], 4), "unit": "samples/s",
                "cores": ra["cores"], "kind": "oracle",
                "sample": f"{ra['cores']} single-threaded oracle processes at once, each "
                          f"{ncc} chains x ({spcc} samples + 1 burn-in sweep) and one full "
                          f"oracle VMC+SR iteration ({ncgc} CG iterations), "
                          f"{ra['seconds']:.1f} s wall",
                "one_core": {"value": round(r["samples"] / r["seconds"], 4), "cores": 1,
                             "sample": f"{nc} chains x ({spc} samples + 1 burn-in sweep), one "
                                       f"full oracle VMC+SR iteration ({ncg} CG iterations), "
                                       f"{r['seconds']:.1f} s"}}
    if args.model in ("supervised", "ffnn"):
        rank, out = (run_gpu_supervised if args.model == "supervised" else run_gpu_ffnn)(args)
        out["cpu_baseline"] = None
        if rank == 0:
            print(json.dumps(out))
        return
    if args.workload == "c4" and args.model != "rbm":
        raise SystemExit("--model symm runs the single-instance workloads (c1, c2, c3, c5)")
    rank, out = run_gpu_batched(args) if args.workload == "c4" else run_gpu(args)
    out["cpu_baseline"] = base
    if rank == 0:
        print(json.dumps(out))


if __name__ == "__main__":
    main()
