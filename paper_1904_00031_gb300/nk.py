"""Thin Python binding of the nk C ABI (include/nk.h): argument marshalling only.

Every function here calls the entry point of the same name in ``libnk.so``
with device pointers of torch tensors.  PyTorch provides device memory and
streams; every step of the computation runs in the library's CUDA kernels.
There is no CPU fallback: if the library is missing or the device is not an
sm_103a GPU, the calls raise.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np
import torch

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libnk.so")

NK_OK = 0
NK_ERR_INVALID_ARG = 1
NK_ERR_TIMEOUT = 6
NK_PREC_FP32 = 0
NK_PREC_BF16X2 = 1
NK_MOVE_FLIP = 0
NK_MOVE_EXCHANGE = 1
NK_LAYOUT_FACTORED = 0
NK_LAYOUT_DENSE = 1
NK_INFO_LEN = 8
INFO_KEYS = ("energy", "energy_imag", "variance", "error", "cg_iters", "cg_resid", "f_norm",
             "flags")

EXPORTS = (
    "nk_status_string", "nk_last_error", "nk_device_supported", "nk_rbm_workspace_bytes",
    "nk_rbm_prepare", "nk_rbm_logpsi", "nk_metropolis_sweep", "nk_operator_bytes",
    "nk_operator_upload", "nk_local_energy", "nk_logderiv", "nk_sr_scratch_bytes", "nk_sr_step",
    "nk_backward_scratch_bytes", "nk_rbm_logpsi_backward", "nk_sr_step_noalloc",
    "nk_metropolis_scratch_bytes", "nk_operator_moves", "nk_local_energy_scratch_bytes",
    "nk_sr_tune", "nk_sr_batch_desc_bytes", "nk_sr_batch_describe", "nk_sr_step_batch",
    "nk_query_status", "nk_debug_bounded_wait", "nk_measure_alu_peaks",
    "nk_batch_logpsi", "nk_batch_sweep", "nk_batch_local_energy",
    "nk_symm_tables_bytes", "nk_symm_upload", "nk_symm_expand", "nk_sr_symm_scratch_bytes",
    "nk_sr_step_symm", "nk_symm_build", "nk_supervised_scratch_bytes", "nk_supervised_step",
    "nk_pt_scratch_bytes", "nk_pt_sweep", "nk_ffnn_scratch_bytes", "nk_ffnn_logpsi",
    "nk_ffnn_backward", "nk_tune_shapes",
)
NK_SR_NOALLOC_MAX_BYTES = 16 << 20


class NkError(RuntimeError):
    pass


class _Rbm(C.Structure):
    _fields_ = [("n", C.c_int32), ("m", C.c_int32), ("is_complex", C.c_int32),
                ("sr_splits", C.c_int32), ("eloc_segs", C.c_int32), ("theta_segs", C.c_int32),
                ("sampler", C.c_int32), ("a", C.c_void_p), ("b", C.c_void_p), ("w", C.c_void_p),
                ("ws", C.c_void_p), ("ws_bytes", C.c_size_t)]


class _RbmSymm(C.Structure):
    _fields_ = [("n", C.c_int32), ("alpha", C.c_int32), ("n_perm", C.c_int32),
                ("is_complex", C.c_int32), ("a", C.c_void_p), ("b", C.c_void_p),
                ("w", C.c_void_p), ("tables", C.c_void_p), ("tables_bytes", C.c_size_t)]


class _Chains(C.Structure):
    _fields_ = [("nc", C.c_int32), ("group_size", C.c_int32), ("sigma", C.c_void_p),
                ("seed", C.c_uint64), ("counter", C.c_uint64), ("counter_dev", C.c_void_p)]


class _Ffnn(C.Structure):
    _fields_ = [("n_layers", C.c_int32), ("is_complex", C.c_int32), ("widths", C.c_void_p),
                ("params", C.c_void_p)]


class _SrBatchItem(C.Structure):
    _fields_ = [("rbm", C.c_void_p), ("sigma", C.c_void_p), ("t", C.c_void_p),
                ("eloc", C.c_void_p), ("weights", C.c_void_p), ("ns", C.c_int64),
                ("n_chains", C.c_int32), ("reserved", C.c_int32), ("scratch", C.c_void_p),
                ("scratch_bytes", C.c_size_t), ("info_out", C.c_void_p)]


class _LogpsiItem(C.Structure):
    _fields_ = [("rbm", C.c_void_p), ("sigma", C.c_void_p), ("ns", C.c_int64),
                ("logpsi_out", C.c_void_p), ("theta_out", C.c_void_p), ("stream", C.c_void_p)]


class _SweepItem(C.Structure):
    _fields_ = [("rbm", C.c_void_p), ("chains", C.c_void_p), ("move", C.c_int32),
                ("n_bonds", C.c_int32), ("bond_i", C.c_void_p), ("bond_k", C.c_void_p),
                ("n_discard", C.c_int32), ("n_samples_per_chain", C.c_int32),
                ("samples_out", C.c_void_p), ("n_accept_out", C.c_void_p),
                ("scratch", C.c_void_p), ("scratch_bytes", C.c_size_t), ("stream", C.c_void_p)]


class _ElocItem(C.Structure):
    _fields_ = [("rbm", C.c_void_p), ("op_dev", C.c_void_p), ("n_moves", C.c_int32),
                ("reserved", C.c_int32), ("sigma", C.c_void_p), ("theta", C.c_void_p),
                ("ns", C.c_int64), ("eloc_out", C.c_void_p), ("t_out", C.c_void_p),
                ("scratch", C.c_void_p), ("scratch_bytes", C.c_size_t), ("stream", C.c_void_p)]


class _Operator(C.Structure):
    _fields_ = [("n", C.c_int32), ("n_site_terms", C.c_int32), ("site_idx", C.c_void_p),
                ("site_mat", C.c_void_p), ("n_bond_terms", C.c_int32), ("reserved", C.c_int32),
                ("bond_i", C.c_void_p), ("bond_k", C.c_void_p), ("bond_mat", C.c_void_p)]


_lib = None


def load_library(path: str = LIB_PATH):
    """Load libnk.so (building nothing); raises if it is missing."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise NkError(f"{path} not found: build it with paper_1904_00031_gb300.build.build()")
    lib = C.CDLL(path)
    P, I32, I64, SZ, D = C.c_void_p, C.c_int32, C.c_int64, C.c_size_t, C.c_double
    sig = {
        "nk_status_string": (C.c_char_p, [I32]),
        "nk_last_error": (C.c_char_p, []),
        "nk_device_supported": (I32, []),
        "nk_rbm_workspace_bytes": (SZ, [I32, I32, I32]),
        "nk_rbm_prepare": (I32, [P, P]),
        "nk_rbm_logpsi": (I32, [P, P, I64, I32, P, P, P]),
        "nk_metropolis_scratch_bytes": (SZ, [I32, I32, I32, I32, I32]),
        "nk_metropolis_sweep": (I32, [P, P, I32, P, P, I32, I32, I32, P, P, P, SZ, P]),
        "nk_operator_bytes": (SZ, [P]),
        "nk_operator_upload": (I32, [P, P, SZ, P]),
        "nk_operator_moves": (I32, [P]),
        "nk_local_energy_scratch_bytes": (SZ, [I32, I32, I32]),
        "nk_local_energy": (I32, [P, P, I32, P, P, I64, P, P, P, SZ, P]),
        "nk_logderiv": (I32, [P, P, P, I64, I32, P, P]),
        "nk_sr_scratch_bytes": (SZ, [I32, I32, I32, I64]),
        "nk_sr_step": (I32, [P, P, P, P, P, I64, I32, D, D, I32, D, I32, P, SZ, P, P]),
        "nk_backward_scratch_bytes": (SZ, [I32, I32, I32, I64]),
        "nk_rbm_logpsi_backward": (I32, [P, P, I64, P, P, I32, P, SZ, P]),
        "nk_sr_step_noalloc": (I32, [P, P, P, P, P, I64, I32, D, D, I32, D, I32, P, P]),
        "nk_sr_tune": (I32, [P, P, P, I64, I32, P, SZ, P]),
        "nk_sr_batch_desc_bytes": (SZ, [I32]),
        "nk_sr_batch_describe": (I32, [P, I32, I32, P, SZ]),
        "nk_sr_step_batch": (I32, [P, I32, P, D, D, I32, D, I32, P]),
        "nk_query_status": (I32, [P, P]),
        "nk_debug_bounded_wait": (I32, [C.c_uint32, P]),
        "nk_measure_alu_peaks": (I32, [P]),
        "nk_batch_logpsi": (I32, [P, I32, I32, P]),
        "nk_batch_sweep": (I32, [P, I32, P]),
        "nk_batch_local_energy": (I32, [P, I32, P]),
        "nk_symm_tables_bytes": (SZ, [I32, I32, I32]),
        "nk_symm_upload": (I32, [P, I32, I32, I32, P, SZ, P]),
        "nk_symm_build": (I32, [P, I32, I32, I32, P, SZ]),
        "nk_symm_expand": (I32, [P, P, P]),
        "nk_sr_symm_scratch_bytes": (SZ, [I32, I32, I32, I32, I64]),
        "nk_sr_step_symm": (I32, [P, P, P, P, P, P, I64, I32, D, D, I32, D, I32, P, SZ, P, P]),
        "nk_supervised_scratch_bytes": (SZ, [I32, I32, I32, I64]),
        "nk_pt_scratch_bytes": (SZ, [I32, I32, I32, I32, I32, I32]),
        "nk_ffnn_scratch_bytes": (SZ, [P, I64]),
        "nk_tune_shapes": (I32, [P, P, I32, P, I64, P, P, P, P, SZ, P]),
        "nk_ffnn_logpsi": (I32, [P, P, I64, P, P, SZ, P]),
        "nk_ffnn_backward": (I32, [P, P, I64, P, P, P, SZ, P]),
        "nk_pt_sweep": (I32, [P, P, I32, I32, P, P, I32, I32, I32, P, P, P, P, SZ, P]),
        "nk_supervised_step": (I32, [P, P, P, P, I64, I32, D, D, D, I32, P, P, P, SZ, P, P]),
    }
    for name, (res, args) in sig.items():
        f = getattr(lib, name)
        f.restype = res
        f.argtypes = args
    _lib = lib
    return lib


def _check(status: int, what: str):
    if status != NK_OK:
        lib = load_library()
        raise NkError(f"{what}: {lib.nk_status_string(status).decode()} "
                      f"({lib.nk_last_error().decode()})")


def _ptr(t):
    return None if t is None else C.c_void_p(t.data_ptr())


def _stream(stream=None):
    s = stream if stream is not None else torch.cuda.current_stream()
    return C.c_void_p(s.cuda_stream)


def _require_gpu(*tensors):
    for t in tensors:
        if t is not None and not t.is_cuda:
            raise NkError("nk: every tensor argument must live on the CUDA device")


# ---------------------------------------------------------------------- RBM

class Rbm:
    """FP64 master parameters on the device plus the library's derived planes."""

    def __init__(self, n: int, m: int, is_complex: bool, device="cuda"):
        lib = load_library()
        self.n, self.m, self.is_complex = int(n), int(m), bool(is_complex)
        dt = torch.float64
        k = 2 if is_complex else 1
        self.a = torch.zeros(n * k, dtype=dt, device=device)
        self.b = torch.zeros(m * k, dtype=dt, device=device)
        self.w = torch.zeros(m * n * k, dtype=dt, device=device)
        nb = lib.nk_rbm_workspace_bytes(n, m, int(is_complex))
        self.ws = torch.empty(nb + 256, dtype=torch.uint8, device=device)
        off = (-self.ws.data_ptr()) % 256
        self._ws_ptr = self.ws.data_ptr() + off
        self._ws_bytes = nb
        self._s = _Rbm(self.n, self.m, int(is_complex), 0, 0, 0, 0, self.a.data_ptr(),
                       self.b.data_ptr(), self.w.data_ptr(), self._ws_ptr, nb)

    @property
    def n_params(self) -> int:
        return self.n + self.m + self.n * self.m

    def struct(self):
        return C.byref(self._s)

    def load(self, a, b, w, stream=None):
        """Copy FP64 parameters (numpy; complex allowed) in and refresh the planes."""
        def flat(x):
            x = np.asarray(x)
            if self.is_complex:
                x = x.astype(np.complex128).reshape(-1)
                return torch.from_numpy(np.stack([x.real, x.imag], axis=1).reshape(-1).copy())
            return torch.from_numpy(np.asarray(x, dtype=np.float64).reshape(-1).copy())
        self.a.copy_(flat(a))
        self.b.copy_(flat(b))
        self.w.copy_(flat(w))
        nk_rbm_prepare(self, stream)

    def params_numpy(self):
        def un(t, shape):
            x = t.detach().cpu().numpy()
            if self.is_complex:
                x = x[0::2] + 1j * x[1::2]
            return x.reshape(shape)
        return un(self.a, (self.n,)), un(self.b, (self.m,)), un(self.w, (self.m, self.n))

    def f32_dtype(self):
        return torch.complex64 if self.is_complex else torch.float32


def nk_query_status(flags=None, stream=None):
    """Enqueue the device status query; returns the int32 device tensor that
    receives the OR of the status bits (read it after the stream passes)."""
    if flags is None:
        flags = torch.zeros(1, dtype=torch.int32, device="cuda")
    _check(load_library().nk_query_status(_ptr(flags), _stream(stream)), "nk_query_status")
    return flags


def nk_measure_alu_peaks() -> dict:
    """FP32 FMA FLOP/s and MUFU ex2 / lg2 / sin op/s measured on the current GPU."""
    out = (C.c_double * 4)()
    _check(load_library().nk_measure_alu_peaks(C.cast(out, C.c_void_p)), "nk_measure_alu_peaks")
    return {"fp32_fma_flops": out[0], "mufu_ex2_ops": out[1], "mufu_lg2_ops": out[2],
            "mufu_sin_ops": out[3]}


def nk_debug_bounded_wait(polls: int, stream=None):
    _check(load_library().nk_debug_bounded_wait(int(polls), _stream(stream)),
           "nk_debug_bounded_wait")


def nk_rbm_prepare(rbm: Rbm, stream=None):
    _check(load_library().nk_rbm_prepare(rbm.struct(), _stream(stream)), "nk_rbm_prepare")


def nk_rbm_logpsi(rbm: Rbm, sigma, prec=NK_PREC_FP32, logpsi_out=None, theta_out=None,
                  stream=None):
    """ln psi (complex128 [ns]); optionally theta into ``theta_out`` ([ns, m] F32)."""
    _require_gpu(sigma, theta_out)
    ns = sigma.shape[0]
    if logpsi_out is None:
        logpsi_out = torch.empty(ns, dtype=torch.complex128, device=sigma.device)
    _check(load_library().nk_rbm_logpsi(rbm.struct(), _ptr(sigma), ns, prec, _ptr(logpsi_out),
                                        _ptr(theta_out), _stream(stream)), "nk_rbm_logpsi")
    return logpsi_out


def nk_rbm_theta(rbm: Rbm, sigma, theta_out, prec=NK_PREC_FP32, stream=None):
    """theta = W sigma + b only ([ns, m] F32 into ``theta_out``): nk_rbm_logpsi
    with a NULL ln psi output, which skips the ln cosh epilogue."""
    _require_gpu(sigma, theta_out)
    _check(load_library().nk_rbm_logpsi(rbm.struct(), _ptr(sigma), sigma.shape[0], prec, None,
                                        _ptr(theta_out), _stream(stream)), "nk_rbm_logpsi")
    return theta_out


class Chains:
    """Persistent Markov chains: device states plus the Philox seed and counter."""

    def __init__(self, sigma0, group_size: int, seed: int, device="cuda",
                 device_counter: bool = False):
        s = torch.as_tensor(np.asarray(sigma0, dtype=np.int8))
        self.sigma = s.to(device).contiguous()
        self.nc, self.n = self.sigma.shape
        self.counter_dev = None
        cptr = None
        if device_counter:
            # uint64 counter on the device (held in an int64 tensor)
            self.counter_dev = torch.zeros(1, dtype=torch.int64, device=device)
            cptr = self.counter_dev.data_ptr()
        self._s = _Chains(self.nc, int(group_size), self.sigma.data_ptr(), int(seed), 0, cptr)

    @property
    def counter(self) -> int:
        if self.counter_dev is not None:
            return int(self.counter_dev.item()) & 0xFFFFFFFFFFFFFFFF
        return int(self._s.counter)

    @counter.setter
    def counter(self, v: int):
        if self.counter_dev is not None:
            self.counter_dev.fill_(int(v))
        self._s.counter = int(v)

    @property
    def group_size(self) -> int:
        return int(self._s.group_size)

    @property
    def seed(self) -> int:
        return int(self._s.seed)


def metropolis_scratch(rbm: Rbm, move: int, n_bonds: int, device="cuda"):
    nb = load_library().nk_metropolis_scratch_bytes(rbm.n, rbm.m, int(rbm.is_complex), move,
                                                     n_bonds)
    return torch.empty(max(nb, 1), dtype=torch.uint8, device=device)


def nk_metropolis_sweep(rbm: Rbm, chains: Chains, move: int, bond_i=None, bond_k=None,
                        n_discard: int = 1, n_samples_per_chain: int = 1, samples_out=None,
                        n_accept_out=None, scratch=None, stream=None):
    _require_gpu(bond_i, bond_k, samples_out, n_accept_out, scratch)
    nb = 0 if bond_i is None else int(bond_i.shape[0])
    if samples_out is None:
        samples_out = torch.empty(chains.nc * n_samples_per_chain, rbm.n, dtype=torch.int8,
                                  device=chains.sigma.device)
    if scratch is None and load_library().nk_metropolis_scratch_bytes(
            rbm.n, rbm.m, int(rbm.is_complex), move, nb) > 0:
        scratch = metropolis_scratch(rbm, move, nb, chains.sigma.device)
    _check(load_library().nk_metropolis_sweep(
        rbm.struct(), C.byref(chains._s), move, _ptr(bond_i), _ptr(bond_k), nb, n_discard,
        n_samples_per_chain, _ptr(samples_out), _ptr(n_accept_out), _ptr(scratch),
        0 if scratch is None else scratch.numel(), _stream(stream)), "nk_metropolis_sweep")
    return samples_out


def pt_scratch(rbm: Rbm, move: int, n_bonds: int, nc: int, device="cuda"):
    nb = load_library().nk_pt_scratch_bytes(rbm.n, rbm.m, int(rbm.is_complex), move, n_bonds, nc)
    return torch.empty(max(nb, 1), dtype=torch.uint8, device=device)


def nk_pt_sweep(rbm: Rbm, chains: Chains, n_replicas: int, move: int, bond_i=None, bond_k=None,
                n_discard: int = 1, n_samples_per_chain: int = 1, samples_out=None,
                n_accept_out=None, n_swap_out=None, scratch=None, stream=None):
    """Parallel tempering over ladders of ``n_replicas`` replicas (chain-major in
    ``chains``); returns the samples of the beta = 1 replicas."""
    _require_gpu(bond_i, bond_k, samples_out, n_accept_out, n_swap_out, scratch)
    nb = 0 if bond_i is None else int(bond_i.shape[0])
    n_lad = chains.nc // n_replicas
    if samples_out is None:
        samples_out = torch.empty(n_lad * n_samples_per_chain, rbm.n, dtype=torch.int8,
                                  device=chains.sigma.device)
    if scratch is None:
        scratch = pt_scratch(rbm, move, nb, chains.nc, chains.sigma.device)
    _check(load_library().nk_pt_sweep(
        rbm.struct(), C.byref(chains._s), n_replicas, move, _ptr(bond_i), _ptr(bond_k), nb,
        n_discard, n_samples_per_chain, _ptr(samples_out), _ptr(n_accept_out), _ptr(n_swap_out),
        _ptr(scratch), scratch.numel(), _stream(stream)), "nk_pt_sweep")
    return samples_out


class Operator:
    """A Hamiltonian (workloads.Operator) compiled into device memory."""

    def __init__(self, op, device="cuda", stream=None):
        lib = load_library()
        self.n = op.n
        self._site_idx = np.ascontiguousarray(op.site_idx, dtype=np.int32)
        self._site_mat = np.ascontiguousarray(
            np.stack([op.site_mat.real, op.site_mat.imag], axis=-1), dtype=np.float64)
        self._bond_i = np.ascontiguousarray(op.bond_i, dtype=np.int32)
        self._bond_k = np.ascontiguousarray(op.bond_k, dtype=np.int32)
        self._bond_mat = np.ascontiguousarray(
            np.stack([op.bond_mat.real, op.bond_mat.imag], axis=-1), dtype=np.float64)
        self._s = _Operator(op.n, op.n_site_terms, self._site_idx.ctypes.data,
                            self._site_mat.ctypes.data, op.n_bond_terms, 0,
                            self._bond_i.ctypes.data, self._bond_k.ctypes.data,
                            self._bond_mat.ctypes.data)
        nb = lib.nk_operator_bytes(C.byref(self._s))
        if nb == 0:
            raise NkError("nk_operator_bytes: invalid operator " + lib.nk_last_error().decode())
        self.n_moves = int(lib.nk_operator_moves(C.byref(self._s)))
        self.dev = torch.empty(nb, dtype=torch.uint8, device=device)
        _check(lib.nk_operator_upload(C.byref(self._s), _ptr(self.dev), nb, _stream(stream)),
               "nk_operator_upload")


def local_energy_scratch(rbm: Rbm, op: Operator, device="cuda"):
    nb = load_library().nk_local_energy_scratch_bytes(rbm.m, int(rbm.is_complex), op.n_moves)
    return torch.empty(max(nb, 1), dtype=torch.uint8, device=device)


def nk_local_energy(rbm: Rbm, op: Operator, sigma, theta, eloc_out=None, t_out=None,
                    scratch=None, stream=None):
    _require_gpu(sigma, theta, t_out, scratch)
    ns = sigma.shape[0]
    if eloc_out is None:
        eloc_out = torch.empty(ns, dtype=torch.complex128, device=sigma.device)
    if scratch is None:
        scratch = local_energy_scratch(rbm, op, sigma.device)
    _check(load_library().nk_local_energy(rbm.struct(), _ptr(op.dev), op.n_moves, _ptr(sigma),
                                          _ptr(theta), ns, _ptr(eloc_out), _ptr(t_out),
                                          _ptr(scratch), scratch.numel(), _stream(stream)),
           "nk_local_energy")
    return eloc_out


def nk_logderiv(rbm: Rbm, sigma, theta, layout=NK_LAYOUT_FACTORED, o_out=None, stream=None):
    _require_gpu(sigma, theta, o_out)
    ns = sigma.shape[0]
    if o_out is None:
        cols = rbm.m if layout == NK_LAYOUT_FACTORED else rbm.n_params
        o_out = torch.empty(ns, cols, dtype=rbm.f32_dtype(), device=sigma.device)
    _check(load_library().nk_logderiv(rbm.struct(), _ptr(sigma), _ptr(theta), ns, layout,
                                      _ptr(o_out), _stream(stream)), "nk_logderiv")
    return o_out


def sr_scratch(rbm: Rbm, ns: int, device="cuda"):
    nb = load_library().nk_sr_scratch_bytes(rbm.n, rbm.m, int(rbm.is_complex), ns)
    return torch.empty(nb, dtype=torch.uint8, device=device)


def nk_sr_step(rbm: Rbm, sigma, t, eloc, n_chains: int, diag_shift: float, lr: float, n_cg: int,
               cg_rtol: float = 1e-12, prec=NK_PREC_FP32, weights=None, scratch=None,
               info_out=None, stream=None):
    _require_gpu(sigma, t, eloc, weights, scratch, info_out)
    ns = sigma.shape[0]
    if scratch is None:
        scratch = sr_scratch(rbm, ns, sigma.device)
    if info_out is None:
        info_out = torch.zeros(NK_INFO_LEN, dtype=torch.float64, device=sigma.device)
    _check(load_library().nk_sr_step(
        rbm.struct(), _ptr(sigma), _ptr(t), _ptr(eloc), _ptr(weights), ns, n_chains,
        float(diag_shift), float(lr), int(n_cg), float(cg_rtol), prec, _ptr(scratch),
        scratch.numel(), _ptr(info_out), _stream(stream)), "nk_sr_step")
    return info_out


def nk_sr_tune(rbm: Rbm, sigma, t, prec=NK_PREC_FP32, scratch=None, stream=None) -> int:
    """Autotune the split-K count of the SR contractions (synchronises); returns it
    and stores it in the RBM for later nk_sr_step calls."""
    _require_gpu(sigma, t, scratch)
    ns = sigma.shape[0]
    if scratch is None:
        scratch = sr_scratch(rbm, ns, sigma.device)
    _check(load_library().nk_sr_tune(rbm.struct(), _ptr(sigma), _ptr(t), ns, prec, _ptr(scratch),
                                     scratch.numel(), _stream(stream)), "nk_sr_tune")
    return int(rbm._s.sr_splits)


def nk_tune_shapes(rbm: Rbm, op: Operator, sigma, theta_tmp, eloc_tmp, scratch, t_tmp=None,
                   stream=None):
    """Autotune the theta / local-energy tile shapes on these samples
    (synchronises); returns (theta_segs, eloc_segs), also stored in the RBM."""
    _require_gpu(sigma, theta_tmp, eloc_tmp, scratch, t_tmp)
    _check(load_library().nk_tune_shapes(rbm.struct(), _ptr(op.dev), op.n_moves, _ptr(sigma),
                                         sigma.shape[0], _ptr(theta_tmp), _ptr(eloc_tmp),
                                         _ptr(t_tmp), _ptr(scratch), scratch.numel(),
                                         _stream(stream)), "nk_tune_shapes")
    return int(rbm._s.theta_segs), int(rbm._s.eloc_segs)


def info_dict(info) -> dict:
    v = info.detach().cpu().numpy()
    return {k: float(x) for k, x in zip(INFO_KEYS, v)}


def backward_scratch(rbm: Rbm, ns: int, device="cuda"):
    nb = load_library().nk_backward_scratch_bytes(rbm.n, rbm.m, int(rbm.is_complex), ns)
    return torch.empty(nb, dtype=torch.uint8, device=device)


def nk_rbm_logpsi_backward(rbm: Rbm, sigma, g, prec=NK_PREC_FP32, grad_out=None, scratch=None,
                           stream=None):
    """grad_k = sum_s conj(O_sk) g_s, F64 [P] (complex128 for a complex RBM)."""
    _require_gpu(sigma, g, grad_out, scratch)
    ns = sigma.shape[0]
    if scratch is None:
        scratch = backward_scratch(rbm, ns, sigma.device)
    if grad_out is None:
        grad_out = torch.empty(rbm.n_params,
                               dtype=torch.complex128 if rbm.is_complex else torch.float64,
                               device=sigma.device)
    g = g.to(torch.complex128).contiguous()
    _check(load_library().nk_rbm_logpsi_backward(rbm.struct(), _ptr(sigma), ns, _ptr(g),
                                                 _ptr(grad_out), prec, _ptr(scratch),
                                                 scratch.numel(), _stream(stream)),
           "nk_rbm_logpsi_backward")
    return grad_out


def nk_sr_step_noalloc(rbm: Rbm, sigma, t, eloc, n_chains: int, diag_shift: float, lr: float,
                       n_cg: int, cg_rtol: float = 1e-12, prec=NK_PREC_FP32, weights=None,
                       info_out=None, stream=None):
    """nk_sr_step with the library's built-in scratch array (no scratch argument);
    for callers that cannot allocate device memory.  Calls must not overlap."""
    _require_gpu(sigma, t, eloc, weights, info_out)
    ns = sigma.shape[0]
    if info_out is None:
        info_out = torch.zeros(NK_INFO_LEN, dtype=torch.float64, device=sigma.device)
    _check(load_library().nk_sr_step_noalloc(
        rbm.struct(), _ptr(sigma), _ptr(t), _ptr(eloc), _ptr(weights), ns, n_chains,
        float(diag_shift), float(lr), int(n_cg), float(cg_rtol), prec, _ptr(info_out),
        _stream(stream)), "nk_sr_step_noalloc")
    return info_out


def supervised_scratch(rbm: Rbm, ns: int, device="cuda"):
    nb = load_library().nk_supervised_scratch_bytes(rbm.n, rbm.m, int(rbm.is_complex), ns)
    return torch.empty(nb, dtype=torch.uint8, device=device)


def nk_supervised_step(rbm: Rbm, sigma, log_target, prec=NK_PREC_FP32, lr: float = 1e-3,
                       beta1: float = 0.9, beta2: float = 0.999, step: int = 1, moments=None,
                       grad_out=None, weights=None, scratch=None, info_out=None, stream=None):
    """One supervised step (loss of Eq. 1, its gradient, AdaMax if ``moments``);
    returns the info tensor [loss, overlap, shift, flags]."""
    _require_gpu(sigma, log_target, weights, moments, grad_out, scratch, info_out)
    ns = sigma.shape[0]
    if scratch is None:
        scratch = supervised_scratch(rbm, ns, sigma.device)
    if info_out is None:
        info_out = torch.zeros(4, dtype=torch.float64, device=sigma.device)
    lt = log_target.to(torch.complex128).contiguous()
    _check(load_library().nk_supervised_step(
        rbm.struct(), _ptr(sigma), _ptr(lt), _ptr(weights), ns, prec, float(lr), float(beta1),
        float(beta2), int(step), _ptr(moments), _ptr(grad_out), _ptr(scratch), scratch.numel(),
        _ptr(info_out), _stream(stream)), "nk_supervised_step")
    return info_out


class Ffnn:
    """A dense ln cosh network (widths [n, w_1, .., w_L]) with FP64 master
    parameters on the device (flat, layer by layer: W_l row-major, then b_l)."""

    def __init__(self, widths, is_complex: bool, device="cuda"):
        load_library()
        self.widths = np.ascontiguousarray(np.asarray(widths, dtype=np.int32))
        self.is_complex = bool(is_complex)
        self.n_params = int(sum(int(self.widths[l]) * (int(self.widths[l - 1]) + 1)
                                for l in range(1, len(self.widths))))
        self.params = torch.zeros(self.n_params * (2 if is_complex else 1), dtype=torch.float64,
                                  device=device)
        self._s = _Ffnn(len(self.widths) - 1, int(is_complex), self.widths.ctypes.data,
                        self.params.data_ptr())

    def struct(self):
        return C.byref(self._s)

    def load(self, flat):
        x = np.asarray(flat)
        if self.is_complex:
            x = x.astype(np.complex128)
            x = np.stack([x.real, x.imag], axis=1).reshape(-1)
        self.params.copy_(torch.from_numpy(np.ascontiguousarray(x, dtype=np.float64)))

    def scratch(self, ns: int, device="cuda"):
        nb = load_library().nk_ffnn_scratch_bytes(self.struct(), ns)
        return torch.empty(max(nb, 1), dtype=torch.uint8, device=device)


def nk_ffnn_logpsi(f: Ffnn, sigma, logpsi_out=None, scratch=None, stream=None):
    _require_gpu(sigma, logpsi_out, scratch)
    ns = sigma.shape[0]
    if logpsi_out is None:
        logpsi_out = torch.empty(ns, dtype=torch.complex128, device=sigma.device)
    if scratch is None:
        scratch = f.scratch(ns, sigma.device)
    _check(load_library().nk_ffnn_logpsi(f.struct(), _ptr(sigma), ns, _ptr(logpsi_out),
                                         _ptr(scratch), scratch.numel(), _stream(stream)),
           "nk_ffnn_logpsi")
    return logpsi_out


def nk_ffnn_backward(f: Ffnn, sigma, g, grad_out=None, scratch=None, stream=None):
    """grad_k = sum_s conj(O_sk) g_s (complex128 [P], or float64 [P] if real)."""
    _require_gpu(sigma, g, grad_out, scratch)
    ns = sigma.shape[0]
    if scratch is None:
        scratch = f.scratch(ns, sigma.device)
    if grad_out is None:
        grad_out = torch.empty(f.n_params,
                               dtype=torch.complex128 if f.is_complex else torch.float64,
                               device=sigma.device)
    g = g.to(torch.complex128).contiguous()
    _check(load_library().nk_ffnn_backward(f.struct(), _ptr(sigma), ns, _ptr(g), _ptr(grad_out),
                                           _ptr(scratch), scratch.numel(), _stream(stream)),
           "nk_ffnn_backward")
    return grad_out


class SrBatch:
    """Many independent SR problems advanced with one launch per kernel
    (nk_sr_step_batch).  ``items`` is a list of dicts with keys rbm (Rbm), sigma,
    t, eloc, scratch, info (device tensors), n_chains and optionally weights.
    The descriptors are built once here; build a new SrBatch if a pointer or a
    size changes."""

    def __init__(self, items, prec=NK_PREC_BF16X2, device="cuda"):
        lib = load_library()
        self.prec = prec
        self._keep = items
        arr = (_SrBatchItem * len(items))()
        for k, it in enumerate(items):
            _require_gpu(it["sigma"], it["t"], it["eloc"], it["scratch"], it["info"],
                         it.get("weights"))
            r = it["rbm"]
            arr[k].rbm = C.addressof(r._s)
            arr[k].sigma = it["sigma"].data_ptr()
            arr[k].t = it["t"].data_ptr()
            arr[k].eloc = it["eloc"].data_ptr()
            w = it.get("weights")
            arr[k].weights = None if w is None else w.data_ptr()
            arr[k].ns = int(it["sigma"].shape[0])
            arr[k].n_chains = int(it["n_chains"])
            arr[k].reserved = 0
            arr[k].scratch = it["scratch"].data_ptr()
            arr[k].scratch_bytes = it["scratch"].numel()
            arr[k].info_out = it["info"].data_ptr()
        self._items = arr
        self.n = len(items)
        nb = lib.nk_sr_batch_desc_bytes(self.n)
        host = np.zeros(nb, dtype=np.uint8)
        _check(lib.nk_sr_batch_describe(C.cast(arr, C.c_void_p), self.n, prec,
                                        host.ctypes.data_as(C.c_void_p), nb),
               "nk_sr_batch_describe")
        self.desc = torch.from_numpy(host).to(device)

    def step(self, diag_shift: float, lr: float, n_cg: int, cg_rtol: float = 1e-12, stream=None):
        _check(load_library().nk_sr_step_batch(
            C.cast(self._items, C.c_void_p), self.n, _ptr(self.desc), float(diag_shift),
            float(lr), int(n_cg), float(cg_rtol), self.prec, _stream(stream)),
            "nk_sr_step_batch")


# ---------------------------------------------------------------------- batches

def _item_stream(st):
    return None if st is None else C.c_void_p(st.cuda_stream).value


def nk_batch_logpsi(jobs, prec=NK_PREC_FP32, stream=None):
    """jobs: list of dicts {rbm, sigma, logpsi_out, theta_out?, stream?}; one call."""
    items = (_LogpsiItem * max(1, len(jobs)))()
    for k, j in enumerate(jobs):
        _require_gpu(j["sigma"], j["logpsi_out"], j.get("theta_out"))
        items[k] = _LogpsiItem(C.addressof(j["rbm"]._s), _ptr(j["sigma"]), int(j["sigma"].shape[0]),
                               _ptr(j["logpsi_out"]), _ptr(j.get("theta_out")),
                               _item_stream(j.get("stream")))
    _check(load_library().nk_batch_logpsi(C.cast(items, C.c_void_p), len(jobs), prec,
                                          _stream(stream)), "nk_batch_logpsi")


def nk_batch_sweep(jobs, stream=None):
    """jobs: list of dicts {rbm, chains, move, bond_i?, bond_k?, n_discard,
    n_samples_per_chain, samples_out, n_accept_out?, scratch?, stream?}."""
    items = (_SweepItem * max(1, len(jobs)))()
    for k, j in enumerate(jobs):
        rbm, ch = j["rbm"], j["chains"]
        bi, bk = j.get("bond_i"), j.get("bond_k")
        _require_gpu(bi, bk, j["samples_out"], j.get("n_accept_out"), j.get("scratch"))
        sc = j.get("scratch")
        items[k] = _SweepItem(C.addressof(rbm._s), C.addressof(ch._s),
                              j["move"], 0 if bi is None else int(bi.shape[0]), _ptr(bi),
                              _ptr(bk), j["n_discard"], j["n_samples_per_chain"],
                              _ptr(j["samples_out"]), _ptr(j.get("n_accept_out")), _ptr(sc),
                              0 if sc is None else sc.numel(), _item_stream(j.get("stream")))
    _check(load_library().nk_batch_sweep(C.cast(items, C.c_void_p), len(jobs), _stream(stream)),
           "nk_batch_sweep")


def nk_batch_local_energy(jobs, stream=None):
    """jobs: list of dicts {rbm, op, sigma, theta, eloc_out, t_out?, scratch, stream?}."""
    items = (_ElocItem * max(1, len(jobs)))()
    for k, j in enumerate(jobs):
        _require_gpu(j["sigma"], j["theta"], j["eloc_out"], j.get("t_out"), j["scratch"])
        items[k] = _ElocItem(C.addressof(j["rbm"]._s), _ptr(j["op"].dev), j["op"].n_moves, 0,
                             _ptr(j["sigma"]), _ptr(j["theta"]), int(j["sigma"].shape[0]),
                             _ptr(j["eloc_out"]), _ptr(j.get("t_out")), _ptr(j["scratch"]),
                             j["scratch"].numel(), _item_stream(j.get("stream")))
    _check(load_library().nk_batch_local_energy(C.cast(items, C.c_void_p), len(jobs),
                                                _stream(stream)), "nk_batch_local_energy")


# ---------------------------------------------------------------------- symmetric RBM

class RbmSymm:
    """Tied FP64 parameters (at [1], bt [alpha], Wt [alpha, n]) of a symmetric RBM
    over the permutation table ``perm`` [n_perm, n], its tie tables on the device,
    and ``rbm``, the untied RBM (m = alpha n_perm) it stands for."""

    def __init__(self, perm, alpha: int, is_complex: bool, device="cuda", stream=None):
        lib = load_library()
        perm = np.ascontiguousarray(np.asarray(perm, dtype=np.int32))
        self.n_perm, self.n = (int(v) for v in perm.shape)
        self.alpha, self.is_complex = int(alpha), bool(is_complex)
        k = 2 if is_complex else 1
        dt = torch.float64
        self.a = torch.zeros(k, dtype=dt, device=device)
        self.b = torch.zeros(self.alpha * k, dtype=dt, device=device)
        self.w = torch.zeros(self.alpha * self.n * k, dtype=dt, device=device)
        nb = lib.nk_symm_tables_bytes(self.n, self.alpha, self.n_perm)
        if nb == 0:
            raise NkError("nk_symm_tables_bytes: sizes out of range")
        self.tables = torch.empty(nb + 256, dtype=torch.uint8, device=device)
        off = (-self.tables.data_ptr()) % 256
        tp = self.tables.data_ptr() + off
        _check(lib.nk_symm_upload(perm.ctypes.data_as(C.c_void_p), self.n, self.alpha,
                                  self.n_perm, C.c_void_p(tp), nb, _stream(stream)),
               "nk_symm_upload")
        self._s = _RbmSymm(self.n, self.alpha, self.n_perm, int(is_complex), self.a.data_ptr(),
                           self.b.data_ptr(), self.w.data_ptr(), tp, nb)
        self.rbm = Rbm(self.n, self.alpha * self.n_perm, is_complex, device)

    @property
    def n_params(self) -> int:
        return 1 + self.alpha + self.alpha * self.n

    def struct(self):
        return C.byref(self._s)

    def load(self, a, b, w, stream=None):
        """Copy tied FP64 parameters (numpy) in and expand them into ``rbm``."""
        def flat(x):
            x = np.asarray(x)
            if self.is_complex:
                x = x.astype(np.complex128).reshape(-1)
                return torch.from_numpy(np.stack([x.real, x.imag], axis=1).reshape(-1).copy())
            return torch.from_numpy(np.asarray(x, dtype=np.float64).reshape(-1).copy())
        self.a.copy_(flat(a))
        self.b.copy_(flat(b))
        self.w.copy_(flat(w))
        nk_symm_expand(self, stream)

    def params_numpy(self):
        def un(t, shape):
            x = t.detach().cpu().numpy()
            if self.is_complex:
                x = x[0::2] + 1j * x[1::2]
            return x.reshape(shape)
        return un(self.a, (1,)), un(self.b, (self.alpha,)), un(self.w, (self.alpha, self.n))


def nk_symm_expand(s: RbmSymm, stream=None):
    _check(load_library().nk_symm_expand(s.struct(), s.rbm.struct(), _stream(stream)),
           "nk_symm_expand")


def sr_symm_scratch(s: RbmSymm, ns: int, device="cuda"):
    nb = load_library().nk_sr_symm_scratch_bytes(s.n, s.alpha, s.n_perm, int(s.is_complex), ns)
    return torch.empty(nb, dtype=torch.uint8, device=device)


def nk_sr_step_symm(s: RbmSymm, sigma, t, eloc, n_chains: int, diag_shift: float, lr: float,
                    n_cg: int, cg_rtol: float = 1e-12, prec=NK_PREC_FP32, weights=None,
                    scratch=None, info_out=None, stream=None):
    _require_gpu(sigma, t, eloc, weights, scratch, info_out)
    ns = sigma.shape[0]
    if scratch is None:
        scratch = sr_symm_scratch(s, ns, sigma.device)
    if info_out is None:
        info_out = torch.zeros(NK_INFO_LEN, dtype=torch.float64, device=sigma.device)
    _check(load_library().nk_sr_step_symm(
        s.struct(), s.rbm.struct(), _ptr(sigma), _ptr(t), _ptr(eloc), _ptr(weights), ns,
        n_chains, float(diag_shift), float(lr), int(n_cg), float(cg_rtol), prec, _ptr(scratch),
        scratch.numel(), _ptr(info_out), _stream(stream)), "nk_sr_step_symm")
    return info_out
