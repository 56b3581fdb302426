"""Host-side checks of the C ABI (no GPU needed): the library loads, exports
every entry point include/nk.h declares, and rejects bad arguments on the
host before touching the device."""
import ctypes as C
import os
import re

import numpy as np
import pytest

from paper_1904_00031_gb300 import build as nkbuild
from paper_1904_00031_gb300 import workloads as W

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    path = nkbuild.build()
    from paper_1904_00031_gb300 import nk
    return nk.load_library(path)


def declared_functions():
    src = open(os.path.join(ROOT, "include", "nk.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(nk_\w+)\s*\(", src)))


def test_header_declares_the_five_entry_points():
    names = declared_functions()
    for f in ("nk_rbm_logpsi", "nk_metropolis_sweep", "nk_local_energy", "nk_logderiv",
              "nk_sr_step"):
        assert f in names


def test_every_declared_symbol_is_exported(lib):
    missing = [f for f in declared_functions() if not hasattr(lib, f)]
    assert not missing, missing
    from paper_1904_00031_gb300 import nk
    assert set(nk.EXPORTS) <= set(declared_functions())


def test_status_strings_and_sizes(lib):
    assert lib.nk_status_string(0) == b"ok"
    assert lib.nk_status_string(2) == b"unsupported shape"
    assert lib.nk_rbm_workspace_bytes(0, 5, 0) == 0
    a = lib.nk_rbm_workspace_bytes(400, 1600, 1)
    b = lib.nk_rbm_workspace_bytes(400, 1600, 0)
    assert a > b > 400 * 1600 * 4
    assert lib.nk_sr_scratch_bytes(40, 80, 1, 16384) > 41 * 81 * 16 * 4
    # backward: one chunk of at most 16384 samples (tanh theta and the adjoint's
    # buffers), not all ns
    assert lib.nk_backward_scratch_bytes(40, 80, 1, 16384) > 16384 * 80 * 8
    assert lib.nk_backward_scratch_bytes(400, 1600, 1, 65536) == \
        lib.nk_backward_scratch_bytes(400, 1600, 1, 16384)
    assert lib.nk_backward_scratch_bytes(400, 1600, 1, 65536) < 65536 * 1600 * 8


@pytest.mark.parametrize("m, cplx, moves", [(1600, 1, 1600), (1600, 0, 1600), (20, 0, 10),
                                            (80, 1, 40), (33, 1, 65), (400, 0, 1)])
def test_local_energy_scratch_layout(lib, m, cplx, moves):
    """The move table ([m rounded to 32][moves rounded to 64] entries of 16 B complex
    or 8 B real, rounded to 256 B), then one FP64 complex factor per move and spin
    pattern."""
    mp = (m + 31) // 32 * 32
    nm_pad = (moves + 63) // 64 * 64
    table = (mp * nm_pad * (16 if cplx else 8) + 255) // 256 * 256
    assert lib.nk_local_energy_scratch_bytes(m, cplx, moves) == table + nm_pad * 4 * 16


def test_sr_batch_host_checks(lib):
    from paper_1904_00031_gb300 import nk
    assert lib.nk_sr_batch_desc_bytes(0) == 0
    one = lib.nk_sr_batch_desc_bytes(1)
    assert one >= 2 * 128 and one % 128 == 0  # two tensor maps, 128-B aligned records
    assert lib.nk_sr_batch_desc_bytes(5) == 5 * one
    items = (nk._SrBatchItem * 1)()
    buf = np.zeros(one, dtype=np.uint8)
    assert lib.nk_sr_batch_describe(C.cast(items, C.c_void_p), 0, 1,
                                    buf.ctypes.data_as(C.c_void_p), one) == 1
    # the batch runs on the tensor-core path only
    assert lib.nk_sr_batch_describe(C.cast(items, C.c_void_p), 1, 0,
                                    buf.ctypes.data_as(C.c_void_p), one) == 7
    # an item without an RBM is rejected before any device work
    assert lib.nk_sr_step_batch(C.cast(items, C.c_void_p), 1, None, 0.01, 0.01, 5, 0.0, 1,
                                None) == 1
    assert lib.nk_sr_step_batch(C.cast(items, C.c_void_p), 1, None, 0.01, 0.01, -1, 0.0, 1,
                                None) == 1


def test_status_query_host_checks(lib):
    # rejected on the host, before any device work
    assert lib.nk_query_status(None, None) == 1
    assert lib.nk_debug_bounded_wait(0, None) == 1
    assert lib.nk_debug_bounded_wait((1 << 20) + 1, None) == 1


def test_host_argument_validation(lib):
    from paper_1904_00031_gb300 import nk
    assert lib.nk_rbm_logpsi(None, None, 4, 0, None, None, None) == 1
    assert b"rbm is NULL" in lib.nk_last_error()
    r = nk._Rbm(0, 10, 0, 0, 0, 0, 0, 8, 8, 8, 256, 1 << 20)
    assert lib.nk_rbm_logpsi(C.byref(r), None, 4, 0, None, None, None) == 2
    r = nk._Rbm(10, 10, 0, 0, 0, 0, 0, 8, 8, 8, 256, 16)
    assert lib.nk_rbm_prepare(C.byref(r), None) == 2
    assert b"workspace" in lib.nk_last_error()
    r = nk._Rbm(10, 10, 0, 0, 0, 0, 0, 8, 8, 8, 256, 1 << 20)
    ch = nk._Chains(4, 64, 8, 1, 0)
    assert lib.nk_metropolis_sweep(C.byref(r), C.byref(ch), 0, None, None, 0, 1, 1, 8, None,
                                   None, 0, None) == 2
    ch = nk._Chains(4, 4, 8, 1, 0)
    assert lib.nk_metropolis_sweep(C.byref(r), C.byref(ch), 1, None, None, 0, 1, 1, 8, None,
                                   None, 0, None) == 1
    # real RBM: one row per site (flips) or bond (exchanges): (C, D) float2 and
    # the increment float per unit, then a 16-byte header (a_i - a_k)
    assert lib.nk_metropolis_scratch_bytes(400, 1600, 0, 0, 800) == 400 * (1600 * 12 + 16)
    assert lib.nk_metropolis_scratch_bytes(400, 1600, 0, 1, 800) == 800 * (1600 * 12 + 16)
    # complex RBM: pair rows of 512 * NU * WPC bytes followed by the row's complex
    # increments and header, sized for the larger of one warp per chain (NU = 64)
    # and two (NU = 26), per site (flips) or bond (exchanges), or the group
    # kernel's rows of 48 bytes per unit pair, sized for its widest padding (3
    # pairs per thread: 288 threads, 864 pairs), whichever is larger
    assert lib.nk_metropolis_scratch_bytes(400, 1600, 1, 0, 800) == max(
        400 * (512 * 64 + 1600 * 8 + 16), 400 * 48 * 864)
    assert lib.nk_metropolis_scratch_bytes(400, 1600, 1, 1, 800) == max(
        800 * (512 * 64 + 1600 * 8 + 16), 800 * 48 * 864)
    assert lib.nk_sr_step(C.byref(r), 8, 8, 8, None, 10, 3, 0.01, 0.01, 5, 0.0, 0, 256, 1 << 20,
                          8, None) == 2  # 10 samples do not split into 3 chains
    assert ch.counter == 0


def test_operator_compilation_sizes(lib):
    from paper_1904_00031_gb300 import nk
    ops = [W.ising(10, W.chain_bonds(10), h=1.0),
           W.heisenberg(40, W.chain_bonds(40), 1.0, True, W.sublattice(40)),
           W.j1j2(4, 1.0, 0.5, True)]
    sizes = []
    for op in ops:
        o = object.__new__(nk.Operator)
        o._site_idx = np.ascontiguousarray(op.site_idx, dtype=np.int32)
        o._site_mat = np.ascontiguousarray(np.stack([op.site_mat.real, op.site_mat.imag], -1))
        o._bond_i = np.ascontiguousarray(op.bond_i, dtype=np.int32)
        o._bond_k = np.ascontiguousarray(op.bond_k, dtype=np.int32)
        o._bond_mat = np.ascontiguousarray(np.stack([op.bond_mat.real, op.bond_mat.imag], -1))
        s = nk._Operator(op.n, op.n_site_terms, o._site_idx.ctypes.data, o._site_mat.ctypes.data,
                         op.n_bond_terms, 0, o._bond_i.ctypes.data, o._bond_k.ctypes.data,
                         o._bond_mat.ctypes.data)
        sizes.append(lib.nk_operator_bytes(C.byref(s)))
    # header 32 B; site 40 B, bond 72 B, move 80 B records (16-B padded blocks)
    assert sizes[0] == 32 + 400 + 720 + 800      # TFIM: 10 diag sites, 10 diag bonds, 10 flips
    assert sizes[1] == 32 + 0 + 2880 + 3200      # Heisenberg: 40 diag bonds, 40 pair moves
    assert sizes[2] == 32 + 0 + 64 * 72 + 64 * 80
    bad = nk._Operator(3, 0, None, None, 1, 0, np.array([0], np.int32).ctypes.data,
                       np.array([7], np.int32).ctypes.data, np.zeros(32).ctypes.data)
    assert lib.nk_operator_bytes(C.byref(bad)) == 0


def test_batch_calls_check_every_item_first(lib):
    """Items are checked on the host, all before any launch: a bad item is named,
    and the shape limits of the single calls apply (no device is touched here:
    every call below has a failing item)."""
    from paper_1904_00031_gb300 import nk

    def sweep_items(m, bad_second):
        n, cplx = 8, 1
        r = nk._Rbm(n, m, cplx, 0, 0, 0, 0, 256, 256, 256, 4096, lib.nk_rbm_workspace_bytes(n, m, cplx))
        ch = nk._Chains(16, 4, 4096, 1, 0, None)
        need = lib.nk_metropolis_scratch_bytes(n, m, cplx, 0, 0)
        good = nk._SweepItem(C.addressof(r), C.addressof(ch), 0, 0, None, None, 1, 2, 4096, None,
                             4096, need, None)
        bad = nk._SweepItem(C.addressof(r), C.addressof(ch), 0, 0, None, None, -1, 2, 4096, None,
                            4096, need, None)
        items = (nk._SweepItem * 2)(good, bad if bad_second else good)
        return items, (r, ch)

    # complex RBM, 4 chains per group: the group kernel holds up to 2304 hidden units
    items, keep = sweep_items(2304, True)     # the widest sampler layer passes its checks
    assert lib.nk_batch_sweep(C.cast(items, C.c_void_p), 2, None) == 1
    assert b"item 1" in lib.nk_last_error()
    items, keep = sweep_items(2305, True)     # one unit too many: item 0 is rejected
    assert lib.nk_batch_sweep(C.cast(items, C.c_void_p), 2, None) == 2
    assert b"item 0" in lib.nk_last_error()
    assert lib.nk_batch_sweep(None, 3, None) == 1
    assert lib.nk_batch_logpsi(None, -1, 0, None) == 1
    assert lib.nk_batch_local_energy(None, 2, None) == 1


def test_symm_host_checks(lib):
    from paper_1904_00031_gb300 import nk
    n, alpha, g = 9, 2, 9
    pa, pa_t = (alpha * g + 1) * (n + 1), (alpha + 1) * (n + 1)
    nb = lib.nk_symm_tables_bytes(n, alpha, g)
    assert nb >= 4 * (g * n + pa + pa_t + 1 + pa - 1) and nb % 256 == 0
    assert lib.nk_symm_tables_bytes(0, alpha, g) == 0
    assert lib.nk_symm_tables_bytes(400, 21, 400) == 0  # alpha n_perm above NK_MAX_M
    assert lib.nk_sr_symm_scratch_bytes(n, alpha, g, 1, 64) > lib.nk_sr_scratch_bytes(
        n, alpha * g, 1, 64)
    # a row that is not a permutation is rejected on the host, nothing copied
    perm = W.square_translations(3).copy()
    perm[4, 0] = perm[4, 1]
    assert lib.nk_symm_upload(perm.ctypes.data_as(C.c_void_p), n, alpha, g, C.c_void_p(256),
                              nb, None) == 1
    assert b"not a permutation" in lib.nk_last_error()
    # the untied RBM must be the expansion (m = alpha n_perm)
    s = nk._RbmSymm(n, alpha, g, 0, 8, 8, 8, 256, nb)
    r = nk._Rbm(n, alpha * g + 1, 0, 0, 0, 0, 0, 8, 8, 8, 256, 1 << 24)
    assert lib.nk_symm_expand(C.byref(s), C.byref(r), None) == 2
    r = nk._Rbm(n, alpha * g, 0, 0, 0, 0, 0, 8, 8, 8, 256, 1 << 24)
    s_small = nk._RbmSymm(n, alpha, g, 0, 8, 8, 8, 256, nb - 256)
    assert lib.nk_symm_expand(C.byref(s_small), C.byref(r), None) == 2
    assert b"tables" in lib.nk_last_error()
    assert lib.nk_sr_step_symm(C.byref(s), C.byref(r), 8, 8, 8, None, 10, 3, 0.01, 0.01, 5, 0.0,
                               0, 256, 1 << 24, 8, None) == 2  # 10 samples, 3 chains


def _sections(n, alpha, g):
    m = alpha * g
    pa, pa_t = (m + 1) * (n + 1), (alpha + 1) * (n + 1)
    sizes = [g * n, pa, pa_t + 1, max(pa - 1, 1)]
    offs, o = [], 0
    for k in sizes:
        offs.append(o // 4)
        o += -(-4 * k // 256) * 256
    return offs, sizes, o


def _aug_full(v, n, m):
    """(a, b, W) flat -> untied augmented [(m + 1)(n + 1)]."""
    out = np.zeros((m + 1, n + 1), dtype=v.dtype)
    out[:m, :n] = v[n + m:].reshape(m, n)
    out[:m, n] = v[n:n + m]
    out[m, :n] = v[:n]
    return out.reshape(-1)


def _aug_tied(x, n, alpha):
    """(at, bt, Wt) flat -> tied augmented [(alpha + 1)(n + 1)]."""
    out = np.zeros((alpha + 1, n + 1), dtype=x.dtype)
    out[:alpha, :n] = x[1 + alpha:].reshape(alpha, n)
    out[:alpha, n] = x[1:1 + alpha]
    out[alpha, 0] = x[0]
    return out.reshape(-1)


@pytest.mark.parametrize("lattice,alpha", [("square3", 2), ("chain7", 3), ("identity5", 2)])
def test_symm_tables_match_the_oracle_ties(lib, lattice, alpha):
    """The C++ tie and fold tables realise the oracle's expand (P x) and fold
    (P^T u) exactly, in the augmented layouts the SR kernels use."""
    from oracle import rbm_symm
    perm = {"square3": W.square_translations(3), "chain7": W.chain_translations(7),
            "identity5": np.arange(5, dtype=np.int32)[None, :]}[lattice]
    g, n = perm.shape
    m = alpha * g
    nb = lib.nk_symm_tables_bytes(n, alpha, g)
    offs, sizes, total = _sections(n, alpha, g)
    assert nb == total
    buf = np.zeros(nb // 4, dtype=np.int32)
    pc = np.ascontiguousarray(perm, dtype=np.int32)
    assert lib.nk_symm_build(pc.ctypes.data_as(C.c_void_p), n, alpha, g,
                             buf.ctypes.data_as(C.c_void_p), nb) == 0
    P, tie, off, idx = (buf[o:o + k] for o, k in zip(offs, sizes))
    assert np.array_equal(P.reshape(g, n), perm)
    rng = np.random.default_rng(4)
    x = rng.normal(size=1 + alpha + alpha * n) + 1j * rng.normal(size=1 + alpha + alpha * n)
    xt = _aug_tied(x, n, alpha)
    got = np.where(tie >= 0, xt[np.maximum(tie, 0)], 0)
    assert np.array_equal(got, _aug_full(rbm_symm.expand_vector(x, n, alpha, perm), n, m))
    u = rng.normal(size=n + m + n * m) + 1j * rng.normal(size=n + m + n * m)
    ua = _aug_full(u, n, m)
    assert np.all(np.diff(off) >= 0) and off[-1] == len(ua) - 1
    fold = np.array([ua[idx[off[q]:off[q + 1]]].sum() for q in range(len(off) - 1)])
    assert np.allclose(fold, _aug_tied(rbm_symm.fold(u, n, alpha, perm), n, alpha), atol=1e-12)
    for q in range(len(off) - 1):  # ascending lists: the fold's fixed summation order
        assert np.all(np.diff(idx[off[q]:off[q + 1]]) > 0)
