"""Host-side checks of the C ABI (no GPU): exports, setup tables, errors.

mrcm_setup builds every table on the host, so the decomposition, the
interface space and the derived sizes can be compared bit-exactly with the
oracle's own enumeration without a GPU.
"""
import ctypes as C
import os
import re

import numpy as np
import pytest

import oracle
from oracle.problem import build_bases
from synth.configs import BETA_ALPHA_H_OVER_K, small, workload

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    from paper_2103_08513_gb300 import build
    from paper_2103_08513_gb300 import _lib
    build()
    return _lib.load()


def declared_symbols():
    hdr = open(os.path.join(ROOT, "include", "mrcm.h")).read()
    hdr = re.sub(r"/\*.*?\*/", "", hdr, flags=re.S)
    return sorted(set(re.findall(r"\b(mrcm_[a-z0-9_]+)\s*\(", hdr)))


def test_library_exports_every_declared_symbol(lib):
    syms = declared_symbols()
    assert "mrcm_setup" in syms and "mrcm_reconstruct" in syms
    for s in syms:
        assert hasattr(lib, s), s
    from paper_2103_08513_gb300._lib import SIGNATURES
    assert set(SIGNATURES) == set(syms)


def _cfg(w, precision=0):
    from paper_2103_08513_gb300._lib import mrcm_config
    cfg = mrcm_config()
    cfg.nx, cfg.ny, cfg.nz = w.n
    cfg.hx, cfg.hy, cfg.hz = w.h
    keep = []
    for a in range(3):
        arr = (C.c_int * len(w.edges[a]))(*w.edges[a])
        keep.append(arr)
        cfg.n_cuts[a] = len(w.edges[a])
        cfg.cuts[a] = C.cast(arr, C.POINTER(C.c_int))
        cfg.patch[a][0], cfg.patch[a][1] = w.patch[a]
    cfg.beta_mode = w.beta_mode
    cfg.alpha = w.alpha
    cfg.beta_const = w.beta_const
    cfg.precision = precision
    cfg.ir_max_sweeps = 4
    cfg.ir_tol = 1e-14
    return cfg, keep


def _setup(lib, w):
    cfg, keep = _cfg(w)
    h = C.c_void_p()
    rc = lib.mrcm_setup(C.byref(cfg), C.byref(h))
    return rc, h


WS = [
    small(),
    small(n=(9, 7, 5), edges=([4, 5], [2, 3, 2], [5]), patch=((2, 2), (3, 2), (2, 3))),
    small(n=(6, 6, 6), edges=([3, 3], [3, 3], [2, 4]), patch=((0, 0), (2, 0), (0, 2)),
          beta_mode=BETA_ALPHA_H_OVER_K),
    small(n=(13, 11, 7), edges=([4, 4, 5], [3, 5, 3], [2, 5]), patch=((2, 3), (4, 1), (3, 3))),
]


@pytest.mark.parametrize("w", WS + ["c1"])
def test_setup_tables_match_oracle(lib, w):
    from paper_2103_08513_gb300._lib import mrcm_sizes
    if isinstance(w, str):
        w = workload(w)
    nx, ny, nz = w.n
    prob = oracle.from_workload(w, K=np.ones((3, nz, ny, nx)), f=np.zeros((nz, ny, nx)))
    bases, sub_bases, _ = build_bases(prob)
    rc, h = _setup(lib, w)
    assert rc == 0, lib.mrcm_last_error(None)
    try:
        sz = mrcm_sizes()
        assert lib.mrcm_query_sizes(h, C.byref(sz)) == 0
        assert sz.n_basis == len(bases)
        assert sz.n_sub == prob.nsub
        assert sz.n_cells == prob.ncells
        assert sz.max_rhs == max(2 * len(I) + 1 for I in sub_bases)
        assert sz.total_rhs == sum(2 * len(I) + 1 for I in sub_bases)
        assert sz.n_faces == 2 * sum(len(b.faces) for b in bases)
        ax, lo, hi, nf = (C.c_int() for _ in range(4))
        for i, b in enumerate(bases):
            assert lib.mrcm_query_basis(h, i, C.byref(ax), C.byref(lo), C.byref(hi), C.byref(nf)) == 0
            assert (ax.value, lo.value, hi.value, nf.value) == (b.axis, b.lo, b.hi, len(b.faces))
    finally:
        lib.mrcm_destroy(h)


def test_c2_sizes(lib):
    from paper_2103_08513_gb300._lib import mrcm_sizes
    rc, h = _setup(lib, workload("c2"))
    assert rc == 0
    sz = mrcm_sizes()
    lib.mrcm_query_sizes(h, C.byref(sz))
    assert sz.n_sub == 2244 and sz.max_rhs == 33 and 2 * sz.n_basis == 32944
    # the emulated trailing updates: whole 32 x 32 tiles, each 8 warps x 36 slice pairs x 2
    # m16n8k16 BF16 MMAs; at C2 every step with a trailing block of >= 24 rows emulates, and the
    # tiles (at most 32 x 32 entries x 2 x 32 FP64-equivalent flops each) cover the update's work
    tile = 8 * 36 * 2 * (2 * 16 * 8 * 16)
    tiles = sz.ldl_update_tensor_flops / tile
    assert tiles == int(tiles) and tiles > 0
    assert tiles * 32 * 32 * 2 * 32 >= sz.ldl_update_flops
    lib.mrcm_destroy(h)


def test_front_sizes_cover_cluster_substitution(lib):
    """The parity case big_fronts has fronts with >= 128 eliminated dofs (the
    cluster substitution kernels) and > 128 boundary dofs (the back
    substitution split into row chunks); C2 has 528 and 768."""
    from paper_2103_08513_gb300._lib import mrcm_sizes
    from test_gpu_parity import CASES
    for w, lo_ne, lo_nb in ((small(**CASES["big_fronts"]), 128, 129), (workload("c2"), 528, 768)):
        rc, h = _setup(lib, w)
        assert rc == 0
        sz = mrcm_sizes()
        lib.mrcm_query_sizes(h, C.byref(sz))
        assert sz.max_front_ne >= lo_ne and sz.max_front_ne <= sz.max_front
        assert sz.max_front_nb >= lo_nb and sz.max_front_nb <= sz.max_front
        lib.mrcm_destroy(h)


def test_c3_uneven_setup(lib):
    from paper_2103_08513_gb300._lib import mrcm_sizes
    w = workload("c3")
    cfg, keep = _cfg(w, precision=1)
    h = C.c_void_p()
    assert lib.mrcm_setup(C.byref(cfg), C.byref(h)) == 0, lib.mrcm_last_error(None)
    sz = mrcm_sizes()
    lib.mrcm_query_sizes(h, C.byref(sz))
    assert sz.n_sub == w.n_sub and sz.max_block == 256
    lib.mrcm_destroy(h)
    # FP64 form: 16x16 slabs (b = 256) factor their packed triangle in a global slot
    cfg, keep = _cfg(w, precision=0)
    assert lib.mrcm_setup(C.byref(cfg), C.byref(h)) == 0, lib.mrcm_last_error(None)
    lib.mrcm_destroy(h)
    # slab blocks above 256 are refused
    big = small(n=(34, 17, 17), edges=([17, 17], [17], [17]))
    cfg, keep = _cfg(big, precision=1)
    assert lib.mrcm_setup(C.byref(cfg), C.byref(h)) == 8


def test_setup_rejects_bad_configs(lib):
    w = small()
    cfg, keep = _cfg(w)
    cfg.nx = 9          # edge list no longer sums to nx
    h = C.c_void_p()
    assert lib.mrcm_setup(C.byref(cfg), C.byref(h)) == 1
    assert b"does not sum" in lib.mrcm_last_error(None)
    cfg, keep = _cfg(small(n=(4, 4, 4), edges=([4], [4], [4])))
    assert lib.mrcm_setup(C.byref(cfg), C.byref(h)) == 1       # one subdomain, no-flow walls
    cfg, keep = _cfg(w)
    cfg.beta_const = -1.0
    assert lib.mrcm_setup(C.byref(cfg), C.byref(h)) == 1
    cfg, keep = _cfg(w)
    cfg.precision = 4
    assert lib.mrcm_setup(C.byref(cfg), C.byref(h)) == 1
    cfg, keep = _cfg(w)
    cfg.fallback_cap = -2
    assert lib.mrcm_setup(C.byref(cfg), C.byref(h)) == 1
    assert b"fallback_cap" in lib.mrcm_last_error(None)
    cfg, keep = _cfg(w)
    cfg.interface_refine = -2
    assert lib.mrcm_setup(C.byref(cfg), C.byref(h)) == 1
    assert b"interface_refine" in lib.mrcm_last_error(None)


def test_device_calls_reject_bad_arguments_without_gpu(lib):
    rc, h = _setup(lib, small())
    assert rc == 0
    # NULL pointers and misaligned workspaces are refused before any CUDA call
    assert lib.mrcm_factor_local(h, None, None, 0, None) == 1
    assert lib.mrcm_solve_mbf(h, C.c_void_p(256), C.c_void_p(256), None) == 9   # out of order
    assert lib.mrcm_factor_local(h, C.c_void_p(256), C.c_void_p(257), 1 << 30, None) == 1
    # the host-buffer solve: workspace, buffers, stream and workspace size are checked first
    ws_bytes, nif = C.c_size_t(), C.c_size_t()
    assert lib.mrcm_query_workspace(h, C.byref(ws_bytes), C.byref(nif)) == 0
    buf = [C.c_void_p(4096 * (q + 1)) for q in range(5)]
    ws, st = C.c_void_p(1 << 20), C.c_void_p(0x100)
    assert lib.mrcm_solve_host(h, *buf, None, None, ws_bytes.value, st, 0) == 1          # no workspace
    assert lib.mrcm_solve_host(h, *buf, None, C.c_void_p((1 << 20) + 8), ws_bytes.value, st, 0) == 1
    assert lib.mrcm_solve_host(h, None, *buf[1:], None, ws, ws_bytes.value, st, 0) == 1  # no K
    assert lib.mrcm_solve_host(h, *buf, None, ws, ws_bytes.value, None, 0) == 1          # default stream
    assert lib.mrcm_solve_host(h, *buf, None, ws, ws_bytes.value - 256, st, 0) == 7      # workspace too small
    lib.mrcm_destroy(h)


def test_query_tuning_reports_the_defaults_without_a_gpu(lib):
    w = small()
    cfg, keep = _cfg(w)
    h = C.c_void_p()
    assert lib.mrcm_setup(C.byref(cfg), C.byref(h)) == 0
    v = [C.c_int(-1) for _ in range(4)]
    assert lib.mrcm_query_tuning(h, *[C.byref(x) for x in v]) == 0
    assert [x.value for x in v] == [0, 0, 1, 0]
    assert lib.mrcm_query_tuning(h, None, None, None, None) == 0
    assert lib.mrcm_query_tuning(None, None, None, None, None) == 1
    lib.mrcm_destroy(h)


@pytest.mark.parametrize("box", [(65536, 65536, 65536), (4097, 1, 1), (1, 1, 1 << 20), (8, 16, 17), (12, 12, 12)])
def test_noalloc_rejects_oversized_boxes_before_any_device_work(lib, box):
    """Boxes beyond the fixed scratch (4096 cells, slab block <= 128, edge x block^2 <= 262144)
    return MRCM_ERR_OOM from the host-side checks, before a CUDA call is made; products of
    the edges that overflow 32 bits are not allowed to wrap past the checks."""
    dummy = (C.c_double * 4)()
    ptr = C.cast(dummy, C.c_void_p)
    flag = (C.c_int * 1)()
    rc = lib.mrcm_box_solve_noalloc((C.c_int * 3)(*box), (C.c_double * 3)(1.0, 1.0, 1.0), (C.c_int * 6)(*[1] * 6),
                                    ptr, ptr, ptr, ptr, ptr, ptr, C.cast(flag, C.c_void_p), None)
    assert rc == 7                           # MRCM_ERR_OOM


def test_local_ldl_cost_matches_oracle(lib):
    """The library's count of the paper's sparse local LDL^T (minimum degree,
    lowest-index ties) equals the oracle's, shape by shape and summed."""
    from oracle.symbolic import ldl_cost
    from paper_2103_08513_gb300 import MRCM
    w = small(n=(14, 9, 7), edges=([4, 10], [3, 6], [7]), patch=((2, 2), (3, 2), (2, 3)))
    s = MRCM(w.n, w.edges, w.patch, precision="fp32_ir", allocate=False)
    ff, sf = s.local_ldl_flops()
    prob = oracle.from_workload(w, K=np.ones((3,) + tuple(w.n[::-1])), f=np.zeros(w.n[::-1]))
    _, sub_bases, _ = build_bases(prob)
    ef = es = 0.0
    for l in range(prob.nsub):
        lo, size = prob.sub_box(l)
        fl, nz = ldl_cost(*size)
        ef += fl
        es += 4.0 * nz * (2 * len(sub_bases[l]) + 1)
    assert ff == ef and sf == es
    # a column of one cell (1-D chain): every vertex eliminated with one neighbour but the last
    fl, nz = ldl_cost(5, 1, 1)
    assert nz == 4 and fl == 4 * 1 * 4
