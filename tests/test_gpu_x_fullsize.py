"""Full-size workloads in the benchmark's own launch configuration, against the oracle.

* C2 (60x220x85, 2244 subdomains): the mixed solve exactly as the benchmark
  times it (autotuned kernels, CUDA-graph replay, the FP64 refinement sweeps,
  per-column stop and interface refinement steps of BENCH_SETTINGS) against the whole staged oracle run over all host
  cores: p, u, X at 1e-8 relative L2, A^int and b^int entrywise.  The FP64 GPU
  form at 1e-10.
* C3 (uneven 8/12/16 blocks) and C5 (32768 blocks of 16x16x8 in
  memory-bounded waves): the oracle is too slow for every subdomain, so a
  seeded 1 % sample of subdomains gets full MBF parity (every column of the
  sample against the oracle's local solve), and the whole GPU result is
  checked by properties that hold at any size: the FP64 residual of the
  interface system at the GPU's X (every row but the F row that the pressure
  constant replaces), per-cell mass balance, and zero-mean p.

Tolerances: mixed mode 1e-8 (the metric's bar) on p, u and X; per-column MBF
parity 1e-8 of the column's largest entry; FP64 mode 1e-10; interface entries
relative to the largest entry.
"""
import os

import numpy as np
import pytest
import scipy.sparse as sp

import oracle
from oracle.mrcm import local_problem, solve_local
from oracle.problem import build_bases
from synth.configs import BENCH_SETTINGS, workload

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

from gpu_helpers import rel_l2  # noqa: E402

CORES = len(os.sched_getaffinity(0))


def _solver(w, precision, settings):
    from paper_2103_08513_gb300 import MRCM
    return MRCM(w.n, w.edges, w.patch, h=w.h, beta_mode=w.beta_mode, alpha=w.alpha, beta_const=w.beta_const,
                precision=precision, ir_max_sweeps=settings["ir_sweeps"], ir_tol=settings["ir_tol"],
                wave_bytes=int(settings["wave_gb"] * (1 << 30)), interface_refine=settings["interface_refine"])


def _bench_solve(s, K, f):
    """The benchmark's launch configuration: factor, autotune, then CUDA-graph replays."""
    Kd, fd = torch.from_numpy(K).cuda(), torch.from_numpy(f).cuda()
    st = torch.cuda.Stream()
    with torch.cuda.stream(st):
        s.factor_local(Kd, stream=st)
        s.autotune(fd, stream=st)
        out = s.outputs()
        for _ in range(2):                      # capture, then one replay
            s.solve(Kd, fd, out=out, stream=st, graph=True)
    torch.cuda.synchronize()
    X, p, u, mres = out
    return p.cpu().numpy().ravel(), u.cpu().numpy(), X.cpu().numpy(), float(mres.cpu()[0])


def _csr(s):
    rowptr, colidx, val, b = s.interface_csr()
    n = len(rowptr) - 1
    return sp.csr_matrix((val, colidx, rowptr), shape=(n, n)), b


def _entrywise(A, B, tol):
    d = (A - B).tocsr()
    scale = abs(B).max()
    return (abs(d).max() if d.nnz else 0.0) <= tol * scale


def test_c2_benchmarked_configuration_matches_oracle():
    w = workload("c2")
    K, f = w.K(), w.f()
    prob = oracle.from_workload(w, K=K, f=f)
    r = oracle.solve_mrcm(prob, keep=False, processes=CORES)
    # mixed precision, as timed
    s = _solver(w, "fp32_ir", BENCH_SETTINGS["c2"])
    p, u, X, mres = _bench_solve(s, K, f)
    code, st = s.read_status()
    print(f"C2 mixed status: {st}")
    assert st["not_spd"] == 0 and st["interface_zero_pivots"] == 0 and st["unconverged"] == 0
    ep, eu, ex = rel_l2(p, r.p), rel_l2(u.ravel(), r.u.ravel()), rel_l2(X, r.X)
    print(f"C2 mixed vs oracle: p {ep:.3e}  u {eu:.3e}  X {ex:.3e}  mass residual {mres:.3e}")
    assert ep < 1e-8 and eu < 1e-8 and ex < 1e-8
    A, b = _csr(s)
    assert _entrywise(A, r.A_int_raw, 1e-8)
    assert np.abs(b - r.b_int_raw).max() <= 1e-8 * np.abs(r.b_int_raw).max()
    # the FP64 GPU form
    s64 = _solver(w, "fp64", BENCH_SETTINGS["c2"])
    p, u, X, mres = _bench_solve(s64, K, f)
    ep, eu, ex = rel_l2(p, r.p), rel_l2(u.ravel(), r.u.ravel()), rel_l2(X, r.X)
    print(f"C2 fp64 vs oracle: p {ep:.3e}  u {eu:.3e}  X {ex:.3e}  mass residual {mres:.3e}")
    assert ep < 1e-10 and eu < 1e-10 and ex < 1e-10
    A, b = _csr(s64)
    assert _entrywise(A, r.A_int_raw, 1e-10)
    assert np.abs(b - r.b_int_raw).max() <= 1e-10 * np.abs(r.b_int_raw).max()
    assert mres <= 1e-9 * np.abs(prob.f).max() * prob.cell_volume


def _sampled_parity(name, frac=0.01, seed=0):
    w = workload(name)
    K, f = w.K(), w.f()
    settings = BENCH_SETTINGS[name]
    s = _solver(w, "fp32_ir", settings)
    p, u, X, mres = _bench_solve(s, K, f)
    code, st = s.read_status()
    print(f"{name} status: {st}")
    assert st["not_spd"] == 0 and st["interface_zero_pivots"] == 0
    prob = oracle.from_workload(w, K=K, f=f)
    bases, sub_bases, face_basis = build_bases(prob)
    rng = np.random.default_rng(seed)
    sample = np.sort(rng.choice(prob.nsub, size=max(1, int(round(frac * prob.nsub))), replace=False))
    worst = 0.0
    for l in sample:
        lp = local_problem(prob, int(l), sub_bases, face_basis)
        Xo = solve_local(lp)
        G = s.mbf_block(int(l), Xo.shape[1], Xo.shape[0]).T
        err = np.abs(G - Xo).max(axis=0) / np.maximum(np.abs(Xo).max(axis=0), 1e-300)
        worst = max(worst, float(err.max()))
    # the FP64 interface residual at the GPU's X.  With no-flow walls the F rows sum
    # to the (zero) total source only up to the MBFs' accuracy, so F row 0 is the
    # one the pressure constant replaces (pi^p_0 = 0): it is left out
    A, b = _csr(s)
    rows = np.arange(1, len(b))
    res = np.linalg.norm((A @ X - b)[rows]) / np.linalg.norm(b[rows])
    mbal = mres / (np.abs(prob.f).max() * prob.cell_volume)
    print(f"{name}: {len(sample)} sampled subdomains, worst MBF column error {worst:.3e}; "
          f"interface residual {res:.3e}; mass residual {mbal:.3e} of max |f| V; mean p {p.mean():.3e}")
    assert worst <= 1e-8
    assert res <= 1e-10
    assert mbal <= 1e-6
    assert abs(p.mean()) <= 1e-12 * np.abs(p).max()


def test_c3_uneven_sampled_mbf_parity_and_invariants():
    _sampled_parity("c3")


def test_c5_waves_sampled_mbf_parity_and_invariants():
    _sampled_parity("c5")
