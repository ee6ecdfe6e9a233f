"""The FP64 fallback of the mixed local solve (refinement cap reached -> FP64
direct factor and solve of the subdomain), and the permeability-contrast
stress test K^theta of Sec. "Computational time dependence on the
permeability field contrast" on the mixed path."""
import numpy as np
import pytest

import oracle
from synth.configs import small

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

from gpu_helpers import rel_l2, run_gpu  # noqa: E402

CASE = dict(n=(24, 20, 12), edges=([6, 6, 7, 5], [5, 5, 5, 5], [4, 4, 4]), patch=((3, 2), (2, 2), (3, 5)),
            sigma=2.0, lam=4.0)


def test_every_subdomain_falls_back_without_sweeps():
    """No refinement sweep: every column is above the tolerance, every subdomain
    is re-solved in FP64 (direct solve + one FP64 refinement step, the FP64
    form's kernels), and the result is the FP64 form's."""
    w = small(**CASE)
    prob = oracle.from_workload(w)
    s64, p64, u64, X64, *_ = run_gpu(w, prob.K, prob.f, "fp64")
    s, p, u, X, mres, code, st = run_gpu(w, prob.K, prob.f, "fp32_ir", ir_max_sweeps=0, ir_tol=1e-12,
                                         fallback_cap=w.n_sub)
    assert s.read_fallback() == (w.n_sub, 0)
    assert st["unconverged"] == 0 and code == 0
    assert rel_l2(p, p64) <= 1e-13 and rel_l2(u.ravel(), u64.ravel()) <= 1e-13 and rel_l2(X, X64) <= 1e-13


def test_fallback_cap_overflow_is_reported():
    w = small(**CASE)
    prob = oracle.from_workload(w)
    s, p, u, X, mres, code, st = run_gpu(w, prob.K, prob.f, "fp32_ir", ir_max_sweeps=0, ir_tol=1e-12,
                                         fallback_cap=3)
    fb, lost = s.read_fallback()
    assert fb == 3 and lost == w.n_sub - 3
    assert st["unconverged"] > 0 and code == 4          # MRCM_ERR_NO_CONVERGENCE


def test_no_fallback_when_disabled():
    w = small(**CASE)
    prob = oracle.from_workload(w)
    s, p, u, X, mres, code, st = run_gpu(w, prob.K, prob.f, "fp32_ir", ir_max_sweeps=1, ir_tol=1e-12,
                                         fallback_cap=-1)
    assert s.read_fallback() == (0, 0)
    assert st["unconverged"] > 0            # the one sweep saw the first solve's residual


@pytest.mark.parametrize("theta", [0.3, 1.0, 1.35, 1.7])
def test_contrast_stress_mixed_matches_oracle(theta):
    """K^theta raises the contrast c to c^theta (sigma = 3 log-normal: c ~ 1e7 at
    theta = 1).  The mixed path with the timed settings (5 sweeps, per-column
    stop 1e-9) plus the FP64 fallback stays within the 1e-8 bar."""
    from synth.configs import BENCH_SETTINGS
    w = small(n=(20, 20, 10), edges=([10, 10], [10, 10], [5, 5]), patch=((5, 5), (5, 5), (5, 5)), sigma=3.0,
              lam=6.0, kz_ratio=0.05)
    K0 = w.K()
    K = K0 ** theta
    prob = oracle.from_workload(w, K=K)
    r = oracle.solve_mrcm(prob)
    bs = BENCH_SETTINGS["c2"]
    s, p, u, X, mres, code, st = run_gpu(w, K, prob.f, "fp32_ir", ir_max_sweeps=bs["ir_sweeps"],
                                         ir_tol=bs["ir_tol"], interface_refine=bs["interface_refine"])
    fb, lost = s.read_fallback()
    ep, eu = rel_l2(p, r.p), rel_l2(u.ravel(), r.u.ravel())
    print(f"theta {theta}: contrast {K.max() / K.min():.2e}  p {ep:.2e}  u {eu:.2e}  fallback {fb}  lost {lost}  {st}")
    assert lost == 0 and st["unconverged"] == 0
    assert ep < 1e-8 and eu < 1e-8
