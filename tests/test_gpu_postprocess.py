"""Mean velocity post-processing on the GPU (mrcm_postprocess_velocity) against
the oracle's (oracle.postprocess.postprocess_mean), element by element.

Tolerances as for the solve: FP64 mode 1e-10 relative L2, mixed mode 1e-8; the
post-processed velocity is single-valued on Gamma (bit-identical copies) and
conservative on the fine scale.
"""
import numpy as np
import pytest

import oracle
from oracle.postprocess import postprocess_mean
from synth.configs import BETA_ALPHA_H_OVER_K, small

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

from gpu_helpers import gpu_solver, rel_l2  # noqa: E402

CASES = {
    "two_by_two": dict(),
    "ragged": dict(n=(9, 7, 5), edges=([4, 5], [2, 3, 2], [5]), patch=((2, 2), (3, 2), (2, 3))),
    "betaHK": dict(n=(6, 6, 6), edges=([3, 3], [3, 3], [2, 4]), patch=((0, 0), (2, 0), (0, 2)),
                   beta_mode=BETA_ALPHA_H_OVER_K, alpha=0.7),
    "aniso_h": dict(n=(8, 4, 4), edges=([2, 3, 3], [4], [2, 2]), patch=((1, 2), (1, 1), (3, 1)),
                    beta_const=0.3, h=(0.5, 1.0, 2.0)),
    "many_tiles": dict(n=(24, 20, 12), edges=([6, 6, 7, 5], [5, 5, 5, 5], [4, 4, 4]),
                       patch=((3, 2), (2, 2), (3, 5)), sigma=2.0, lam=4.0),
    "blocks_128": dict(n=(32, 16, 16), edges=([16, 16], [16], [8, 8]), patch=((0, 0), (0, 0), (0, 0)),
                       sigma=3.0, lam=8.0),
}


def _run(w, prob, precision):
    s = gpu_solver(w, precision, ir_max_sweeps=8, ir_tol=1e-13)
    K = torch.from_numpy(prob.K).cuda()
    f = torch.from_numpy(prob.f).cuda()
    p, u, X, mres = s.solve(K, f)
    u_ms = u.clone()
    up, mres_pp = s.postprocess_velocity(u_ms)
    torch.cuda.synchronize()
    code, st = s.read_status()
    return s, u_ms.cpu().numpy(), up.cpu().numpy(), float(mres_pp.cpu()[0]), st


@pytest.mark.parametrize("prec,tol", [("fp64", 1e-10), ("fp32_ir", 1e-8)])
@pytest.mark.parametrize("name", list(CASES))
def test_postprocess_matches_oracle(name, prec, tol):
    w = small(**CASES[name])
    prob = oracle.from_workload(w)
    r = oracle.solve_mrcm(prob)
    ref = postprocess_mean(prob, r.u)
    s, u_ms, up, mres, st = _run(w, prob, prec)
    assert st["not_spd"] == 0, st
    print(f"{name} {prec}: rel err {rel_l2(up.ravel(), ref.ravel()):.3e}, mass residual {mres:.3e}, "
          f"unconverged columns {st['unconverged']}")
    assert rel_l2(up.ravel(), ref.ravel()) < tol
    assert st["unconverged"] == 0                 # backward error <= 1e-13 after the FP64 steps
    # conservative on the fine scale, at the solve's accuracy
    fv = np.abs(prob.f).max() * prob.cell_volume
    assert mres <= (1e-11 if prec == "fp64" else 1e-7) * max(fv, 1.0)
    # single-valued on every Gamma face (both sides write the same mean)
    sub = prob.sub_of_cell()
    for a in range(3):
        ax = 2 - a
        lo = [slice(None)] * 3
        hi = [slice(None)] * 3
        lo[ax], hi[ax] = slice(0, -1), slice(1, None)
        lo, hi = tuple(lo), tuple(hi)
        g = sub[lo] != sub[hi]
        assert np.array_equal(up[2 * a + 1][lo][g], up[2 * a][hi][g])


def test_solve_after_postprocess_needs_a_new_factorisation():
    from paper_2103_08513_gb300._lib import MRCMError
    w = small(**CASES["ragged"])
    prob = oracle.from_workload(w)
    s, *_ = _run(w, prob, "fp64")
    with pytest.raises(MRCMError):
        s.solve_mbf(torch.from_numpy(prob.f).cuda())
    # a full solve starts from the factorisation again and gives the solve's result
    r = oracle.solve_mrcm(prob)
    p, u, X, _ = s.solve(torch.from_numpy(prob.K).cuda(), torch.from_numpy(prob.f).cuda())
    assert rel_l2(p.cpu().numpy().ravel(), r.p) < 1e-10
