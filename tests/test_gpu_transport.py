"""Two-phase IMPES on the GPU (mrcm_impes) against the oracle's
(oracle.transport.impes): saturation after several Darcy cycles with the
skipping constant, element by element.  The transport step is explicit, so
the velocity's error (1e-10 FP64, 1e-8 mixed) carries into S at that level."""
import numpy as np
import pytest

import oracle
from oracle.transport import impes as oracle_impes
from synth.configs import small

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

from gpu_helpers import gpu_solver, rel_l2  # noqa: E402


@pytest.mark.parametrize("prec,tol", [("fp64", 1e-10), ("fp32_ir", 1e-8)])
@pytest.mark.parametrize("C_skip,n_steps", [(1, 3), (4, 10)])
def test_impes_matches_oracle(prec, tol, C_skip, n_steps):
    w = small(n=(12, 12, 4), edges=([6, 6], [6, 6], [4]), patch=((3, 2), (3, 2), (3, 3)), sigma=1.5, lam=4.0,
              wells="five_spot")
    prob = oracle.from_workload(w)
    S0 = np.zeros(prob.f.shape)
    S_ref, t_ref, solves = oracle_impes(prob, S0, 1.0, 5.0, 0.9, C_skip, n_steps)
    s = gpu_solver(w, prec, ir_max_sweeps=8, ir_tol=1e-13)
    K = torch.from_numpy(prob.K).cuda()
    f = torch.from_numpy(prob.f).cuda()
    S = torch.from_numpy(S0.copy()).cuda()
    t = s.impes(K, f, S, mu_w=1.0, mu_o=5.0, cfl=0.9, C_skip=C_skip, n_steps=n_steps)
    torch.cuda.synchronize()
    Sg = S.cpu().numpy()
    err = rel_l2(Sg.ravel(), S_ref.ravel())
    print(f"{prec} C={C_skip} steps={n_steps}: S rel err {err:.3e}  t {float(t.cpu()[0]):.6e} vs {t_ref:.6e}")
    assert err < tol
    assert abs(float(t.cpu()[0]) - t_ref) <= tol * t_ref
    assert Sg.min() >= -1e-14 and Sg.max() <= 1 + 1e-14
