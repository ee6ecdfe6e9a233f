"""mrcm_solve_host (the host-buffer entry point): its outputs equal the device
solve's bit for bit (same kernels, same order) and the oracle's at the mixed
bar, without and with graph capture."""
import numpy as np
import pytest

import oracle
from synth.configs import small

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

from gpu_helpers import rel_l2  # noqa: E402


@pytest.mark.parametrize("graph", [False, True])
def test_host_buffer_solve_equals_device_solve(graph):
    from paper_2103_08513_gb300 import MRCM
    w = small(n=(24, 20, 12), edges=([6, 6, 7, 5], [5, 5, 5, 5], [4, 4, 4]), patch=((3, 2), (2, 2), (3, 5)),
              sigma=2.0, lam=4.0)
    prob = oracle.from_workload(w)
    r = oracle.solve_mrcm(prob)
    s = MRCM(w.n, w.edges, w.patch, precision="fp32_ir", ir_max_sweeps=8, ir_tol=1e-13)
    st = torch.cuda.Stream()
    with torch.cuda.stream(st):
        Kd = torch.from_numpy(prob.K).cuda()
        fd = torch.from_numpy(prob.f).cuda()
        p_d, u_d, X_d, m_d = s.solve(Kd, fd, stream=st)
        p_d, u_d, X_d = p_d.cpu(), u_d.cpu(), X_d.cpu()
        Kh = torch.from_numpy(prob.K).pin_memory()
        fh = torch.from_numpy(prob.f).pin_memory()
        nx, ny, nz = w.n
        ph = torch.full((nz, ny, nx), np.nan, dtype=torch.float64).pin_memory()
        uh = torch.full((6, nz, ny, nx), np.nan, dtype=torch.float64).pin_memory()
        Xh = torch.full((max(s.n_interface, 1),), np.nan, dtype=torch.float64).pin_memory()
        mh = torch.full((1,), np.nan, dtype=torch.float64).pin_memory()
        for _ in range(2):                                  # graph: capture, then replay
            s.solve_host(Kh, fh, Xh, ph, uh, mh, stream=st, graph=graph)
        st.synchronize()
    assert torch.equal(ph, p_d) and torch.equal(uh, u_d) and torch.equal(Xh, X_d)
    assert np.isfinite(float(mh[0]))
    assert rel_l2(Xh.numpy(), r.X) < 1e-8
    assert rel_l2(uh.numpy().ravel(), r.u.ravel()) < 1e-8
