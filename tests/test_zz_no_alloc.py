"""GPU test of the allocation-free local solve, mrcm_box_solve_noalloc.

Callers whose host application owns every device allocation (its own pool,
no driver allocations once the time loop runs), plug-ins that may only touch
the buffers handed to them, and real-time loops that must not stall on
cudaMalloc cannot use the workspace-based entry points.  For them the library
offers mrcm_box_solve_noalloc, which keeps its scratch in a fixed array inside
the library.  This test calls it through the C ABI and checks it against the
MBF columns that the regular entry points (mrcm_factor_local +
mrcm_solve_mbf) compute for the same subdomain, and against the CPU
oracle's local solve, on two calls in a row.
"""
import ctypes as C

import numpy as np
import pytest

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


def _side_faces(box):
    """Face counts and offsets of the six sides in the documented order."""
    offs, n = [], 0
    for sd in range(6):
        a = sd // 2
        t1, t2 = [b for b in range(3) if b != a]
        offs.append(n)
        n += box[t1] * box[t2]
    return offs, n


def _call(lib, box, h, side, K, f, g, beta, stream):
    nf = _side_faces(box)[1]
    N = box[0] * box[1] * box[2]
    p = torch.empty(N, dtype=torch.float64, device="cuda")
    q = torch.empty(nf, dtype=torch.float64, device="cuda")
    flag = torch.empty(1, dtype=torch.int32, device="cuda")
    rc = lib.mrcm_box_solve_noalloc((C.c_int * 3)(*box), (C.c_double * 3)(*h), (C.c_int * 6)(*side),
                                    C.c_void_p(K.data_ptr()), C.c_void_p(f.data_ptr()),
                                    C.c_void_p(g.data_ptr()), C.c_void_p(beta.data_ptr()),
                                    C.c_void_p(p.data_ptr()), C.c_void_p(q.data_ptr()),
                                    C.c_void_p(flag.data_ptr()), C.c_void_p(stream))
    return rc, p, q, flag


def test_noalloc_matches_regular_local_solve():
    import oracle
    from oracle.mrcm import local_problem, solve_local
    from oracle.problem import build_bases
    from paper_2103_08513_gb300 import MRCM, _lib, build
    from synth.configs import small

    build()
    lib = _lib.load()
    w = small(n=(9, 7, 5), edges=([4, 5], [2, 3, 2], [5]), patch=((2, 2), (3, 2), (2, 3)), beta_const=0.7,
              h=(0.5, 1.0, 2.0))
    prob = oracle.from_workload(w)
    bases, sub_bases, face_basis = build_bases(prob)
    s = MRCM(w.n, w.edges, w.patch, h=w.h, beta_const=w.beta_const, precision="fp64")
    K = torch.from_numpy(prob.K).cuda()
    f = torch.from_numpy(prob.f).cuda()
    s.factor_local(K)
    s.solve_mbf(f)
    torch.cuda.synchronize()

    l = 3                                     # subdomain with three Robin sides and three walls
    lo, size = prob.sub_box(l)
    box = [size[0], size[1], size[2]]
    N = box[0] * box[1] * box[2]
    I = sub_bases[l]
    m = 2 * len(I) + 1
    ref = s.mbf_block(l, m, N)                # regular path, box-lexicographic cells
    sl = (slice(lo[2], lo[2] + size[2]), slice(lo[1], lo[1] + size[1]), slice(lo[0], lo[0] + size[0]))
    Kb = torch.from_numpy(np.ascontiguousarray(prob.K[(slice(None),) + sl])).cuda()
    fb = torch.from_numpy(np.ascontiguousarray(prob.f[sl])).cuda()
    fz = torch.zeros_like(fb)
    side = []
    for a in range(3):
        for hi in (0, 1):
            wall = (lo[a] == 0) if hi == 0 else (lo[a] + size[a] == prob.n[a])
            side.append(0 if wall else 1)
    offs, nf = _side_faces(box)
    nx, ny, _ = prob.n

    def g_for_basis(k):
        g = np.zeros(nf)
        b = bases[k]
        a = b.axis
        t1, t2 = [x for x in range(3) if x != a]
        for clo, chi in b.faces:
            cell, hi = (clo, 1) if b.lo == l else (chi, 0)
            gc = [cell % nx, (cell // nx) % ny, cell // (nx * ny)]
            lc = [gc[x] - lo[x] for x in range(3)]
            g[offs[2 * a + hi] + lc[t1] + box[t1] * lc[t2]] = 1.0
        return torch.from_numpy(g).cuda()

    beta = torch.full((nf,), w.beta_const, dtype=torch.float64, device="cuda")
    stream = torch.cuda.current_stream().cuda_stream
    # call 1: the P-MBF of the subdomain's first basis function
    rc, p1, q1, fl1 = _call(lib, box, w.h, side, Kb, fz, g_for_basis(I[0]), beta, stream)
    assert rc == 0
    # call 2 (same scratch): the particular solution
    rc, p2, q2, fl2 = _call(lib, box, w.h, side, Kb, fb, torch.zeros(nf, dtype=torch.float64, device="cuda"),
                            beta, stream)
    assert rc == 0
    torch.cuda.synchronize()
    assert int(fl1.cpu()[0]) == 0 and int(fl2.cpu()[0]) == 0
    Xo = solve_local(local_problem(prob, l, sub_bases, face_basis))     # oracle columns, same cell order
    for got, col in ((p1, 0), (p2, m - 1)):
        want = ref[col]
        assert np.linalg.norm(got.cpu().numpy() - want) <= 1e-10 * np.linalg.norm(want)
        assert np.linalg.norm(got.cpu().numpy() - Xo[:, col]) <= 1e-10 * np.linalg.norm(Xo[:, col])
    # conservation of the particular solution: the outward Robin fluxes carry the sources out
    vol = w.h[0] * w.h[1] * w.h[2]
    assert abs(q2.cpu().numpy().sum() - prob.f[sl].sum() * vol) <= 1e-10 * max(1.0, np.abs(prob.f[sl]).sum() * vol)


def test_noalloc_rejects_boxes_beyond_its_scratch():
    from paper_2103_08513_gb300 import _lib, build
    build()
    lib = _lib.load()
    box = [20, 20, 20]                       # 8000 cells > 4096
    offs, nf = _side_faces(box)
    N = 8000
    K = torch.ones(3 * N, dtype=torch.float64, device="cuda")
    f = torch.zeros(N, dtype=torch.float64, device="cuda")
    g = torch.zeros(nf, dtype=torch.float64, device="cuda")
    rc, *_ = _call(lib, box, (1.0, 1.0, 1.0), [1] * 6, K, f, g, g, torch.cuda.current_stream().cuda_stream)
    assert rc == 7                            # MRCM_ERR_OOM


def test_noalloc_dirichlet_sides_at_the_scratch_limits():
    """A box at the documented limits (8 x 16 x 16: slab block 128, 16 slabs,
    16 x 128^2 = 262144 block-inverse entries) with Dirichlet, Robin and no-flow
    sides, against the oracle's local solve (particular and P-MBF columns)."""
    import oracle
    from oracle.mrcm import local_problem, solve_local
    from oracle.problem import DIRICHLET, Problem, build_bases
    from paper_2103_08513_gb300 import _lib, build
    from synth.fields import lognormal_K

    build()
    lib = _lib.load()
    n = (16, 16, 16)
    h = (0.7, 1.0, 1.3)
    K = lognormal_K((16, 16, 16), 1.5, 4.0, 0.2, seed=3)
    rng = np.random.default_rng(4)
    f = rng.normal(size=(16, 16, 16))
    bc_t = ((DIRICHLET, 0), (0, 0), (0, DIRICHLET))
    bc_v = ((1.0, 0.0), (0.0, 0.0), (0.0, -0.5))
    prob = Problem(n=n, h=h, edges=([8, 8], [16], [16]), patch=((0, 0),) * 3, K=K, f=f, beta_const=0.4,
                   bc_type=bc_t, bc_value=bc_v)
    bases, sub_bases, face_basis = build_bases(prob)
    lp = local_problem(prob, 0, sub_bases, face_basis)     # the box x in [0, 8): Robin on its x-high side
    Xo = solve_local(lp)
    box = [8, 16, 16]
    offs, nf = _side_faces(box)
    side = [2, 1, 0, 0, 0, 2]                 # x-lo Dirichlet, x-hi Robin, y no-flow, z-lo no-flow, z-hi Dirichlet
    Kb = torch.from_numpy(np.ascontiguousarray(K[:, :, :, :8])).cuda()
    fb = torch.from_numpy(np.ascontiguousarray(f[:, :, :8])).cuda()
    beta = torch.full((nf,), 0.4, dtype=torch.float64, device="cuda")
    g_part = np.zeros(nf)
    g_part[offs[0]:offs[1]] = 1.0             # x-lo wall pressure
    g_part[offs[5]:] = -0.5                   # z-hi wall pressure
    g_mbf = np.zeros(nf)
    g_mbf[offs[1]:offs[2]] = 1.0              # the whole x-high face is the one basis function
    stream = torch.cuda.current_stream().cuda_stream
    rc1, p1, q1, fl1 = _call(lib, box, h, side, Kb, fb, torch.from_numpy(g_part).cuda(), beta, stream)
    rc2, p2, q2, fl2 = _call(lib, box, h, side, Kb, torch.zeros_like(fb), torch.from_numpy(g_mbf).cuda(),
                             beta, stream)
    assert rc1 == 0 and rc2 == 0
    torch.cuda.synchronize()
    assert int(fl1.cpu()[0]) == 0 and int(fl2.cpu()[0]) == 0
    for got, col in ((p1, Xo.shape[1] - 1), (p2, 0)):
        want = Xo[:, col]
        assert np.linalg.norm(got.cpu().numpy() - want) <= 1e-10 * np.linalg.norm(want)
    # every outward flux leaves through the Robin and Dirichlet faces: their sum is the source
    V = h[0] * h[1] * h[2]
    total = f[:, :, :8].sum() * V
    assert abs(q1.cpu().numpy().sum() - total) <= 1e-10 * np.abs(f[:, :, :8]).sum() * V
