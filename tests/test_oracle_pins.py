"""Pins of the CPU oracle against facts fixed by the paper and by mathematics.

Each test checks the oracle against something other than itself: integers the
paper prints, closed-form solutions, the coincidence of the MRCM with the fine
TPFA solution when the interface spaces are the fine-face spaces
(Sec. "Domain decomposition and Darcy solvers"), a dense monolithic solve of
the same equations, and structural invariants that follow from the equations.
"""
import json
import os

import numpy as np
import pytest

import oracle
from oracle.mrcm import (assemble_interface, build_bases, local_problem, mbf_rhs,
                         solve_local, traces)
from oracle.problem import DIRICHLET, Problem
from synth.configs import BETA_ALPHA_H_OVER_K, small

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _prob(n=(8, 6, 4), edges=([4, 4], [3, 3], [2, 2]), patch=((2, 1), (2, 1), (2, 2)), **kw):
    return oracle.from_workload(small(n=n, edges=edges, patch=patch, **kw))


# ---------------------------------------------------------------- Eq. dof_PH
def test_interface_dof_counts_match_paper_tables():
    d = json.load(open(os.path.join(GOLDEN, "paper_interface_dofs.json")))
    exact = 0
    for row in d["rows"]:
        n_gamma = 2 * oracle.count_interface_dofs(row["Nd"], (1, 1, 1))
        # printed to 0.1K; three rows of Table wsc_res differ in the last digit
        assert abs(n_gamma / 1000.0 - row["printed_K"]) <= 0.1 + 1e-9, row
        exact += round(n_gamma / 1000.0, 1) == row["printed_K"]
    assert exact >= 11


def test_rhs_counts_match_paper():
    d = json.load(open(os.path.join(GOLDEN, "paper_interface_dofs.json")))
    for row in d["rhs_counts"]:
        assert oracle.interior_rhs_count(row["per_face_dofs"]) == row["nrhs"]


def test_basis_enumeration_matches_dof_formula():
    # uniform decomposition, patches dividing the faces: enumeration == Eq. dof_PH
    p = _prob(n=(12, 8, 6), edges=([4, 4, 4], [4, 4], [3, 3]), patch=((2, 3), (2, 1), (2, 2)))
    bases, sub_bases, _ = build_bases(p)
    # per-axis H/Hbar: x faces tangential (y, z) -> 4/2, 3/3; compare per orientation
    per_face = [(4 // 2) * (3 // 3), (4 // 2) * (3 // 1), (4 // 2) * (4 // 2)]
    expect = sum((p.Nd[a] - 1) * np.prod([p.Nd[b] for b in range(3) if b != a]) * per_face[a]
                 for a in range(3))
    assert len(bases) == expect
    # every basis touches exactly two subdomains, one on each side
    for b in bases:
        assert b.lo != b.hi


def test_c1_interface_size():
    from synth.configs import workload
    w = workload("c1")
    p = oracle.from_workload(w, K=np.ones((3, 8, 40, 40)), f=np.zeros((8, 40, 40)))
    bases, sub_bases, _ = build_bases(p)
    assert len(bases) == 352
    assert max(2 * len(I) + 1 for I in sub_bases) == 53


# ---------------------------------------------------------------- TPFA
def test_tpfa_series_resistance_closed_form():
    # 1-D column with Dirichlet ends: the flux is dp / sum(h/K) (series resistances),
    # which fixes the harmonic mean and the half-cell wall transmissibility.
    rng = np.random.default_rng(3)
    nx = 7
    kx = np.exp(rng.normal(size=nx))
    K = np.ones((3, 1, 1, nx))
    K[0, 0, 0, :] = kx
    h = (0.5, 2.0, 3.0)
    prob = Problem(n=(nx, 1, 1), h=h, edges=([nx], [1], [1]), patch=((0, 0),) * 3, K=K,
                   f=np.zeros((1, 1, nx)),
                   bc_type=((DIRICHLET, DIRICHLET), (0, 0), (0, 0)), bc_value=((2.0, -1.0), (0, 0), (0, 0)))
    p, u = oracle.solve_fine(prob)
    flux = 3.0 / np.sum(h[0] / kx)
    assert np.allclose(u[0].ravel(), flux, rtol=1e-13)
    assert np.allclose(u[1].ravel(), flux, rtol=1e-13)
    # pressure drops linearly in the accumulated resistance
    R = np.concatenate([[h[0] / (2 * kx[0])], h[0] / 2 * (1 / kx[:-1] + 1 / kx[1:])])
    assert np.allclose(p, 2.0 - flux * np.cumsum(R), rtol=0, atol=1e-13)


def test_tpfa_linear_pressure_exact_homogeneous():
    nx, ny, nz = 6, 5, 4
    K = np.empty((3, nz, ny, nx))
    K[0], K[1], K[2] = 2.0, 0.7, 0.1
    h = (1.0, 0.5, 2.0)
    prob = Problem(n=(nx, ny, nz), h=h, edges=([nx], [ny], [nz]), patch=((0, 0),) * 3, K=K,
                   f=np.zeros((nz, ny, nx)),
                   bc_type=((DIRICHLET, DIRICHLET), (0, 0), (0, 0)), bc_value=((1.0, 0.0), (0, 0), (0, 0)))
    p, u = oracle.solve_fine(prob)
    x = (np.arange(nx) + 0.5) * h[0]
    exact = 1.0 - x / (nx * h[0])
    assert np.allclose(p.reshape(nz, ny, nx), exact[None, None, :], atol=1e-13)
    assert np.allclose(u[0], 2.0 / (nx * h[0]), rtol=1e-12)


def test_fine_matrix_is_symmetric_m_matrix():
    prob = _prob()
    A, _ = oracle.fine_system(prob)
    A = A.toarray()
    assert np.allclose(A, A.T, rtol=0, atol=1e-14 * np.abs(A).max())
    off = A - np.diag(np.diag(A))
    assert (off <= 0).all()
    assert np.allclose(A.sum(axis=1), 0.0, atol=1e-13 * np.abs(A).max())


# ---------------------------------------------------------------- MRCM
CASES = [
    dict(),
    dict(n=(9, 7, 5), edges=([4, 5], [2, 3, 2], [5]), patch=((2, 2), (3, 2), (2, 3))),
    dict(n=(6, 6, 6), edges=([3, 3], [3, 3], [2, 4]), patch=((0, 0), (2, 0), (0, 2)),
         beta_mode=BETA_ALPHA_H_OVER_K, alpha=0.7),
    dict(n=(8, 4, 4), edges=([2, 3, 3], [4], [2, 2]), patch=((1, 2), (1, 1), (3, 1)), beta_const=0.3,
         h=(0.5, 1.0, 2.0)),
    # beta = alpha H / K with non-unit anisotropic h: H in length units, each side's own K
    dict(n=(6, 5, 4), edges=([2, 4], [3, 2], [1, 3]), patch=((2, 2), (3, 0), (1, 2)),
         beta_mode=BETA_ALPHA_H_OVER_K, alpha=1.3, h=(0.4, 1.7, 0.9), sigma=1.5),
]


@pytest.mark.parametrize("kw", CASES)
def test_staged_equals_monolithic(kw):
    prob = _prob(**kw)
    r = oracle.solve_mrcm(prob)
    pm, Xm = oracle.solve_monolithic(prob)
    scale = np.abs(pm).max()
    assert np.abs(r.p - pm).max() <= 1e-12 * scale
    assert np.abs(r.X - Xm).max() <= 1e-11 * max(1.0, np.abs(Xm).max())


@pytest.mark.parametrize("kw", CASES)
def test_fine_face_patches_reproduce_fine_solution(kw):
    kw = dict(kw)
    kw["patch"] = ((1, 1), (1, 1), (1, 1))
    prob = _prob(**kw)
    r = oracle.solve_mrcm(prob)
    pf, uf = oracle.solve_fine(prob)
    ep, ev = oracle.relative_errors(prob, r.p, r.u, pf, uf)
    assert ep < 1e-11 and ev < 1e-11


def test_coarse_patches_differ_from_fine():
    # the coincidence is specific to fine-face spaces: coarse patches give an O(1) error
    prob = _prob(patch=((0, 0), (0, 0), (0, 0)))
    r = oracle.solve_mrcm(prob)
    pf, uf = oracle.solve_fine(prob)
    ep, ev = oracle.relative_errors(prob, r.p, r.u, pf, uf)
    assert ep > 1e-4


def test_one_dimensional_column_is_exact():
    nx = 12
    rng = np.random.default_rng(5)
    K = np.exp(rng.normal(size=(3, 1, 1, nx)))
    f = np.zeros((1, 1, nx)); f[0, 0, 0] = 1.0; f[0, 0, -1] = -1.0
    prob = Problem(n=(nx, 1, 1), h=(1, 1, 1), edges=([3, 5, 1, 3], [1], [1]), patch=((0, 0),) * 3,
                   K=K, f=f)
    r = oracle.solve_mrcm(prob)
    pf, uf = oracle.solve_fine(prob)
    assert oracle.relative_errors(prob, r.p, r.u, pf, uf)[0] < 1e-12


def test_linear_pressure_exact_with_coarse_patches_normal_to_gradient():
    nx, ny, nz = 8, 6, 4
    K = np.empty((3, nz, ny, nx)); K[0], K[1], K[2] = 1.5, 0.4, 0.2
    prob = Problem(n=(nx, ny, nz), h=(1, 1, 1), edges=([2, 3, 3], [ny], [nz]), patch=((0, 0),) * 3,
                   K=K, f=np.zeros((nz, ny, nx)),
                   bc_type=((DIRICHLET, DIRICHLET), (0, 0), (0, 0)), bc_value=((1.0, 0.0), (0, 0), (0, 0)))
    r = oracle.solve_mrcm(prob)
    x = np.arange(nx) + 0.5
    assert np.allclose(r.p.reshape(nz, ny, nx), (1.0 - x / nx)[None, None, :], atol=1e-12)


@pytest.mark.parametrize("kw", CASES)
def test_interface_matrix_structure(kw):
    prob = _prob(**kw)
    r = oracle.solve_mrcm(prob)
    A = r.A_int_raw.toarray()
    NV = A.shape[0] // 2
    App, Apu, Aup, Auu = A[:NV, :NV], A[:NV, NV:], A[NV:, :NV], A[NV:, NV:]
    s = np.abs(A).max()
    assert np.abs(App - App.T).max() <= 1e-13 * s
    assert np.abs(Auu - Auu.T).max() <= 1e-13 * s
    assert np.abs(Aup + Apu.T).max() <= 1e-13 * s
    # pressure null vector: pi^p = 1, pi^u = 0
    z = np.concatenate([np.ones(NV), np.zeros(NV)])
    assert np.abs(A @ z).max() <= 1e-12 * s


@pytest.mark.parametrize("kw", CASES)
def test_mbf_invariants(kw):
    prob = _prob(**kw)
    bases, sub_bases, face_basis = build_bases(prob)
    for l in range(prob.nsub):
        lp = local_problem(prob, l, sub_bases, face_basis)
        X = solve_local(lp)
        m = len(lp.I)
        P = X[:, :m]
        # partition of unity (no-flow walls): sum_k P-MBF_k == 1, with zero traces
        assert np.allclose(P.sum(axis=1), 1.0, atol=1e-12)
        Q = traces(lp, X)
        assert np.abs(Q[:, :m].sum(axis=1)).max() < 1e-12
        # maximum principle
        assert P.min() > -1e-13 and P.max() < 1 + 1e-13
        # U-MBF = -beta s P-MBF when beta is constant over the patch
        if prob.beta_mode == 0:
            for c in range(m):
                s = [fc.s for fc in lp.faces if fc.col == c][0]
                assert np.allclose(X[:, m + c], -prob.beta_const * s * P[:, c], atol=1e-13)


@pytest.mark.parametrize("kw", CASES)
def test_conservation_and_weak_continuity(kw):
    prob = _prob(**kw)
    r = oracle.solve_mrcm(prob)
    assert r.mass_residual_max < 1e-12
    bases, _, _ = build_bases(prob)
    uf = r.u.reshape(6, -1)
    for b in bases:
        a = b.axis
        jump = sum(uf[2 * a + 1, clo] - uf[2 * a, chi] for clo, chi in b.faces)
        assert abs(jump) * prob.face_area(a) < 1e-11


@pytest.mark.parametrize("kw", CASES[:2])
def test_reconstruction_options_agree(kw):
    prob = _prob(**kw)
    r1 = oracle.solve_mrcm(prob, option=1)
    r2 = oracle.solve_mrcm(prob, option=2)
    assert np.abs(r1.p - r2.p).max() <= 1e-12 * np.abs(r1.p).max()
    assert np.abs(r1.u - r2.u).max() <= 1e-12 * np.abs(r1.u).max()


# ---------------------------------------------------------------- beta = alpha H / K (Eq. Robin_par)
def _two_by_two_closed_form(h, kL, kR, kyL, kyR, alpha, q):
    """Hand-derived MRCM solution of a 2 x 2 x 1 grid cut into two 1 x 2 x 1 subdomains.

    One x-interface with two fine faces forms a single patch (coarse patch).
    Cells: a = (0,0), b = (0,1) on the left, c = (1,0), d = (1,1) on the right;
    sources q = (q_a, q_b, q_c, q_d) with zero sum; every wall no-flow.

    Each local problem (Eq. localomegaint) with Robin data g has the solution
    g + w, where w solves the 2 x 2 system [[T_y + T_R, -T_y], [-T_y, T_y + T_R]] w = q
    (constants pass through the y-coupling).  Its sum and difference give
    w_a + w_b = (q_a + q_b) / T_R and w_a - w_b = (q_a - q_b) / (2 T_y + T_R).
    The F row (Eq. weakcont_f) is the zero total source (pinned by pi^p = 0);
    the U row (Eq. weakcont_p) with Q_L = q_a + q_b = -Q_R reads
    beta_L (Q_L - 2 A_x pi^u) + beta_R (Q_L - 2 A_x pi^u) = 0, so
    pi^u = Q_L / (2 A_x).  Robin data: g_L = pi^p - beta_L pi^u (s = +1),
    g_R = pi^p + beta_R pi^u (s = -1).  beta_side = alpha H / K_x of the side's
    own cell, H = one cell's length along x (reading R3).
    """
    hx, hy, hz = h
    Ax = hy * hz
    bL, bR = alpha * hx / kL, alpha * hx / kR
    TRL, TRR = Ax / (hx / (2 * kL) + bL), Ax / (hx / (2 * kR) + bR)
    TyL, TyR = hx * hz * kyL / hy, hx * hz * kyR / hy
    qa, qb, qc, qd = q

    def local(Ty, TR, q1, q2):
        S = (q1 + q2) / TR
        D = (q1 - q2) / (2 * Ty + TR)
        return (S + D) / 2, (S - D) / 2

    wa, wb = local(TyL, TRL, qa, qb)
    wc, wd = local(TyR, TRR, qc, qd)
    piu = (qa + qb) / (2 * Ax)
    gL, gR = -bL * piu, bR * piu
    p = np.array([gL + wa, gR + wc, gL + wb, gR + wd])    # global order: x fastest
    return p - p.mean(), np.array([0.0, piu]), (TRL * wa / Ax, TRL * wb / Ax)


def test_beta_alpha_H_over_K_closed_form():
    """beta = alpha H / K changes the answer, and the oracle matches the hand solution.

    Non-unit anisotropic h (H in length units differs from H in cells), K_x
    differing across Gamma (the side's own K differs from the neighbour's), and
    a two-face patch (the Robin data is not the fine-face trace).
    """
    h = (0.5, 2.0, 0.7)
    kL, kR, kyL, kyR, alpha = 2.0, 0.25, 0.6, 3.0, 0.8
    q = (1.0, 0.0, 0.0, -1.0)
    V = h[0] * h[1] * h[2]
    K = np.empty((3, 1, 2, 2))
    K[0, 0, :, 0], K[0, 0, :, 1] = kL, kR
    K[1, 0, :, 0], K[1, 0, :, 1] = kyL, kyR
    K[2] = 1.0
    f = np.array([[[q[0], q[2]], [q[1], q[3]]]]) / V     # [z][y][x]: a, c on y = 0; b, d on y = 1
    prob = Problem(n=(2, 2, 1), h=h, edges=([1, 1], [2], [1]), patch=((0, 0),) * 3, K=K, f=f,
                   beta_mode=1, alpha=alpha)
    p_ref, X_ref, (va, vb) = _two_by_two_closed_form(h, kL, kR, kyL, kyR, alpha, q)
    r = oracle.solve_mrcm(prob)
    assert np.abs(r.p - p_ref).max() <= 1e-12 * np.abs(p_ref).max()
    assert np.abs(r.X - X_ref).max() <= 1e-12 * np.abs(X_ref).max()
    # Gamma velocities seen from the left cells (x-high faces of a and b)
    assert abs(r.u[1, 0, 0, 0] - va) <= 1e-12 * abs(va)
    assert abs(r.u[1, 0, 1, 0] - vb) <= 1e-12 * abs(vb)
    # the monolithic assembly (written separately) agrees
    pm, Xm = oracle.solve_monolithic(prob)
    assert np.abs(pm - p_ref).max() <= 1e-12 * np.abs(p_ref).max()
    # beta matters here: the answer with a constant beta is different
    p_c, _, _ = _two_by_two_closed_form(h, kL, kR, kyL, kyR, 0.0, q)
    assert np.abs(p_c - p_ref).max() > 1e-2 * np.abs(p_ref).max()


def test_relative_errors_weighting():
    """Eq. of Sec. "Numerical setup": volume-weighted L2 pressure error and the
    K^-1-weighted velocity error with the trapezoidal rule per cell."""
    rng = np.random.default_rng(11)
    n = (3, 2, 2)
    h = (0.5, 1.5, 2.0)
    V = h[0] * h[1] * h[2]
    K = np.exp(rng.normal(size=(3, 2, 2, 3)))
    prob = Problem(n=n, h=h, edges=([3], [2], [2]), patch=((0, 0),) * 3, K=K, f=np.zeros((2, 2, 3)))
    p_ref = np.ones(12)
    p = p_ref.copy()
    p[5] += 0.3
    u_ref = np.ones((6, 2, 2, 3))
    u = u_ref.copy()
    u[3, 1, 0, 2] += 0.25                          # y-high face of cell (2, 0, 1)
    ep, ev = oracle.relative_errors(prob, p, u, p_ref, u_ref)
    assert abs(ep - np.sqrt(V * 0.09) / np.sqrt(12 * V)) <= 1e-14
    num = 0.5 * V * 0.25 ** 2 / K[1, 1, 0, 2]
    den = sum(2 * 0.5 * V * (1.0 / K[a]).sum() for a in range(3))     # two faces per axis and cell
    assert abs(ev - np.sqrt(num / den)) <= 1e-14


def test_pooled_oracle_equals_serial():
    """The worker pool changes where the per-subdomain work runs, not what it computes."""
    prob = _prob(**CASES[1])
    r1 = oracle.solve_mrcm(prob)
    r2 = oracle.solve_mrcm(prob, processes=2)
    assert np.array_equal(r1.p, r2.p) and np.array_equal(r1.u, r2.u) and np.array_equal(r1.X, r2.X)
    assert (r1.A_int_raw != r2.A_int_raw).nnz == 0
