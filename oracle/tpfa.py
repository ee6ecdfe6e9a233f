"""Two-point flux (TPFA) discretisation and the global fine-grid solver (ORACLE).

Test infrastructure only: the product path never imports this module.

Eq. aijk gives the 7-point stencil of Eq. darcy-discrete with coefficients
K~/h^2, K~ the harmonic mean 2 K_a K_b / (K_a + K_b) of the two cells' diagonal
permeability along the face normal.  Multiplying a cell's equation by its
volume gives the integrated (symmetric for any h) form used here: the face
transmissibility is T = A_f * K~ / h_n, A_f the face area and h_n the cell size
along the normal, and sum_faces T (p_c - p_nb) = f_c V_c.

Walls: the paper uses no-flow walls in all its experiments (Sec. "Numerical
setup").  For the closed-form tests, a wall may instead carry a Dirichlet
pressure g, imposed through the half-cell transmissibility 2 K A_f / h_n
(the boundary-face modification the paper defers to its reference; this is the
reading used throughout).

Eq. two_point recovers the face velocity u = -K~ (p_{i+1} - p_i) / h.
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp
import scipy.sparse.linalg as spla

from .problem import DIRICHLET, Problem


def harmonic(ka, kb):
    return 2.0 * ka * kb / (ka + kb)


def interior_T(prob: Problem, a):
    """Transmissibilities of interior faces normal to axis a.

    Returns an array of shape (nz, ny, nx) with the last index along ``a``
    shortened by one: entry [..., i, ...] is the face between cell i and i+1.
    """
    Ka = prob.K[a]
    ax = 2 - a  # array axis of grid axis a in (nz, ny, nx) layout
    lo = [slice(None)] * 3
    hi = [slice(None)] * 3
    lo[ax] = slice(0, -1)
    hi[ax] = slice(1, None)
    return prob.face_area(a) * harmonic(Ka[tuple(lo)], Ka[tuple(hi)]) / prob.h[a]


def fine_system(prob: Problem):
    """Global matrix A^h and right-hand side f^h of Eq. darcy-discrete-fine-grid."""
    nx, ny, nz = prob.n
    N = prob.ncells
    idx = np.arange(N).reshape(nz, ny, nx)
    rows, cols, vals = [], [], []
    diag = np.zeros(N)
    rhs = (prob.f * prob.cell_volume).ravel().copy()
    for a in range(3):
        ax = 2 - a
        T = interior_T(prob, a).ravel()
        lo = [slice(None)] * 3
        hi = [slice(None)] * 3
        lo[ax] = slice(0, -1)
        hi[ax] = slice(1, None)
        ia = idx[tuple(lo)].ravel()
        ib = idx[tuple(hi)].ravel()
        rows += [ia, ib]
        cols += [ib, ia]
        vals += [-T, -T]
        np.add.at(diag, ia, T)
        np.add.at(diag, ib, T)
        for side in (0, 1):
            if prob.bc_type[a][side] != DIRICHLET:
                continue
            wall = [slice(None)] * 3
            wall[ax] = 0 if side == 0 else prob.n[a] - 1
            cw = idx[tuple(wall)].ravel()
            Kw = prob.K[a][tuple(wall)].ravel()
            TD = prob.face_area(a) * 2.0 * Kw / prob.h[a]
            np.add.at(diag, cw, TD)
            np.add.at(rhs, cw, TD * prob.bc_value[a][side])
    rows.append(np.arange(N))
    cols.append(np.arange(N))
    vals.append(diag)
    A = sp.csr_matrix((np.concatenate(vals), (np.concatenate(rows), np.concatenate(cols))),
                      shape=(N, N))
    return A, rhs


def normalise_pressure(prob: Problem, p):
    """Remove the additive constant (zero volume-weighted mean) when no wall fixes p."""
    if prob.has_dirichlet():
        return p
    return p - p.mean()


def cell_face_velocity_fine(prob: Problem, p):
    """Per-cell face velocities (+axis component) from Eq. two_point.

    Returns u of shape (6, nz, ny, nx): rows (x-lo, x-hi, y-lo, y-hi, z-lo, z-hi).
    Interior faces carry -K~ (p_hi - p_lo) / h_n; no-flow walls carry 0; a
    Dirichlet wall carries the half-cell flux.
    """
    nx, ny, nz = prob.n
    P = p.reshape(nz, ny, nx)
    u = np.zeros((6, nz, ny, nx))
    for a in range(3):
        ax = 2 - a
        Ka = prob.K[a]
        lo = [slice(None)] * 3
        hi = [slice(None)] * 3
        lo[ax] = slice(0, -1)
        hi[ax] = slice(1, None)
        vel = -harmonic(Ka[tuple(lo)], Ka[tuple(hi)]) * (P[tuple(hi)] - P[tuple(lo)]) / prob.h[a]
        u[2 * a + 1][tuple(lo)] = vel
        u[2 * a][tuple(hi)] = vel
        for side in (0, 1):
            if prob.bc_type[a][side] != DIRICHLET:
                continue
            wall = [slice(None)] * 3
            wall[ax] = 0 if side == 0 else prob.n[a] - 1
            g = prob.bc_value[a][side]
            Kw = Ka[tuple(wall)]
            Pw = P[tuple(wall)]
            if side == 0:   # +axis velocity entering through the low wall
                u[2 * a][tuple(wall)] = -2.0 * Kw * (Pw - g) / prob.h[a]
            else:
                u[2 * a + 1][tuple(wall)] = -2.0 * Kw * (g - Pw) / prob.h[a]
    return u


def solve_fine(prob: Problem):
    """Global fine-grid TPFA solve by sparse direct LU (the paper's comparison system).

    With no-flow walls the pressure is fixed only up to a constant: cell 0's
    equation is replaced by p_0 = 0 and the result is shifted to zero mean.
    Returns (p, u) with u per cell as in ``cell_face_velocity_fine``.
    """
    A, rhs = fine_system(prob)
    if not prob.has_dirichlet():
        A = A.tolil()
        A[0, :] = 0.0
        A[0, 0] = 1.0
        A = A.tocsr()
        rhs = rhs.copy()
        rhs[0] = 0.0
    lu = spla.splu(A.tocsc())
    p = lu.solve(rhs)
    p = normalise_pressure(prob, p)
    return p, cell_face_velocity_fine(prob, p)
