"""Monolithic form of the MRCM, assembled on its own and solved densely (ORACLE).

Test infrastructure only: the product path never imports this module.

The MRCM solution is the solution of one linear system whose unknowns are the
pressures of all cells together with the interface coefficients
(pi^p, pi^u):

* the TPFA balance of every cell (Eq. darcy-discrete with the coefficients of
  Eq. aijk, times the cell volume), in which a face between two cells of the
  same subdomain couples them, a face on Gamma carries the Robin condition
  -beta u.n + p = g of Eq. localomegaint with g = P_H - beta s U_H left as
  unknowns, and a wall is no-flow or Dirichlet;
* the weak flux condition Eq. weakcont_f, one row per basis function;
* the weak pressure condition Eq. weakcont_p, one row per basis function.

This module assembles that system directly from the global grid: it walks
over every fine face once, in global cell numbering, and needs neither the
staged oracle's local problems nor its MBFs, interface matrix or
superposition.  The only thing it shares with the staged form is the
enumeration of the patch basis (``build_bases``, pinned by Eq. dof_PH).
Solving it with numpy.linalg.solve therefore checks the staged algorithm's
assembly (TPFA, Robin transmissibility, beta, the signs s) as well as its
superposition.  When the walls leave p free, F row 0 is replaced by
pi^p_0 = 0 as in the staged form.
"""
from __future__ import annotations

import numpy as np

from .problem import DIRICHLET, Problem, build_bases


def _robin_beta(prob: Problem, sub_edge_cells, a, Kn):
    """beta of Eq. Robin_par on one side of a Gamma face (reading: the side's own cell)."""
    if prob.beta_mode == 0:
        return prob.beta_const
    H = sub_edge_cells * prob.h[a]          # the subdomain's extent along the normal, in length units
    return prob.alpha * H / Kn


def assemble_monolithic(prob: Problem):
    """Dense matrix and right-hand side of the monolithic MRCM system.

    Unknown order: p (global cells, x fastest), then pi^p_0..pi^p_{NV-1}, then
    pi^u_0..pi^u_{NV-1}.
    """
    nx, ny, nz = prob.n
    ncell = prob.ncells
    bases, _, face_basis = build_bases(prob)
    NV = len(bases)
    n = ncell + 2 * NV
    M = np.zeros((n, n))
    r = np.zeros(n)
    V = prob.cell_volume
    sub = prob.sub_of_cell()                              # (nz, ny, nx)
    # per-axis subdomain index of every cell coordinate, and that subdomain's edge
    sub_axis = [np.repeat(np.arange(prob.Nd[a]), prob.edges[a]) for a in range(3)]
    edge_of = [np.asarray(prob.edges[a])[sub_axis[a]] for a in range(3)]
    r[:ncell] = prob.f.ravel() * V
    PP = lambda k: ncell + k               # noqa: E731  column of pi^p_k
    UU = lambda k: ncell + NV + k          # noqa: E731  column of pi^u_k

    for k in range(nz):
        for j in range(ny):
            for i in range(nx):
                ijk = (i, j, k)
                c = i + nx * (j + ny * k)
                for a in range(3):
                    A_f = prob.face_area(a)
                    h_a = prob.h[a]
                    Kc = prob.K[a, k, j, i]
                    # the face on the +a side of cell c
                    if ijk[a] + 1 < prob.n[a]:
                        nb = list(ijk)
                        nb[a] += 1
                        d = nb[0] + nx * (nb[1] + ny * nb[2])
                        Kd = prob.K[a, nb[2], nb[1], nb[0]]
                        if sub[k, j, i] == sub[nb[2], nb[1], nb[0]]:
                            # TPFA face inside one subdomain: T = A_f K~ / h_a, K~ the harmonic mean
                            T = A_f * (2.0 * Kc * Kd / (Kc + Kd)) / h_a
                            M[c, c] += T
                            M[d, d] += T
                            M[c, d] -= T
                            M[d, c] -= T
                        else:
                            # Gamma face: cell c is on the lower side (s = +1), d on the upper (s = -1)
                            kb = face_basis[(a, c)]
                            for cell, s, Kn, coord in ((c, +1, Kc, ijk[a]), (d, -1, Kd, nb[a])):
                                beta = _robin_beta(prob, int(edge_of[a][coord]), a, Kn)
                                TR = A_f / (h_a / (2.0 * Kn) + beta)
                                # cell balance: + TR (p_c - g), g = pi^p - beta s pi^u
                                M[cell, cell] += TR
                                M[cell, PP(kb)] -= TR
                                M[cell, UU(kb)] += TR * beta * s
                                # F row kb: + q_f = TR (p_c - g)
                                M[PP(kb), cell] += TR
                                M[PP(kb), PP(kb)] -= TR
                                M[PP(kb), UU(kb)] += TR * beta * s
                                # U row kb: + beta (s q_f - A_f pi^u)
                                M[UU(kb), cell] += beta * s * TR
                                M[UU(kb), PP(kb)] -= beta * s * TR
                                M[UU(kb), UU(kb)] += beta * s * TR * beta * s - beta * A_f
                    # walls
                    for side, at_wall in ((0, ijk[a] == 0), (1, ijk[a] == prob.n[a] - 1)):
                        if at_wall and prob.bc_type[a][side] == DIRICHLET:
                            TD = 2.0 * Kc * A_f / h_a
                            M[c, c] += TD
                            r[c] += TD * prob.bc_value[a][side]
    if not prob.has_dirichlet() and NV > 0:
        M[ncell, :] = 0.0
        M[ncell, ncell] = 1.0
        r[ncell] = 0.0
    return M, r, NV


def solve_monolithic(prob: Problem):
    """Solve the monolithic system densely; returns (p normalised, X = (pi^p, pi^u))."""
    M, r, NV = assemble_monolithic(prob)
    sol = np.linalg.solve(M, r)
    ncell = prob.ncells
    p = sol[:ncell].copy()
    if not prob.has_dirichlet():
        p = p - p.mean()
    return p, sol[ncell:]
