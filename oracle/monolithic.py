"""Monolithic form of the MRCM, solved densely on tiny grids (ORACLE).

Test infrastructure only: the product path never imports this module.

The MRCM solution is the solution of one linear system whose unknowns are all
subdomains' cell pressures together with the interface coefficients
(pi^p, pi^u):

* every subdomain's TPFA equations with Robin data g = P_H - beta s U_H left as
  unknowns (Eq. localomegapar + Eq. localomegaint combined, since the local
  solution is the sum of the particular solution and the MBF part);
* the weak flux condition Eq. weakcont_f, one row per basis function;
* the weak pressure condition Eq. weakcont_p, one row per basis function.

Solving it directly (numpy.linalg.solve on a dense matrix) needs no MBFs, no
interface matrix and no superposition, so it checks the staged algorithm
independently.  The same pinning as the staged form (F row 0 replaced by
pi^p_0 = 0 when the walls leave p free) makes it non-singular.
"""
from __future__ import annotations

import numpy as np

from .mrcm import local_problem
from .problem import Problem, build_bases


def solve_monolithic(prob: Problem):
    bases, sub_bases, face_basis = build_bases(prob)
    NV = len(bases)
    locs = [local_problem(prob, l, sub_bases, face_basis) for l in range(prob.nsub)]
    offs = np.cumsum([0] + [lp.A.shape[0] for lp in locs])
    ncell = int(offs[-1])
    n = ncell + 2 * NV
    M = np.zeros((n, n))
    r = np.zeros(n)
    for lp, o in zip(locs, offs[:-1]):
        nl = lp.A.shape[0]
        M[o:o + nl, o:o + nl] = lp.A.toarray()
        r[o:o + nl] = lp.rhs_part
        for fc in lp.faces:
            row = o + fc.local_cell
            # A p - T_R g = rhs, g = pi^p - beta s pi^u
            M[row, ncell + fc.basis] -= fc.T_R
            M[row, ncell + NV + fc.basis] += fc.T_R * fc.beta * fc.s
            # q_f = T_R (p_c - pi^p + beta s pi^u)
            fr = ncell + fc.basis
            M[fr, row] += fc.T_R
            M[fr, ncell + fc.basis] -= fc.T_R
            M[fr, ncell + NV + fc.basis] += fc.T_R * fc.beta * fc.s
            # beta (s q_f - A_f pi^u)
            ur = ncell + NV + fc.basis
            M[ur, row] += fc.beta * fc.s * fc.T_R
            M[ur, ncell + fc.basis] -= fc.beta * fc.s * fc.T_R
            M[ur, ncell + NV + fc.basis] += fc.beta * fc.s * fc.T_R * fc.beta * fc.s
            M[ur, ncell + NV + fc.basis] -= fc.beta * fc.area
    if not prob.has_dirichlet() and NV > 0:
        M[ncell, :] = 0.0
        M[ncell, ncell] = 1.0
        r[ncell] = 0.0
    sol = np.linalg.solve(M, r)
    p = np.zeros(prob.ncells)
    for lp, o in zip(locs, offs[:-1]):
        p[lp.cells] = sol[o:o + lp.A.shape[0]]
    if not prob.has_dirichlet():
        p = p - p.mean()
    return p, sol[ncell:]
