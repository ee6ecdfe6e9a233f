"""Mean velocity post-processing of the MRCM solution (ORACLE - test infrastructure only).

The product path never imports this module.

Sec. "two-phase flow" of the paper, Eq. locprob_submean (the "Mean" method):
the MRCM velocity is conservative on the patch scale only (Eq. weakcont_f)
and two-valued on the fine faces of Gamma.  A single flux is defined on every
fine Gamma face as the average of the two sides' normal velocities,

    Ubar = (u^+ + u^-) / 2     (the +axis component, seen from either side),

which by Eq. weakcont_f carries the same mass through every patch as the
multiscale solution.  Each subdomain then solves its local Darcy problem
again with Neumann data: Ubar.n on its Gamma faces and the multiscale
solution's own normal velocity on the domain walls.  The discrete form is
the subdomain's TPFA system (Eq. aijk with harmonic means) with no Robin or
Dirichlet terms: for every cell

    sum_{interior faces} T (p_c - p_nb) = f_c V - sum_{boundary faces} q_out,

q_out = the prescribed outward flux (velocity times area).  The pure Neumann
matrix is singular; the data is compatible (the outward fluxes sum to the
sources), so one cell's pressure is fixed at 0 by removing its equation and
unknown.  The post-processed velocity is TPFA on the new pressure inside,
Ubar on Gamma, the given wall velocity on the walls; it is conservative cell
by cell on the fine scale.
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp
import scipy.sparse.linalg as spla

from .mrcm import local_problem
from .problem import Problem, build_bases


def mean_gamma_velocity(prob: Problem, u):
    """u with every fine Gamma face replaced by the mean of its two sides (both copies)."""
    sub = prob.sub_of_cell()
    out = u.copy()
    for a in range(3):
        ax = 2 - a
        lo = [slice(None)] * 3
        hi = [slice(None)] * 3
        lo[ax] = slice(0, -1)
        hi[ax] = slice(1, None)
        lo, hi = tuple(lo), tuple(hi)
        gamma = sub[lo] != sub[hi]                       # faces between two subdomains
        ubar = 0.5 * (u[2 * a + 1][lo] + u[2 * a][hi])
        up = out[2 * a + 1][lo]
        dn = out[2 * a][hi]
        up[gamma] = ubar[gamma]
        dn[gamma] = ubar[gamma]
        out[2 * a + 1][lo] = up
        out[2 * a][hi] = dn
    return out


def postprocess_mean(prob: Problem, u):
    """The post-processed velocity (6, nz, ny, nx) of Eq. locprob_submean."""
    ub = mean_gamma_velocity(prob, u)
    bases, sub_bases, face_basis = build_bases(prob)
    nx, ny, nz = prob.n
    uf = ub.reshape(6, -1)
    out = ub.copy()
    of = out.reshape(6, -1)
    V = prob.cell_volume
    for l in range(prob.nsub):
        lp = local_problem(prob, l, sub_bases, face_basis)      # for its cells and interior faces
        n = len(lp.cells)
        rows, cols, vals = [], [], []
        diag = np.zeros(n)
        for (c, d, a, T) in lp.interior:
            rows += [c, d]
            cols += [d, c]
            vals += [-T, -T]
            diag[c] += T
            diag[d] += T
        A = sp.csr_matrix((vals + list(diag), (rows + list(range(n)), cols + list(range(n)))), shape=(n, n))
        rhs = prob.f.ravel()[lp.cells] * V
        lo, size = lp.lo, lp.size
        for c, gc in enumerate(lp.cells):
            co = [gc % nx, (gc // nx) % ny, gc // (nx * ny)]
            for a in range(3):
                A_f = prob.face_area(a)
                if co[a] - lo[a] == size[a] - 1:            # the box face on the +a side
                    rhs[c] -= uf[2 * a + 1, gc] * A_f
                if co[a] - lo[a] == 0:                      # the box face on the -a side
                    rhs[c] += uf[2 * a, gc] * A_f
        # fix the pressure of local cell 0: drop its (implied) equation and unknown
        keep = np.arange(1, n)
        p = np.zeros(n)
        if n > 1:
            Ar = A[keep][:, keep].tocsc()
            p[1:] = spla.splu(Ar).solve(rhs[1:])
        for (c, d, a, T) in lp.interior:
            vel = T * (p[c] - p[d]) / prob.face_area(a)
            of[2 * a + 1, lp.cells[c]] = vel
            of[2 * a, lp.cells[d]] = vel
    return out
