"""Two-phase IMPES transport with a skipping constant (ORACLE - test infrastructure only).

The product path never imports this module.

Model (Sec. "Domain decomposition and Darcy solvers", Eq. Buckley-Leverett,
Eq. darcy with the total mobility): water saturation S, time rescaled by the
porosity,

    S_t + div(phi(S) u) = source,     u = -lambda(S) K grad p,   div u = f,
    lambda(S) = S^2 / mu_w + (1 - S)^2 / mu_o,
    phi(S)    = M S^2 / (M S^2 + (1 - S)^2),   M = mu_o / mu_w.

Transport step (Sec. "The fine grid transport solver", Eq. transporte_discreto
with the upwind fractional flow of Eq. flux_disc_up).  The printed update is
garbled in its signs; the reading used here is the conservative upwind
finite-volume step written with the compensation term of the paper (the
divergence of the frozen velocity is removed with phi of the cell itself,
which keeps the scheme monotone):

    S_c^{n+1} = S_c^n - (dt / V) sum_faces (phi_f - phi(S_c^n)) q_f
                + dt max(f_c, 0) (1 - phi(S_c^n)),

q_f the outward integrated flux of the (post-processed) velocity through
face f, phi_f = phi of the upwind cell (the cell itself when q_f >= 0, the
neighbour otherwise; no flux through walls), injection wells (f > 0) bring
pure water and production wells take out the local mixture (their term
vanishes in this form).

Time step (Eq. CFL): dt = cfl * min(h) / (phi'_max * max_faces |u|), with
phi'_max the maximum of phi'(S) = 2 M S (1 - S) / (M S^2 + (1 - S)^2)^2 over
S = k / 1000, k = 0..1000 (a bound of phi' over [0, 1], so the condition
holds for every saturation the step can meet).

IMPES with skipping constant C (Alg. overview-code): every C transport steps
the Darcy problem is solved again with K_eff = lambda(S) K (the MRCM solve and
its mean velocity post-processing, Eq. locprob_submean), and the velocity and
time step stay frozen in between.
"""
from __future__ import annotations

import numpy as np

from . import mrcm as _mrcm
from .postprocess import postprocess_mean
from .problem import Problem


def mobility(S, mu_w, mu_o):
    return S ** 2 / mu_w + (1.0 - S) ** 2 / mu_o


def frac_flow(S, mu_w, mu_o):
    M = mu_o / mu_w
    return M * S ** 2 / (M * S ** 2 + (1.0 - S) ** 2)


def frac_flow_slope_max(mu_w, mu_o):
    M = mu_o / mu_w
    S = np.arange(1001) / 1000.0
    d = 2.0 * M * S * (1.0 - S) / (M * S ** 2 + (1.0 - S) ** 2) ** 2
    return float(d.max())


def cfl_dt(prob: Problem, u, mu_w, mu_o, cfl):
    umax = float(np.abs(u).max())
    if umax == 0.0:
        return 0.0
    return cfl * min(prob.h) / (frac_flow_slope_max(mu_w, mu_o) * umax)


def transport_step(prob: Problem, S, u, dt, mu_w, mu_o):
    """One explicit upwind step; S (nz, ny, nx), u (6, nz, ny, nx) single-valued on every face."""
    phi = frac_flow(S, mu_w, mu_o)
    V = prob.cell_volume
    acc = np.zeros_like(S)
    for a in range(3):
        ax = 2 - a
        A = prob.face_area(a)
        lo = [slice(None)] * 3
        hi = [slice(None)] * 3
        lo[ax], hi[ax] = slice(0, -1), slice(1, None)
        lo, hi = tuple(lo), tuple(hi)
        q = u[2 * a + 1][lo] * A                 # flux from the low cell into the high cell
        up = np.where(q >= 0.0, phi[lo], phi[hi])
        # low cell: outward flux q through its high face; high cell: outward flux -q
        acc[lo] -= (up - phi[lo]) * q
        acc[hi] -= (up - phi[hi]) * (-q)
    return S + dt / V * acc + dt * np.maximum(prob.f, 0.0) * (1.0 - phi)


def impes(prob: Problem, S0, mu_w, mu_o, cfl, C, n_steps, processes=None):
    """Alg. overview-code with the MRCM Darcy solver; returns (S, t, number of Darcy solves)."""
    S = np.array(S0, dtype=float)
    t = 0.0
    solves = 0
    u = None
    dt = 0.0
    for n in range(n_steps):
        if n % C == 0:
            K_eff = mobility(S, mu_w, mu_o)[None] * prob.K
            sub = Problem(n=prob.n, h=prob.h, edges=prob.edges, patch=prob.patch, K=K_eff, f=prob.f,
                          beta_mode=prob.beta_mode, alpha=prob.alpha, beta_const=prob.beta_const,
                          bc_type=prob.bc_type, bc_value=prob.bc_value)
            r = _mrcm.solve_mrcm(sub, keep=False, processes=processes)
            u = postprocess_mean(sub, r.u)
            dt = cfl_dt(sub, u, mu_w, mu_o, cfl)
            solves += 1
        S = transport_step(prob, S, u, dt, mu_w, mu_o)
        t += dt
    return S, t, solves
