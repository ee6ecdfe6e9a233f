"""Pins of the alpha limits of the Robin parameter (Sec. "Choice of multiscale method").

With beta = alpha H / K (Eq. Robin_par), alpha -> 0+ makes the multiscale
pressure continuous at every fine face of Gamma (the Robin condition becomes
p = P_H on both sides) and alpha -> infinity makes the normal velocity
continuous (u.n -> U_H on both sides).  The jumps vanish linearly in alpha and
in 1/alpha; both are checked on the oracle, and that refining the interface
spaces (Hbar = H/2) enlarges the system fourfold on interior faces and
reduces the error against the fine solution.
"""
import numpy as np
import pytest

import oracle
from oracle.problem import build_bases
from synth.configs import BETA_ALPHA_H_OVER_K, small


def _prob(alpha, patch=((0, 0), (0, 0), (0, 0)), n=(8, 8, 4), edges=([4, 4], [4, 4], [4])):
    return oracle.from_workload(small(n=n, edges=edges, patch=patch, beta_mode=BETA_ALPHA_H_OVER_K, alpha=alpha,
                                      sigma=1.5, lam=3.0))


def gamma_jumps(prob, p, u):
    """Max over fine Gamma faces of the jump of the face pressure and of the normal velocity.

    Face pressure seen from a side: p_f = p_c - (u.n_out) h / (2 K), the half-cell
    two-point relation of the Robin faces."""
    sub = prob.sub_of_cell()
    P = p.reshape(prob.f.shape)
    jp = ju = 0.0
    for a in range(3):
        ax = 2 - a
        lo = [slice(None)] * 3
        hi = [slice(None)] * 3
        lo[ax], hi[ax] = slice(0, -1), slice(1, None)
        lo, hi = tuple(lo), tuple(hi)
        g = sub[lo] != sub[hi]
        if not g.any():
            continue
        ulo, uhi = u[2 * a + 1][lo][g], u[2 * a][hi][g]
        Klo, Khi = prob.K[a][lo][g], prob.K[a][hi][g]
        pf_lo = P[lo][g] - ulo * prob.h[a] / (2 * Klo)
        pf_hi = P[hi][g] + uhi * prob.h[a] / (2 * Khi)
        jp = max(jp, np.abs(pf_lo - pf_hi).max())
        ju = max(ju, np.abs(ulo - uhi).max())
    return jp / np.abs(p).max(), ju / np.abs(u).max()


def test_alpha_to_zero_gives_pressure_continuity():
    j = [gamma_jumps(pr, r.p, r.u) for pr in (_prob(1.0), _prob(1e-3), _prob(1e-6))
         for r in [oracle.solve_mrcm(pr)]]
    assert j[0][0] > 1e-3                      # alpha = 1: discontinuous pressure
    assert j[1][0] < 1e-2 * j[0][0]            # shrinks with alpha ...
    assert j[2][0] < 2e-3 * j[1][0]            # ... linearly (1000x from 1e-3 to 1e-6)
    assert j[2][1] > 1e-3                      # the velocity stays discontinuous


def test_alpha_to_infinity_gives_velocity_continuity():
    j = [gamma_jumps(pr, r.p, r.u) for pr in (_prob(1.0), _prob(1e3), _prob(1e6))
         for r in [oracle.solve_mrcm(pr)]]
    assert j[0][1] > 1e-3
    assert j[1][1] < 1e-2 * j[0][1]
    assert j[2][1] < 2e-3 * j[1][1]
    assert j[2][0] > 1e-3                      # the pressure stays discontinuous


@pytest.mark.parametrize("alpha", [1e-6, 1.0, 1e6])
def test_staged_equals_monolithic_at_extreme_alpha(alpha):
    prob = _prob(alpha, patch=((2, 2), (2, 2), (2, 2)), n=(6, 4, 4), edges=([3, 3], [2, 2], [4]))
    r = oracle.solve_mrcm(prob)
    pm, Xm = oracle.solve_monolithic(prob)
    assert np.abs(r.p - pm).max() <= 1e-9 * np.abs(pm).max()


def test_halving_the_interface_elements():
    """Hbar = H/2: four times the dofs on each interior face, and a smaller error."""
    whole = _prob(1e-6)
    half = _prob(1e-6, patch=((2, 2), (2, 2), (2, 2)))
    nb_whole = len(build_bases(whole)[0])
    nb_half = len(build_bases(half)[0])
    assert nb_half == 4 * nb_whole
    pf, uf = oracle.solve_fine(whole)
    e_whole = oracle.relative_errors(whole, oracle.solve_mrcm(whole).p, oracle.solve_mrcm(whole).u, pf, uf)
    rh = oracle.solve_mrcm(half)
    e_half = oracle.relative_errors(half, rh.p, rh.u, pf, uf)
    assert e_half[0] < e_whole[0] and e_half[1] < e_whole[1]
