"""Pins of the oracle's IMPES transport (Eq. transporte_discreto, Eq. CFL,
Alg. overview-code): a hand-computed upwind step, the global water balance
that the conservative upwind form implies, the maximum principle under the
CFL step, and the closed-form maximum of phi'."""
import numpy as np
import pytest

import oracle
from oracle.problem import Problem
from oracle.transport import (cfl_dt, frac_flow, frac_flow_slope_max, impes, mobility, transport_step)
from synth.configs import small


def test_hand_computed_upwind_step():
    """1-D column [water, water, oil, oil] with a uniform rightward flux U A on the
    interior faces: only the first oil cell changes, by dt U / h (upwind water)."""
    h = (0.5, 1.0, 2.0)
    prob = Problem(n=(4, 1, 1), h=h, edges=([4], [1], [1]), patch=((0, 0),) * 3,
                   K=np.ones((3, 1, 1, 4)), f=np.zeros((1, 1, 4)))
    S = np.array([1.0, 1.0, 0.0, 0.0]).reshape(1, 1, 4)
    U = 0.7
    u = np.zeros((6, 1, 1, 4))
    u[1, 0, 0, :3] = U          # x-high faces of cells 0..2
    u[0, 0, 0, 1:] = U          # x-low faces of cells 1..3 (the same faces)
    dt = 0.3
    S1 = transport_step(prob, S, u, dt, 1.0, 4.0)
    assert np.allclose(S1.ravel(), [1.0, 1.0, dt * U / h[0], 0.0], rtol=0, atol=1e-15)


def test_fractional_flow_slope_maximum():
    """phi'(S) = 2 M S (1 - S) / (M S^2 + (1 - S)^2)^2; for M = 1 its maximum is 2, at S = 1/2."""
    assert abs(frac_flow_slope_max(1.0, 1.0) - 2.0) < 1e-12
    # central difference of phi agrees with the slope formula's maximum for another ratio
    S = np.arange(1001) / 1000.0
    num = (frac_flow(S[2:], 1.0, 5.0) - frac_flow(S[:-2], 1.0, 5.0)) / 0.002
    assert abs(num.max() - frac_flow_slope_max(1.0, 5.0)) < 1e-3 * num.max()
    assert mobility(0.0, 1.0, 5.0) == 0.2 and mobility(1.0, 1.0, 5.0) == 1.0


def _two_phase_problem():
    w = small(n=(12, 12, 4), edges=([6, 6], [6, 6], [4]), patch=((3, 2), (3, 2), (3, 3)), sigma=1.5, lam=4.0,
              wells="five_spot")
    return oracle.from_workload(w)


def test_water_balance_and_maximum_principle():
    """With the post-processed (cell-conservative) velocity, the upwind fluxes
    cancel between neighbours: the water volume changes by the injected water
    minus the water the producers take out at their cells' fractional flow."""
    from oracle.postprocess import postprocess_mean
    prob = _two_phase_problem()
    mu_w, mu_o = 1.0, 5.0
    S = np.zeros(prob.f.shape)
    r = oracle.solve_mrcm(prob)
    u = postprocess_mean(prob, r.u)
    dt = cfl_dt(prob, u, mu_w, mu_o, 0.9)
    V = prob.cell_volume
    for _ in range(30):
        S1 = transport_step(prob, S, u, dt, mu_w, mu_o)
        phi = frac_flow(S, mu_w, mu_o)
        f = prob.f
        expect = dt * (np.sum(f[f > 0]) * V + np.sum(f[f < 0] * phi[f < 0]) * V)
        assert abs((S1 - S).sum() * V - expect) <= 1e-12 * max(1.0, abs(expect))
        assert S1.min() >= -1e-14 and S1.max() <= 1.0 + 1e-14
        S = S1
    assert S.max() > 0.05                       # water has entered


def test_impes_runs_the_darcy_solve_every_C_steps():
    prob = _two_phase_problem()
    S, t, solves = impes(prob, np.zeros(prob.f.shape), 1.0, 5.0, 0.9, C=4, n_steps=10)
    assert solves == 3 and t > 0
    assert S.min() >= -1e-14 and S.max() <= 1.0 + 1e-14
