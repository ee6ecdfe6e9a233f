"""Pins of the oracle's mean velocity post-processing (Eq. locprob_submean).

Each check is a property that the paper states or that follows from the
equations: the post-processed velocity is conservative cell by cell on the
fine scale, single-valued on Gamma, carries the multiscale flux through every
patch (Eq. weakcont_f), and changes nothing when the multiscale velocity is
already single-valued (fine-face interface spaces, where the MRCM reproduces
the fine TPFA solution).
"""
import numpy as np
import pytest

import oracle
from oracle.postprocess import mean_gamma_velocity, postprocess_mean
from oracle.problem import build_bases
from synth.configs import BETA_ALPHA_H_OVER_K, small

CASES = [
    dict(),
    dict(n=(9, 7, 5), edges=([4, 5], [2, 3, 2], [5]), patch=((2, 2), (3, 2), (2, 3))),
    dict(n=(6, 6, 6), edges=([3, 3], [3, 3], [2, 4]), patch=((0, 0), (2, 0), (0, 2)),
         beta_mode=BETA_ALPHA_H_OVER_K, alpha=0.7),
    dict(n=(8, 4, 4), edges=([2, 3, 3], [4], [2, 2]), patch=((1, 2), (1, 1), (3, 1)), beta_const=0.3,
         h=(0.5, 1.0, 2.0)),
]


def _prob(n=(8, 6, 4), edges=([4, 4], [3, 3], [2, 2]), patch=((2, 1), (2, 1), (2, 2)), **kw):
    return oracle.from_workload(small(n=n, edges=edges, patch=patch, **kw))


@pytest.mark.parametrize("kw", CASES)
def test_postprocessed_velocity_is_conservative_and_single_valued(kw):
    prob = _prob(**kw)
    r = oracle.solve_mrcm(prob)
    # the multiscale velocity is two-valued on Gamma with coarse patches
    jump = np.abs(mean_gamma_velocity(prob, r.u) - r.u).max()
    assert jump > 1e-8
    up = postprocess_mean(prob, r.u)
    res = oracle.mass_residual(prob, up)
    assert np.abs(res).max() <= 1e-12 * max(1.0, np.abs(prob.f).max() * prob.cell_volume)
    bases, _, _ = build_bases(prob)
    uf, mf = up.reshape(6, -1), r.u.reshape(6, -1)
    for b in bases:
        a = b.axis
        # single-valued on every fine face of the patch
        for clo, chi in b.faces:
            assert uf[2 * a + 1, clo] == uf[2 * a, chi]
        # the patch carries the multiscale solution's flux (Eq. weakcont_f)
        flux_pp = sum(uf[2 * a + 1, clo] for clo, _ in b.faces)
        flux_ms = sum(mf[2 * a + 1, clo] for clo, _ in b.faces)
        assert abs(flux_pp - flux_ms) <= 1e-11 * max(1.0, np.abs(mf).max())


@pytest.mark.parametrize("kw", CASES)
def test_postprocessing_is_identity_for_fine_face_spaces(kw):
    """With one-face patches the MRCM velocity equals the fine TPFA velocity,
    already single-valued and conservative: the Neumann re-solve returns it."""
    kw = dict(kw)
    kw["patch"] = ((1, 1), (1, 1), (1, 1))
    prob = _prob(**kw)
    r = oracle.solve_mrcm(prob)
    pf, uf = oracle.solve_fine(prob)
    up = postprocess_mean(prob, r.u)
    assert np.abs(up - uf).max() <= 1e-11 * np.abs(uf).max()


def test_postprocessing_reduces_the_error_against_the_fine_solution():
    """The post-processed velocity is the fine-scale conservative one the
    transport needs; with coarse patches it stays close to the fine solution
    (its error is of the multiscale method's size, not larger)."""
    prob = _prob(n=(12, 12, 4), edges=([6, 6], [6, 6], [4]), patch=((3, 2), (3, 2), (3, 3)))
    r = oracle.solve_mrcm(prob)
    pf, uf = oracle.solve_fine(prob)
    up = postprocess_mean(prob, r.u)
    e_ms = oracle.relative_errors(prob, r.p, r.u, pf, uf)[1]
    e_pp = oracle.relative_errors(prob, r.p, up, pf, uf)[1]
    assert e_pp < 2.0 * e_ms
