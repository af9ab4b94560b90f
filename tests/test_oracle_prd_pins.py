"""Pins of the oracle's partial redistribution for the two-level atom.

The redistribution function's marginal against numerical quadrature, the
discrete matrix's symmetry and marginals, the CRD limits (no coherence, a
frequency-flat radiation field), photon conservation of the emission
profile, and the multigrid invariants with the lagged field.
"""

import math

import numpy as np
import pytest

from oracle import mg3d_oracle as O
from paper_1701_01607_gb300 import synth

special = pytest.importorskip("scipy.special")
integrate = pytest.importorskip("scipy.integrate")

PARAMS = dict(nu_fmg=4, nu0=4, nu1=2, nu2=2, nu3=32)


def _box(gamma, nx=8, nz=17, eps=1e-3, n_freq=9, x_max=3.0):
    atom = synth.TwoLevelAtom(gamma_prd=gamma, n_freq=n_freq, x_max=x_max)
    return synth.stratified_two_level(nx, nx, nz, eps=eps, sigma=0.3, seed=3, atom=atom)


def test_redistribution_function_marginal_is_the_doppler_profile():
    """int R(x', x) dx = exp(-x'^2)/sqrt(pi) for R = erfc(max(|x|, |x'|))/2."""
    for xp in (0.0, 0.3, 1.1, 2.5):
        f = lambda x: 0.5 * special.erfc(max(abs(x), abs(xp)))
        val = sum(integrate.quad(f, a, b, limit=200)[0]
                  for a, b in ((-np.inf, -abs(xp)), (-abs(xp), abs(xp)), (abs(xp), np.inf)))
        assert abs(val - math.exp(-xp * xp) / math.sqrt(math.pi)) < 1e-10


def test_discrete_matrix_is_symmetric_with_profile_marginals():
    for n_freq, x_max in ((9, 3.0), (17, 5.0), (1, 3.0)):
        atm, atom = _box(0.5, n_freq=n_freq, x_max=x_max)
        p = O.TwoLevelProblem(atm, atom)
        assert np.allclose(p.R, p.R.T, rtol=0, atol=1e-15)
        assert np.allclose((p.R * p.wq[:, None]).sum(axis=0), p.phi, rtol=1e-13)
        assert np.all(p.R > 0)


def test_vanishing_coherence_and_flat_field_reduce_to_crd():
    atm, atom = _box(0.0)
    crd = O.TwoLevelProblem(atm, atom)
    n = crd.zero_radiation(1)
    n, _ = crd.mali_sweep(1, n)
    ref = crd.formal_solution(1, n)
    # gamma -> 0 through the PRD code path
    atom.gamma_prd = 1e-14
    p = O.TwoLevelProblem(atm, atom)
    p.jnu[1] = np.abs(np.random.default_rng(1).normal(size=p.jnu[1].shape)) + 0.1
    for a, b in zip(p.formal_solution(1, n), ref):
        assert np.allclose(a, b, rtol=1e-12)
    # full coherence, but a radiation field flat in frequency: rho = 1
    atom.gamma_prd = 1.0
    q = O.TwoLevelProblem(atm, atom)
    q.jnu[1] = np.broadcast_to(np.linspace(0.2, 3.0, q.jnu[1].shape[1]), q.jnu[1].shape).copy()
    assert np.allclose(q.prd_profile_ratio(1), 1.0, rtol=0, atol=1e-13)
    for a, b in zip(q.formal_solution(1, n), ref):
        assert np.allclose(a, b, rtol=1e-12)


def test_emission_profile_conserves_photons():
    """sum_f w phi rho = 1 at every node for any positive field."""
    atm, atom = _box(0.8)
    p = O.TwoLevelProblem(atm, atom)
    p.jnu[1] = np.exp(np.random.default_rng(2).normal(size=p.jnu[1].shape))
    rho = p.prd_profile_ratio(1)
    assert np.allclose(p.wphi @ rho, 1.0, rtol=0, atol=1e-13)
    assert np.max(np.abs(rho - 1.0)) > 1e-2          # the field is not flat


def test_prd_conservation_multigrid_agreement_and_effect():
    atm, atom = _box(0.9, nx=4, nz=9, eps=1e-2)
    p = O.TwoLevelProblem(atm, atom, n_grids=3)
    n = p.zero_radiation(3)
    for _ in range(3):
        n, _ = p.mali_sweep(3, n)
        assert np.max(np.abs(n.sum(axis=0) / atm.n_tot - 1.0)) < 1e-13
    p1 = O.TwoLevelProblem(atm, atom, n_grids=3)
    n_mali = p1.zero_radiation(3)
    for _ in range(400):
        n_mali, C = p1.mali_sweep(3, n_mali)
        if C < 1e-13:
            break
    n_fas, _ = O.fas_solve(O.TwoLevelProblem(atm, atom, n_grids=3), 1e-11, PARAMS)
    n_fmg, _ = O.fmg_solve(O.TwoLevelProblem(atm, atom, n_grids=3), 1e-11, PARAMS)
    assert O.max_rel_error(n_fas, n_mali) < 1e-8
    assert O.max_rel_error(n_fmg, n_mali) < 1e-8
    atom.gamma_prd = 0.0
    n_crd, _ = O.mali_solve(O.TwoLevelProblem(atm, atom, n_grids=3), 1e-11)
    assert O.max_rel_error(n_crd, n_mali) > 1e-4


# ------------------------------------------------------ damping (Voigt, R_II-A)

def test_voigt_profile_matches_scipy():
    x = np.linspace(-6, 6, 25)
    for a in (0.01, 0.1, 1.0):
        ref = special.voigt_profile(x, 1.0 / math.sqrt(2.0), a)
        assert np.allclose(O.line_profile(x, a), ref, rtol=1e-12, atol=1e-15)
    assert np.allclose(O.line_profile(x, 0.0), np.exp(-x * x) / math.sqrt(math.pi))


def test_r2a_marginal_is_the_voigt_profile():
    """int R_II-A(x, x') dx' = H(a, x)/sqrt(pi): the angle-averaged function
    redistributes exactly the absorbed profile."""
    for a, x in ((0.05, 1.0), (0.5, 2.5)):
        m = sum(integrate.quad(lambda xp: O.redistribution_r2a(x, xp, a), lo, hi,
                               epsabs=1e-11, limit=200)[0]
                for lo, hi in ((-np.inf, -x), (-x, x), (x, np.inf)))
        assert abs(m / O.line_profile(np.array([x]), a)[0] - 1.0) < 1e-9


def test_r2a_limits_and_symmetries():
    r = O.redistribution_r2a
    assert abs(r(0.7, 1.3, 1e-6) - 0.5 * special.erfc(1.3)) < 1e-5
    assert abs(r(0.7, 1.3, 0.1) - r(1.3, 0.7, 0.1)) < 1e-14
    assert abs(r(-0.7, -1.3, 0.1) - r(0.7, 1.3, 0.1)) < 1e-14
    # coherent in the atom's frame: far-wing photons stay in their wing
    assert r(-3.5, 4.0, 0.05) < 1e-3 * r(3.5, 4.0, 0.05)


def test_prd_with_damping_conserves_and_fas_matches_mali():
    atom = synth.TwoLevelAtom(gamma_prd=1.0, a_damp=0.05, n_freq=13, x_max=5.0)
    atm, atom = synth.stratified_two_level(4, 4, 9, eps=3e-2, sigma=0.3, seed=3, atom=atom)
    p = O.TwoLevelProblem(atm, atom, n_grids=3)
    assert np.allclose((p.R * p.wq[:, None]).sum(axis=0), p.phi, rtol=1e-13)
    n = p.zero_radiation(3)
    for _ in range(3):
        n, _ = p.mali_sweep(3, n)
        assert np.max(np.abs(n.sum(axis=0) / atm.n_tot - 1.0)) < 1e-13
    p1 = O.TwoLevelProblem(atm, atom, n_grids=3)
    n_mali = p1.zero_radiation(3)
    for _ in range(400):
        n_mali, C = p1.mali_sweep(3, n_mali)
        if C < 1e-13:
            break
    n_fas, _ = O.fas_solve(O.TwoLevelProblem(atm, atom, n_grids=3), 1e-11, PARAMS)
    assert O.max_rel_error(n_fas, n_mali) < 1e-8
