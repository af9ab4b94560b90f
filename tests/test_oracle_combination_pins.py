"""Pins of the oracle on variant combinations: a flow with the Hermite-spline
upwind interpolation or with damped (Voigt) profiles, partial redistribution
with the Hermite upwind interpolation or in a flow (redistribution in the
comoving frame), and the multi-level atom in a flow with the Hermite upwind.

Each combination reduces in a limit to a path pinned on its own (zero flow
gives the static path, vanishing coherence gives CRD), follows the
closed form of horizontally homogeneous columns, is symmetric under reversal
of the flow, and keeps the multigrid invariants (conservation, MALI = FAS =
FMG).  The Voigt profile is pinned to closed forms that do not go through
the Faddeeva routine it calls.
"""

import math

import numpy as np
import pytest

from oracle import mg3d_oracle as O
from paper_1701_01607_gb300 import synth

special = pytest.importorskip("scipy.special")
integrate = pytest.importorskip("scipy.integrate")

PARAMS = dict(nu_fmg=4, nu0=4, nu1=2, nu2=2, nu3=32)

# (upwind interpolation, damping) of a flow: Hermite, Voigt, both
FLOW_VARIANTS = [(1, 0.0), (0, 0.05), (1, 0.05)]


def _box(nx=8, nz=17, eps=1e-2, velocity=1.0, seed=3, n_freq=9, x_max=3.0, a_damp=0.0,
         gamma=0.0):
    atom = synth.TwoLevelAtom(n_freq=n_freq, x_max=x_max, a_damp=a_damp, gamma_prd=gamma)
    return synth.stratified_two_level(nx, nx, nz, eps=eps, sigma=0.3, seed=seed, atom=atom,
                                      velocity=velocity)


# ------------------------------------------------------------ Voigt profile

def _w_asymptotic(z, terms=8):
    """w(z) ~ (i/(sqrt(pi) z)) sum_k (2k-1)!!/(2 z^2)^k for large |z| in the
    upper half plane (the exp(-z^2) part is below 1e-600 where used)."""
    s, t = 0j, 1 + 0j
    for k in range(terms):
        s += t
        t *= (2 * k + 1) / (2 * z * z)
    return 1j * s / (math.sqrt(math.pi) * z)


def test_voigt_profile_closed_forms():
    # line centre: H(a, 0) = exp(a^2) erfc(a)
    for a in (0.01, 0.3, 1.0, 3.0):
        ref = math.exp(a * a) * math.erfc(a) / math.sqrt(math.pi)
        assert abs(O.line_profile(np.array([0.0]), a)[0] / ref - 1.0) < 1e-13
    # far wings: the asymptotic series of w(x + i a)
    for a in (0.05, 0.5, 2.0):
        for x in (40.0, -55.0, 80.0):
            ref = _w_asymptotic(complex(x, a)).real / math.sqrt(math.pi)
            assert abs(O.line_profile(np.array([x]), a)[0] / ref - 1.0) < 1e-12
    # unit area, even in x
    for a in (0.02, 0.5):
        area = 2.0 * sum(integrate.quad(lambda x: O.line_profile(np.array([x]), a)[0],
                                        lo, hi, limit=400, epsabs=1e-13)[0]
                         for lo, hi in ((0.0, 6.0), (6.0, np.inf)))
        assert abs(area - 1.0) < 1e-9
        x = np.linspace(0.1, 7.0, 11)
        assert np.array_equal(O.line_profile(x, a), O.line_profile(-x, a))


# --------------------------------------------------- two-level atom in a flow

@pytest.mark.parametrize("interp,a_damp", FLOW_VARIANTS)
def test_zero_flow_equals_the_static_path(interp, a_damp):
    atm, atom = _box(velocity=0.0, a_damp=a_damp)
    assert atm.vel is None
    static = O.TwoLevelProblem(atm, atom, sc_interp=interp)
    n = static.zero_radiation(1)
    n, _ = static.mali_sweep(1, n)
    ref = static.formal_solution(1, n)
    atm.vel = np.zeros((3,) + atm.shape)
    got = O.TwoLevelProblem(atm, atom, sc_interp=interp).formal_solution(1, n)
    for a, b in zip(got, ref):
        assert np.allclose(a, b, rtol=1e-13, atol=0)


@pytest.mark.parametrize("interp,a_damp", FLOW_VARIANTS)
def test_homogeneous_columns_in_a_flow_closed_form(interp, a_damp):
    """Planes of constant chi0, S and velocity u(z): any upwind interpolation
    returns the plane value, so along each ray I = S + (I_in - S) exp(-tau)
    with the trapezoid optical depth of the ray's shifted profile (Voigt when
    damped), and Jbar is the renormalised profile average over frequencies
    and rays."""
    nx, nz = 4, 17
    atm, atom = _box(nx=nx, nz=nz, a_damp=a_damp)
    z = atm.z
    zz = (z - z[0]) / (z[-1] - z[0])
    uz = np.stack([0.8 * np.sin(3 * zz), -0.5 * zz, 1.2 * np.cos(2 * zz) - 0.4])
    atm.vel = np.ascontiguousarray(np.broadcast_to(uz[:, :, None, None], (3, nz, nx, nx)))
    atm.n_tot = np.ascontiguousarray(np.broadcast_to(atm.n_tot[:, :1, :1], atm.shape))
    p = O.TwoLevelProblem(atm, atom, sc_interp=interp)
    B = float(p.planck(atm.T[0, 0, 0]))
    S0 = 0.5 * B
    g = atom.g_ratio
    n = np.empty((2,) + atm.shape)
    n[0] = atm.n_tot / (1.0 + S0 * g / (1.0 + S0))
    n[1] = atm.n_tot - n[0]
    Jbar, _, _ = p.formal_solution(1, n)
    chi0 = atom.kappa * (n[0, :, 0, 0] * g - n[1, :, 0, 0])
    wq = p.wphi / p.phi
    J = np.zeros(nz)
    for r in range(24):
        mu = p.mu[r]
        sx = p.x[:, None] - (mu @ uz)[None, :]
        prof = (special.voigt_profile(sx, 1.0 / math.sqrt(2.0), a_damp) if a_damp > 0
                else np.exp(-sx ** 2) / math.sqrt(math.pi))
        dtau = 0.5 * (chi0[None, 1:] * prof[:, 1:] + chi0[None, :-1] * prof[:, :-1]) * \
            np.diff(z)[None, :] / abs(mu[2])
        zero = np.zeros((len(p.x), 1))
        if mu[2] > 0:
            I = S0 + (B - S0) * np.exp(-np.concatenate([zero, np.cumsum(dtau, axis=1)], axis=1))
        else:
            tau = np.concatenate([np.cumsum(dtau[:, ::-1], axis=1)[:, ::-1], zero], axis=1)
            I = S0 - S0 * np.exp(-tau)
        w = wq[:, None] * prof
        J += p.wray[r] * np.sum(w / w.sum(axis=0) * I, axis=0)
    assert np.allclose(Jbar, J[:, None, None], rtol=1e-12)


@pytest.mark.parametrize("interp,a_damp", FLOW_VARIANTS)
def test_reversed_flow_same_mean_intensity(interp, a_damp):
    """The frequency grid is symmetric and both profiles are even: reversing
    the flow maps frequency x onto -x along every ray, for any upwind
    interpolation, so Jbar and U keep their values."""
    atm, atom = _box(nx=4, nz=9, a_damp=a_damp)
    p = O.TwoLevelProblem(atm, atom, sc_interp=interp)
    n = p.zero_radiation(1)
    n, _ = p.mali_sweep(1, n)
    a = p.formal_solution(1, n)
    atm.vel = -atm.vel
    b = O.TwoLevelProblem(atm, atom, sc_interp=interp).formal_solution(1, n)
    for x, y in zip(a, b):
        assert np.allclose(x, y, rtol=1e-12)


def test_damped_flow_dense_lambda_solve_matches_converged_mali():
    """Linear upwind interpolation keeps the formal solution affine in S at
    fixed opacity, with Voigt profiles too: the converged MALI source
    function solves S = (1 - eps) Lambda S + (1 - eps) J_bc + eps B."""
    atm, atom = _box(nx=4, nz=9, eps=0.1, a_damp=0.05)
    p = O.TwoLevelProblem(atm, atom)
    n_conv, _ = O.mali_solve(p, 1e-13)
    g = atom.g_ratio
    nl, nu = n_conv[0], n_conv[1]
    diff = nl * g - nu
    S = nu / diff
    nvox = S.size

    def jbar(Sv):
        m = np.empty_like(n_conv)
        m[1] = Sv.reshape(nl.shape) * diff
        m[0] = (diff + m[1]) / g
        return p.formal_solution(1, m)[0].reshape(-1)

    J_bc = jbar(np.zeros(nvox))
    Lam = np.empty((nvox, nvox))
    for i in range(nvox):
        e = np.zeros(nvox)
        e[i] = 1.0
        Lam[:, i] = jbar(e) - J_bc
    lev = p.levels[1]
    epsp = lev.c_ul.reshape(-1) * (-np.expm1(-atom.theta / lev.T.reshape(-1))) / atom.a_ul
    eps = epsp / (1.0 + epsp)
    Bn = p.planck(lev.T).reshape(-1)
    S_direct = np.linalg.solve(np.eye(nvox) - (1.0 - eps)[:, None] * Lam,
                               eps * Bn + (1.0 - eps) * J_bc)
    assert np.max(np.abs(S.reshape(-1) - S_direct) / S_direct) < 1e-10


def _agreement(atm, atom, interp, n_grids=3):
    p = O.TwoLevelProblem(atm, atom, n_grids=n_grids, sc_interp=interp)
    n = p.zero_radiation(n_grids)
    for _ in range(3):
        n, _ = p.mali_sweep(n_grids, n)
        assert np.max(np.abs(n.sum(axis=0) / atm.n_tot - 1.0)) < 1e-13
    q = O.TwoLevelProblem(atm, atom, n_grids=n_grids, sc_interp=interp)
    n_mali = q.zero_radiation(n_grids)
    for _ in range(600):
        n_mali, C = q.mali_sweep(n_grids, n_mali)
        if C < 1e-13:
            break
    n_fas, _ = O.fas_solve(O.TwoLevelProblem(atm, atom, n_grids=n_grids, sc_interp=interp),
                           1e-11, PARAMS)
    n_fmg, _ = O.fmg_solve(O.TwoLevelProblem(atm, atom, n_grids=n_grids, sc_interp=interp),
                           1e-11, PARAMS)
    assert O.max_rel_error(n_fas, n_mali) < 1e-8
    assert O.max_rel_error(n_fmg, n_mali) < 1e-8
    return n_mali


@pytest.mark.parametrize("interp,a_damp", FLOW_VARIANTS)
def test_flow_variants_conserve_and_multigrid_agrees(interp, a_damp):
    atm, atom = _box(nx=4, nz=9, eps=3e-2, a_damp=a_damp, n_freq=11, x_max=4.0)
    n_flow = _agreement(atm, atom, interp)
    atm.vel = None
    n_static = _agreement(atm, atom, interp)
    assert O.max_rel_error(n_flow, n_static) > 1e-4      # the flow matters


# -------------------------------------- partial redistribution, Hermite upwind

def test_prd_with_hermite_reduces_to_crd_hermite():
    """Vanishing coherence, and full coherence in a frequency-flat field,
    both give the CRD formal solution with the same upwind interpolation."""
    atm, atom = _box(velocity=0.0)
    crd = O.TwoLevelProblem(atm, atom, sc_interp=1)
    n = crd.zero_radiation(1)
    n, _ = crd.mali_sweep(1, n)
    ref = crd.formal_solution(1, n)
    atom.gamma_prd = 1e-14
    p = O.TwoLevelProblem(atm, atom, sc_interp=1)
    p.jnu[1] = np.abs(np.random.default_rng(1).normal(size=p.jnu[1].shape)) + 0.1
    for a, b in zip(p.formal_solution(1, n), ref):
        assert np.allclose(a, b, rtol=1e-12)
    atom.gamma_prd = 1.0
    q = O.TwoLevelProblem(atm, atom, sc_interp=1)
    q.jnu[1] = np.broadcast_to(np.linspace(0.2, 3.0, q.jnu[1].shape[1]),
                               q.jnu[1].shape).copy()
    for a, b in zip(q.formal_solution(1, n), ref):
        assert np.allclose(a, b, rtol=1e-12)


@pytest.mark.parametrize("a_damp", [0.0, 0.05])
def test_prd_with_hermite_conserves_and_multigrid_agrees(a_damp):
    atm, atom = _box(nx=4, nz=9, eps=1e-2, velocity=0.0, gamma=0.9, a_damp=a_damp,
                     n_freq=11, x_max=4.0)
    n_prd = _agreement(atm, atom, interp=1)
    atom.gamma_prd = 0.0
    n_crd = _agreement(atm, atom, interp=1)
    assert O.max_rel_error(n_prd, n_crd) > 1e-4          # redistribution matters


# --------------------------------------- multi-level atom, flow and Hermite

def _ml(velocity, nx=4, nz=9, scattering=0.0):
    atom = synth.hydrogen_like_atom(line_freq=5, cont_freq=3, seed=2)
    atm = synth.chromosphere(nx, nx, nz, atom, seed=2, velocity=velocity, scattering=scattering)
    return atm, atom


def test_multilevel_hermite_zero_flow_equals_static_path():
    atm, atom = _ml(velocity=0.0)
    p0 = O.MultiLevelProblem(atm, atom, sc_interp=1)
    n = p0.zero_radiation(1)
    J0, U0, t0 = p0.formal_solution(1, n)
    atm.vel = np.zeros((3,) + atm.shape)
    p1 = O.MultiLevelProblem(atm, atom, sc_interp=1)
    J1, U1, t1 = p1.formal_solution(1, n)
    for a, b in ((t1["qa"] * J1, t0["qa"] * J0), (t1["qb"] * J1, t0["qb"] * J0),
                 (t1["qe"] * U1, t0["qe"] * U0)):
        err = np.max(np.abs(a - b), axis=1) / np.max(np.abs(b), axis=1)
        assert np.max(err) < 1e-12
    assert O.max_rel_error(p1.mali_sweep(1, n)[0], p0.mali_sweep(1, n)[0]) < 1e-10


def test_multilevel_hermite_flow_reversal_conservation_and_fas():
    atm, atom = _ml(velocity=1.0, scattering=1.0)
    # each problem starts itself: the start also Lambda-iterates its own
    # background field
    p = O.MultiLevelProblem(atm, atom, sc_interp=1)
    na = p.mali_sweep(1, p.mali_sweep(1, p.zero_radiation(1))[0])[0]
    atm.vel = -atm.vel
    q = O.MultiLevelProblem(atm, atom, sc_interp=1)
    nb = q.mali_sweep(1, q.mali_sweep(1, q.zero_radiation(1))[0])[0]
    assert O.max_rel_error(nb, na) < 1e-10
    r = O.MultiLevelProblem(atm, atom, n_grids=2, sc_interp=1)
    n2 = r.zero_radiation(2)
    for _ in range(3):
        n2, _ = r.mali_sweep(2, n2)
        assert np.max(np.abs(n2.sum(axis=0) / atm.n_tot - 1.0)) < 1e-13
    n_fas, _ = O.fas_solve(O.MultiLevelProblem(atm, atom, n_grids=2, sc_interp=1), 1e-10,
                           PARAMS, max_cycles=60)
    m = O.MultiLevelProblem(atm, atom, n_grids=1, sc_interp=1)
    n_mali = m.zero_radiation(1)
    for _ in range(60):
        n_mali, C = m.mali_sweep(1, n_mali)
        if C < 1e-12:
            break
    assert O.max_rel_error(n_fas, n_mali) < 1e-9


# ------------------------------ partial redistribution in a flow (two-level)

@pytest.mark.parametrize("interp", [0, 1])
def test_prd_in_a_flow_reduces_to_static_prd_and_moving_crd(interp):
    """Zero flow: the static PRD oracle (sweeps, a V-cycle, the lagged
    field) with either upwind interpolation; vanishing coherence: the moving
    CRD oracle."""
    atm, atom = _box(nx=4, nz=9, velocity=0.0, gamma=0.9)
    ps = O.TwoLevelProblem(atm, atom, n_grids=2, sc_interp=interp)
    ns = ps.zero_radiation(2)
    atm.vel = np.zeros((3,) + atm.shape)
    pm = O.TwoLevelProblem(atm, atom, n_grids=2, sc_interp=interp)
    nm = pm.zero_radiation(2)
    for _ in range(3):
        ns, cs = ps.mali_sweep(2, ns)
        nm, cm = pm.mali_sweep(2, nm)
        assert abs(cm - cs) < 1e-12
    ns, _ = ps.fas_cycle(ns, False, PARAMS)
    nm, _ = pm.fas_cycle(nm, False, PARAMS)
    assert O.max_rel_error(nm, ns) < 1e-12
    assert np.allclose(pm.jnu[2], ps.jnu[2], rtol=1e-12)
    atm2, atom2 = _box(nx=4, nz=9, gamma=1e-14)
    atm3, atom3 = _box(nx=4, nz=9, gamma=0.0)
    q = O.TwoLevelProblem(atm2, atom2)
    q.jnu[1] = np.exp(np.random.default_rng(4).normal(size=q.jnu[1].shape))
    n0 = q.zero_radiation(1)
    q.jnu[1] = np.exp(np.random.default_rng(4).normal(size=q.jnu[1].shape))
    got = q.formal_solution(1, n0)
    ref = O.TwoLevelProblem(atm3, atom3).formal_solution(1, n0)
    for a, b in zip(got, ref):
        assert np.allclose(a, b, rtol=1e-12)


def test_prd_in_a_uniform_flow_tends_to_static_prd():
    """A uniform flow is a Galilean shift: with redistribution in the
    comoving frame the converged populations approach the static PRD ones
    at second order in the frequency step (linear interpolation in
    frequency); a wrong sign in either frequency shift leaves a gap near
    0.025 that refinement does not close."""
    gaps = []
    for n_freq in (41, 81):
        atm, atom = _box(nx=4, nz=9, velocity=0.0, gamma=1.0, n_freq=n_freq, x_max=6.0)
        n_static, _ = O.mali_solve(O.TwoLevelProblem(atm, atom), 1e-12)
        atm.vel = np.empty((3,) + atm.shape)
        atm.vel[0], atm.vel[1], atm.vel[2] = 0.4, -0.3, 0.6
        n_flow, _ = O.mali_solve(O.TwoLevelProblem(atm, atom), 1e-12)
        gaps.append(O.max_rel_error(n_flow, n_static))
    assert gaps[1] < 1e-3 and gaps[1] < 0.3 * gaps[0], gaps


def test_prd_in_a_flow_conserves_and_multigrid_agrees():
    atm, atom = _box(nx=4, nz=9, eps=3e-2, gamma=0.9, n_freq=11, x_max=4.0)
    n_prd = _agreement(atm, atom, interp=0)
    atom.gamma_prd = 0.0
    n_crd = _agreement(atm, atom, interp=0)
    assert O.max_rel_error(n_prd, n_crd) > 1e-4


def test_prd_in_a_flow_keeps_mali_positive_when_scattering_dominates():
    """eps = 1e-3, full coherence, a flow of rms 1 Doppler width on a grid
    of +-3 widths: with the emission ratio scaled per node and ray to
    conserve photons, MALI stays positive and converges (without that
    scaling the second sweep already drives populations negative)."""
    atm, atom = _box(nx=4, nz=17, eps=1e-3, velocity=1.0, gamma=1.0)
    p = O.TwoLevelProblem(atm, atom)
    n = p.zero_radiation(1)
    for _ in range(200):
        n, C = p.mali_sweep(1, n)
        assert np.all(n > 0)
        if C < 1e-8:
            break
    assert C < 1e-8
