"""Pins of the oracle's moving-atmosphere formal solution and iterations.

Closed forms for horizontally homogeneous columns with height-dependent
velocities, the static limit, the reversal symmetry of a symmetric frequency
grid, the Galilean limit of a uniform flow, a dense solve of the discrete
Lambda operator and the multigrid invariants.
"""

import math

import numpy as np

from oracle import mg3d_oracle as O
from paper_1701_01607_gb300 import synth

PARAMS = dict(nu_fmg=4, nu0=4, nu1=2, nu2=2, nu3=32)


def _box(nx=8, nz=17, eps=1e-2, velocity=1.0, seed=3, n_freq=9, x_max=3.0):
    atom = synth.TwoLevelAtom(n_freq=n_freq, x_max=x_max)
    return synth.stratified_two_level(nx, nx, nz, eps=eps, sigma=0.3, seed=seed, atom=atom,
                                      velocity=velocity)


def test_zero_velocity_equals_static_path():
    atm, atom = _box(velocity=0.0)
    assert atm.vel is None
    static = O.TwoLevelProblem(atm, atom)
    n = static.zero_radiation(1)
    ref = static.formal_solution(1, n)
    atm.vel = np.zeros((3,) + atm.shape)
    got = O.TwoLevelProblem(atm, atom).formal_solution(1, n)
    for a, b in zip(got, ref):
        assert np.allclose(a, b, rtol=1e-13, atol=0)


def test_homogeneous_columns_with_velocity_closed_form():
    """Planes of constant chi0, S and velocity u(z): along each ray the
    solution is I = S + (I_in - S) exp(-tau) with the trapezoid optical depth
    of the ray's Doppler-shifted profile, and Jbar is the renormalised
    profile average of it over frequencies and rays."""
    nx, nz = 4, 17
    atm, atom = _box(nx=nx, nz=nz)
    z = atm.z
    zz = (z - z[0]) / (z[-1] - z[0])
    uz = np.stack([0.8 * np.sin(3 * zz), -0.5 * zz, 1.2 * np.cos(2 * zz) - 0.4])   # [3, nz]
    atm.vel = np.ascontiguousarray(np.broadcast_to(uz[:, :, None, None], (3, nz, nx, nx)))
    atm.n_tot = np.ascontiguousarray(np.broadcast_to(atm.n_tot[:, :1, :1], atm.shape))
    p = O.TwoLevelProblem(atm, atom)
    # populations with a constant source function S0 = B/2 (not B: I_in != S)
    B = float(p.planck(atm.T[0, 0, 0]))
    S0 = 0.5 * B
    g = atom.g_ratio
    n = np.empty((2,) + atm.shape)
    n[0] = atm.n_tot / (1.0 + S0 * g / (1.0 + S0))
    n[1] = atm.n_tot - n[0]
    Jbar, _, _ = p.formal_solution(1, n)
    chi0 = atom.kappa * (n[0, :, 0, 0] * g - n[1, :, 0, 0])                     # [nz]
    wq = p.wphi / p.phi
    J = np.zeros(nz)
    for r in range(24):
        mu = p.mu[r]
        ur = mu @ uz                                                            # [nz]
        prof = np.exp(-(p.x[:, None] - ur[None, :]) ** 2) / math.sqrt(math.pi)  # [nf, nz]
        chi = chi0[None, :] * prof
        dtau = 0.5 * (chi[:, 1:] + chi[:, :-1]) * np.diff(z)[None, :] / abs(mu[2])
        if mu[2] > 0:
            tau = np.concatenate([np.zeros((len(p.x), 1)), np.cumsum(dtau, axis=1)], axis=1)
            I = S0 + (B - S0) * np.exp(-tau)
        else:
            tau = np.concatenate([np.cumsum(dtau[:, ::-1], axis=1)[:, ::-1],
                                  np.zeros((len(p.x), 1))], axis=1)
            I = S0 - S0 * np.exp(-tau)
        w = wq[:, None] * prof
        J += p.wray[r] * np.sum(w / w.sum(axis=0) * I, axis=0)
    assert np.allclose(Jbar, J[:, None, None], rtol=1e-12)


def test_reversed_flow_gives_the_same_mean_intensity():
    """On a frequency grid symmetric about line centre, reversing the flow
    maps phi(x - mu.u) onto phi(-x + mu.u): the same profile values over the
    grid, so Jbar and U do not change."""
    atm, atom = _box(nx=4, nz=9)
    p = O.TwoLevelProblem(atm, atom)
    n = p.zero_radiation(1)
    a = p.formal_solution(1, n)
    atm.vel = -atm.vel
    b = O.TwoLevelProblem(atm, atom).formal_solution(1, n)
    for x, y in zip(a, b):
        assert np.allclose(x, y, rtol=1e-12)
    # the flow does change the solution
    atm.vel = np.zeros_like(atm.vel)
    c = O.TwoLevelProblem(atm, atom).formal_solution(1, n)
    assert np.max(np.abs(c[0] - a[0]) / a[0]) > 1e-3


def test_uniform_flow_tends_to_the_static_solution():
    """A uniform flow is a Galilean shift: with a frequency grid wide and
    fine enough for the shifted profile the converged populations approach
    the static ones, and the gap closes as the grid widens."""
    gaps = []
    for n_freq, x_max in ((17, 4.0), (41, 6.0)):
        atm, atom = _box(nx=4, nz=9, velocity=0.0, n_freq=n_freq, x_max=x_max)
        n_static, _ = O.mali_solve(O.TwoLevelProblem(atm, atom), 1e-12)
        atm.vel = np.empty((3,) + atm.shape)
        atm.vel[0], atm.vel[1], atm.vel[2] = 0.4, -0.3, 0.6
        n_flow, _ = O.mali_solve(O.TwoLevelProblem(atm, atom), 1e-12)
        gaps.append(O.max_rel_error(n_flow, n_static))
    assert gaps[1] < 1e-4 and gaps[1] < 0.1 * gaps[0], gaps


def test_moving_dense_lambda_solve_matches_converged_mali():
    """The moving formal solution is linear in S: Jbar = Lambda S + J_bc.
    Lambda is built column by column (S = e_i, no incident radiation) and
    the converged MALI source function solves S = (1 - eps) Jbar + eps B."""
    atm, atom = _box(nx=4, nz=9, eps=0.1)
    p = O.TwoLevelProblem(atm, atom)
    n_conv, _ = O.mali_solve(p, 1e-13)
    g = atom.g_ratio
    nl, nu = n_conv[0], n_conv[1]
    S = nu / (nl * g - nu)
    nvox = S.size
    # Jbar(S) is affine in S at fixed opacity; the opacity depends on n, so
    # keep chi0 = n_l g - n_u fixed by scaling n_l with S
    def jbar(Sv):
        Sv = Sv.reshape(nl.shape)
        diff = nl * g - nu
        m = np.empty_like(n_conv)
        m[1] = Sv * diff
        m[0] = (diff + m[1]) / g
        return p.formal_solution(1, m)[0].reshape(-1)

    J_bc = jbar(np.zeros(nvox))
    Lam = np.empty((nvox, nvox))
    for i in range(nvox):
        e = np.zeros(nvox)
        e[i] = 1.0
        Lam[:, i] = jbar(e) - J_bc
    lev = p.levels[1]
    c_ul = lev.c_ul.reshape(-1)
    epsp = c_ul * (-np.expm1(-atom.theta / lev.T.reshape(-1))) / atom.a_ul
    eps = epsp / (1.0 + epsp)
    B = p.planck(lev.T).reshape(-1)
    S_direct = np.linalg.solve(np.eye(nvox) - (1.0 - eps)[:, None] * Lam,
                               eps * B + (1.0 - eps) * J_bc)
    assert np.max(np.abs(S.reshape(-1) - S_direct) / S_direct) < 1e-10


def test_moving_conservation_and_multigrid_agreement():
    atm, atom = _box(nx=4, nz=9, eps=3e-2)
    p = O.TwoLevelProblem(atm, atom, n_grids=3)
    n = p.zero_radiation(3)
    for _ in range(3):
        n, _ = p.mali_sweep(3, n)
        assert np.max(np.abs(n.sum(axis=0) / atm.n_tot - 1.0)) < 1e-13
    n_mali, _ = O.mali_solve(O.TwoLevelProblem(atm, atom, n_grids=3), 1e-11)
    n_fas, _ = O.fas_solve(O.TwoLevelProblem(atm, atom, n_grids=3), 1e-11, PARAMS)
    n_fmg, _ = O.fmg_solve(O.TwoLevelProblem(atm, atom, n_grids=3), 1e-11, PARAMS)
    assert O.max_rel_error(n_fas, n_mali) < 1e-8
    assert O.max_rel_error(n_fmg, n_mali) < 1e-8
    # the coarse grids carry the full-weighted flow
    assert np.allclose(p.levels[2].vel, O.restrict_fw(atm.vel))


# ------------------------------------------------------- multi-level atom

def _ml(velocity=1.0, nx=4, nz=9, scattering=0.0):
    atom = synth.hydrogen_like_atom(line_freq=5, cont_freq=3, seed=2)
    atm = synth.chromosphere(nx, nx, nz, atom, seed=2, velocity=velocity, scattering=scattering)
    return atm, atom


def test_multilevel_zero_flow_equals_static_path():
    """With u = 0 the weighted angle sums times the profile-free line weights
    equal the static sums times the static weights, frequency by frequency,
    so the rates and the MALI update agree."""
    atm, atom = _ml(velocity=0.0)
    p0 = O.MultiLevelProblem(atm, atom)
    n = p0.zero_radiation(1)
    J0, U0, t0 = p0.formal_solution(1, n)
    atm.vel = np.zeros((3,) + atm.shape)
    p1 = O.MultiLevelProblem(atm, atom)
    J1, U1, t1 = p1.formal_solution(1, n)
    for a, b in ((t1["qa"] * J1, t0["qa"] * J0), (t1["qb"] * J1, t0["qb"] * J0),
                 (t1["qe"] * U1, t0["qe"] * U0)):
        # on each frequency's scale: the sums differ in rounding order only
        err = np.max(np.abs(a - b), axis=1) / np.max(np.abs(b), axis=1)
        assert np.max(err) < 1e-12
    na, _ = p0.mali_sweep(1, n)
    nb, _ = p1.mali_sweep(1, n)
    # the rate solve amplifies the rounding-order differences of the sums
    assert O.max_rel_error(nb, na) < 1e-10


def test_multilevel_reversed_flow_gives_the_same_populations():
    """Line frequency grids are symmetric about line centre and continua do
    not shift, so reversing the flow permutes each line's profile values
    over its grid: the rates, and so the MALI iterates, do not change."""
    atm, atom = _ml()
    p = O.MultiLevelProblem(atm, atom)
    n = p.zero_radiation(1)
    na, _ = p.mali_sweep(1, n)
    na, _ = p.mali_sweep(1, na)
    atm.vel = -atm.vel
    q = O.MultiLevelProblem(atm, atom)
    nb, _ = q.mali_sweep(1, n)
    nb, _ = q.mali_sweep(1, nb)
    assert O.max_rel_error(nb, na) < 1e-10
    atm.vel = np.zeros_like(atm.vel)
    s = O.MultiLevelProblem(atm, atom)
    ns, _ = s.mali_sweep(1, n)
    ns, _ = s.mali_sweep(1, ns)
    assert O.max_rel_error(ns, na) > 1e-4


def test_multilevel_moving_conservation_and_fas():
    atm, atom = _ml(nx=8, nz=17, scattering=1.0)
    p = O.MultiLevelProblem(atm, atom, n_grids=2)
    n = p.zero_radiation(2)
    for _ in range(3):
        n, _ = p.mali_sweep(2, n)
        assert np.max(np.abs(n.sum(axis=0) / atm.n_tot - 1.0)) < 1e-13
    n_fas, _ = O.fas_solve(p, 1e-10, PARAMS, max_cycles=60)
    p1 = O.MultiLevelProblem(atm, atom, n_grids=1)
    n_mali = p1.zero_radiation(1)
    for _ in range(40):
        n_mali, _ = p1.mali_sweep(1, n_mali)
    assert O.max_rel_error(n_fas, n_mali) < 1e-9
    assert np.allclose(p.levels[1].vel, O.restrict_fw(atm.vel))
