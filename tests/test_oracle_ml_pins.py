"""Pins of the multi-level oracle (lines, bound-free continua, background).

* with one line, no continuum and no background it must reproduce the
  two-level oracle (itself pinned to closed forms in test_oracle_pins.py);
* with collisions dominating it must give Saha-Boltzmann populations;
* with the radiation field set to the Planck function (and no local
  operator) the radiative rates alone must be in detailed balance with the
  Saha-Boltzmann populations, transition by transition;
* particle conservation, the FAS fixed point, and MALI/FAS/FMG agreement;
* damped (Voigt) lines: the profile's closed forms, one damped line at
  T = t_ref equal to the damped two-level oracle, conservation and FAS.
"""

import math

import numpy as np
import pytest

from oracle import mg3d_oracle as O
from paper_1701_01607_gb300 import synth


def ml_box(nx=8, nz=17, seed=2, **kw):
    atom = synth.hydrogen_like_atom(line_freq=7, cont_freq=4, seed=seed)
    atm = synth.chromosphere(nx, nx, nz, atom, seed=seed, **kw)
    return atm, atom


def test_ml_reduces_to_two_level():
    atm2, atom2 = synth.stratified_two_level(8, 8, 17, eps=1e-2, sigma=0.3, seed=4)
    line = synth.Line(0, 1, 1.0, atom2.a_ul, atom2.kappa, atom2.n_freq, atom2.x_max)
    ml_atom = synth.MultiLevelAtom(g=np.array([1.0, 1.0]), theta=np.array([0.0, atom2.theta]),
                                   theta_ref=atom2.theta, lines=[line], continua=[],
                                   t_ref=5000.0)
    c = np.zeros((2, 2) + atm2.shape)
    c[1, 0] = atm2.c_ul
    c[0, 1] = atm2.c_ul * np.exp(-atom2.theta / atm2.T)
    ml_atm = synth.MultiLevelAtmosphere(atm2.nx, atm2.ny, atm2.nz, atm2.dx, atm2.dy, atm2.z,
                                        atm2.T, atm2.n_tot, np.zeros(atm2.shape), c,
                                        np.zeros((2,) + atm2.shape))
    p2 = O.TwoLevelProblem(atm2, atom2)
    pm = O.MultiLevelProblem(ml_atm, ml_atom)
    n2 = p2.zero_radiation(1)
    nm = pm.zero_radiation(1)
    assert np.allclose(nm, n2, rtol=1e-13)
    for _ in range(4):
        n2, c2 = p2.mali_sweep(1, n2)
        nm, cm = pm.mali_sweep(1, nm)
    assert np.allclose(nm, n2, rtol=1e-12)
    assert abs(cm - c2) < 1e-10


def test_ml_lte_limit():
    atm, atom = ml_box()
    atm.c = atm.c * 1e12
    p = O.MultiLevelProblem(atm, atom)
    n = p.zero_radiation(1)
    n, _ = p.mali_sweep(1, n)
    lte = p.lte_populations(1)
    assert np.allclose(n, lte, rtol=1e-9)


def test_ml_radiative_detailed_balance():
    atm, atom = ml_box(nx=2, nz=5)
    atm.c[:] = 0.0
    p = O.MultiLevelProblem(atm, atom)
    lte = p.lte_populations(1)
    terms, _ = p.transition_terms(1, lte)
    nvox = atm.T.size
    B = np.empty((len(p.freqs), nvox))
    T = atm.T.reshape(-1)
    for f, (kind, ti, xv, wv) in enumerate(p.freqs):
        rho = atom.lines[ti].rho if kind == "line" else atom.continua[ti].rho * xv
        B[f] = rho ** 3 / np.expm1(atom.theta_ref * rho / T)
    M = p.rate_matrix_from(1, B, np.ones_like(B), terms)
    W = p.apply(M, lte)
    # rows 1..N-1 vanish; compare with the size of the individual rates
    scale = np.abs(np.einsum("vij,jv->vi", np.abs(M), lte.reshape(p.N, -1))).T
    assert np.max(np.abs(W[1:].reshape(p.N - 1, -1)) / scale[1:]) < 1e-12
    assert np.allclose(W[0], atm.n_tot, rtol=1e-13)


def test_ml_conservation_and_positivity():
    atm, atom = ml_box()
    p = O.MultiLevelProblem(atm, atom)
    n = p.zero_radiation(1)
    for _ in range(3):
        n, _ = p.mali_sweep(1, n)
        assert np.allclose(n.sum(axis=0), atm.n_tot, rtol=1e-13)
        assert np.all(n > 0)


def test_ml_fas_fixed_point_and_agreement():
    atm, atom = ml_box(nx=8, nz=17)
    # the first cycle needs pre-smoothing from the zero-radiation start, as
    # the paper found for its hydrogen atom (nu0 >= 15, Table 1)
    params = dict(nu_fmg=8, nu0=10, nu1=2, nu2=4, nu3=16)
    p = O.MultiLevelProblem(atm, atom, n_grids=2)
    n_mali, it = O.mali_solve(p, 1e-11)
    n2, c2 = p.fas_cycle(n_mali, False, params)
    assert c2 < 1e-9
    p2 = O.MultiLevelProblem(atm, atom, n_grids=2)
    n_fas, cyc = O.fas_solve(p2, 1e-10, params)
    p3 = O.MultiLevelProblem(atm, atom, n_grids=2)
    n_fmg, cyc3 = O.fmg_solve(p3, 1e-10, params)
    assert O.max_rel_error(n_fas, n_mali) < 1e-8
    assert O.max_rel_error(n_fmg, n_mali) < 1e-8


# ------------------------------------------------- background scattering

def test_mean_intensity_of_constant_source():
    """Constant S everywhere and on both boundaries: I = S on every ray, so the
    mean intensity equals S whatever the opacity (pins the J accumulation)."""
    rng = np.random.default_rng(1)
    nf, nz, ny, nx = 3, 9, 4, 4
    chi = rng.uniform(0.1, 5.0, (nf, nz, ny, nx))
    S = 2.5
    mu, w = O.a4_quadrature()
    Jx, Ux, J = O.formal_solution_nu_raw(np.linspace(0.0, 8.0, nz), 1.0, 1.0, mu, w, chi, S,
                                         0.0, 0.0, S, S, want_j=True)
    assert np.max(np.abs(J - S)) < 1e-14
    assert np.max(np.abs(Jx - S)) < 1e-14     # sl = 0: Jx is J
    assert np.max(np.abs(Ux - 1.0)) < 1e-14   # fl = 0


def test_background_scattering_converges_to_direct_solve():
    """Lines and continua of negligible opacity in a background with equal
    absorption and coherent scattering (epsilon = 1/2): the background source
    function is S = eps B + (1 - eps) J at every frequency, which a dense
    solve with the Lambda matrix (built column by column from unit source
    functions) gives directly; repeated sweeps, each replacing the
    background field by the new mean intensity, must converge to it."""
    atom = synth.hydrogen_like_atom(line_freq=3, cont_freq=2, seed=2, kappa_line=1e-30,
                                    kappa_cont=1e-30)
    atm = synth.chromosphere(4, 4, 9, atom, seed=3, scattering=1.0)
    p = O.MultiLevelProblem(atm, atom)
    assert p.scatter
    n = p.zero_radiation(1)
    for _ in range(80):
        n, _ = p.mali_sweep(1, n)
    lev = p.levels[1]
    nz, ny, nx = lev.shape
    nvox = nx * ny * nz
    chi = (lev.chi_c + lev.sigma_c).reshape(-1)
    eps = (lev.chi_c / (lev.chi_c + lev.sigma_c)).reshape(-1)
    terms, Ib = p.transition_terms(1, n)
    mu, w = p.mu, p.wray
    for f, (kind, ti, xv, wv) in enumerate(p.freqs):
        if kind == "line":
            B = p.planck_rho(atom.lines[ti].rho, lev.T).reshape(-1)
        else:
            ct = atom.continua[ti]
            B = p.planck_rho(ct.rho * xv, lev.T).reshape(-1)

        def fs(S, ib):
            _, _, J = O.formal_solution_nu_raw(lev.z, lev.dx, lev.dy, mu, w,
                                               chi.reshape(1, nz, ny, nx),
                                               S.reshape(1, nz, ny, nx), 0.0, 0.0,
                                               ib.reshape(1, ny, nx), 0.0, want_j=True)
            return J.reshape(-1)

        Lam = np.empty((nvox, nvox))
        for i in range(nvox):
            e = np.zeros(nvox)
            e[i] = 1.0
            Lam[:, i] = fs(e, np.zeros(ny * nx))
        J_bc = fs(np.zeros(nvox), Ib[f])
        S = np.linalg.solve(np.eye(nvox) - (1.0 - eps)[:, None] * Lam,
                            eps * B + (1.0 - eps) * J_bc)
        J_direct = Lam @ S + J_bc
        assert np.max(np.abs(p.jbg[1][f] - J_direct) / J_direct) < 1e-10, f


def test_background_scattering_conservation_and_fas():
    """Scattering background: particle conservation in every sweep; FAS from
    the zero-radiation start converges (C < 1e-8) with the background field
    restricted on each coarse-grid entry, and FAS and FMG reach MALI's
    solution (the coarse field is frozen after its Lambda-iteration, so a
    converged fine solution gets no correction)."""
    atom = synth.hydrogen_like_atom(line_freq=5, cont_freq=3, seed=2)
    atm = synth.chromosphere(8, 8, 17, atom, seed=2, scattering=2.0)
    p = O.MultiLevelProblem(atm, atom, n_grids=2)
    n = p.zero_radiation(2)
    for _ in range(3):
        n, _ = p.mali_sweep(2, n)
        assert np.max(np.abs(n.sum(axis=0) / atm.n_tot - 1.0)) < 1e-13
    params = dict(nu_fmg=8, nu0=10, nu1=2, nu2=4, nu3=16)
    n, cyc = O.fas_solve(p, 1e-8, params, max_cycles=60)
    assert np.all(n > 0) and cyc < 60
    n, _ = O.fas_solve(O.MultiLevelProblem(atm, atom, n_grids=2), 1e-11, params)
    n_fmg, _ = O.fmg_solve(O.MultiLevelProblem(atm, atom, n_grids=2), 1e-11, params)
    p1 = O.MultiLevelProblem(atm, atom)
    n1 = p1.zero_radiation(1)
    for _ in range(40):
        n1, _ = p1.mali_sweep(1, n1)
    assert O.max_rel_error(n, n1) < 1e-9 and O.max_rel_error(n_fmg, n1) < 1e-9


# ------------------------------------------------------------ damped lines

def test_ml_line_profile_closed_forms():
    """phi(x; d, a) = H(a/d, x/d)/(sqrt(pi) d): the two-level profile at
    d = 1, the Doppler profile at a = 0, unit area at any d, and the line
    centre value exp(a'^2) erfc(a')/(sqrt(pi) d) with a' = a/d."""
    integrate = pytest.importorskip("scipy.integrate")
    x = np.linspace(-5.0, 5.0, 21)
    assert np.array_equal(O.ml_line_profile(x, 1.0, 0.05), O.line_profile(x, 0.05))
    for d in (0.7, 1.3):
        assert np.allclose(O.ml_line_profile(x, d, 0.0),
                           np.exp(-(x / d) ** 2) / (math.sqrt(math.pi) * d), rtol=1e-15)
        for a in (0.02, 0.4):
            ap = a / d
            ref = math.exp(ap * ap) * math.erfc(ap) / (math.sqrt(math.pi) * d)
            assert abs(O.ml_line_profile(0.0, d, a) / ref - 1.0) < 1e-13
            area = 2.0 * sum(integrate.quad(lambda v: float(O.ml_line_profile(v, d, a)), lo, hi,
                                            limit=400, epsabs=1e-13)[0]
                             for lo, hi in ((0.0, 6.0 * d), (6.0 * d, np.inf)))
            assert abs(area - 1.0) < 1e-9


def test_ml_damped_reduces_to_two_level_damped():
    """One damped line at T = t_ref (d = 1), no continuum, no background:
    the two-level oracle with the same Voigt profile."""
    a = 0.05
    atom2 = synth.TwoLevelAtom(a_damp=a, n_freq=13, x_max=5.0)
    atm2, atom2 = synth.stratified_two_level(8, 8, 17, eps=1e-2, sigma=0.3, seed=4, atom=atom2)
    assert np.all(atm2.T == 5000.0)
    line = synth.Line(0, 1, 1.0, atom2.a_ul, atom2.kappa, atom2.n_freq, atom2.x_max, a)
    ml_atom = synth.MultiLevelAtom(g=np.array([1.0, 1.0]), theta=np.array([0.0, atom2.theta]),
                                   theta_ref=atom2.theta, lines=[line], continua=[],
                                   t_ref=5000.0)
    c = np.zeros((2, 2) + atm2.shape)
    c[1, 0] = atm2.c_ul
    c[0, 1] = atm2.c_ul * np.exp(-atom2.theta / atm2.T)
    ml_atm = synth.MultiLevelAtmosphere(atm2.nx, atm2.ny, atm2.nz, atm2.dx, atm2.dy, atm2.z,
                                        atm2.T, atm2.n_tot, np.zeros(atm2.shape), c,
                                        np.zeros((2,) + atm2.shape))
    p2 = O.TwoLevelProblem(atm2, atom2)
    pm = O.MultiLevelProblem(ml_atm, ml_atom)
    n2 = p2.zero_radiation(1)
    nm = pm.zero_radiation(1)
    for _ in range(4):
        n2, c2 = p2.mali_sweep(1, n2)
        nm, cm = pm.mali_sweep(1, nm)
    assert np.allclose(nm, n2, rtol=1e-12)
    assert abs(cm - c2) < 1e-10
    # and the damping matters
    line.a_damp = 0.0
    pd = O.MultiLevelProblem(ml_atm, ml_atom)
    nd = pd.zero_radiation(1)
    for _ in range(4):
        nd, _ = pd.mali_sweep(1, nd)
    assert O.max_rel_error(nd, nm) > 1e-4


def test_ml_damped_conservation_multigrid_and_flow():
    atom = synth.hydrogen_like_atom(line_freq=9, cont_freq=4, seed=2, a_damp=0.03)
    atm = synth.chromosphere(8, 8, 17, atom, seed=2)
    p = O.MultiLevelProblem(atm, atom, n_grids=2)
    n = p.zero_radiation(2)
    for _ in range(3):
        n, _ = p.mali_sweep(2, n)
        assert np.allclose(n.sum(axis=0), atm.n_tot, rtol=1e-13)
        assert np.all(n > 0)
    params = dict(nu_fmg=8, nu0=10, nu1=2, nu2=4, nu3=16)
    n_mali, _ = O.mali_solve(O.MultiLevelProblem(atm, atom, n_grids=2), 1e-11)
    n_fas, _ = O.fas_solve(O.MultiLevelProblem(atm, atom, n_grids=2), 1e-10, params)
    assert O.max_rel_error(n_fas, n_mali) < 1e-8
    # zero flow takes the static damped path, frequency by frequency
    q0 = O.MultiLevelProblem(atm, atom)
    n0 = q0.zero_radiation(1)
    J0, U0, t0 = q0.formal_solution(1, n0)
    atm.vel = np.zeros((3,) + atm.shape)
    q1 = O.MultiLevelProblem(atm, atom)
    J1, U1, t1 = q1.formal_solution(1, n0)
    for a, b in ((t1["qa"] * J1, t0["qa"] * J0), (t1["qe"] * U1, t0["qe"] * U0)):
        err = np.max(np.abs(a - b), axis=1) / np.max(np.abs(b), axis=1)
        assert np.max(err) < 1e-12


# ------------------------------------------------- partial redistribution

def _two_level_pair(gamma, nx=8, nz=17):
    atom2 = synth.TwoLevelAtom(gamma_prd=gamma, n_freq=9, x_max=3.0)
    atm2, atom2 = synth.stratified_two_level(nx, nx, nz, eps=1e-2, sigma=0.3, seed=4, atom=atom2)
    line = synth.Line(0, 1, 1.0, atom2.a_ul, atom2.kappa, atom2.n_freq, atom2.x_max, 0.0, gamma)
    ml_atom = synth.MultiLevelAtom(g=np.array([1.0, 1.0]), theta=np.array([0.0, atom2.theta]),
                                   theta_ref=atom2.theta, lines=[line], continua=[],
                                   t_ref=5000.0)
    c = np.zeros((2, 2) + atm2.shape)
    c[1, 0] = atm2.c_ul
    c[0, 1] = atm2.c_ul * np.exp(-atom2.theta / atm2.T)
    ml_atm = synth.MultiLevelAtmosphere(atm2.nx, atm2.ny, atm2.nz, atm2.dx, atm2.dy, atm2.z,
                                        atm2.T, atm2.n_tot, np.zeros(atm2.shape), c,
                                        np.zeros((2,) + atm2.shape))
    return (atm2, atom2), (ml_atm, ml_atom)


def test_ml_prd_reduces_to_two_level_prd():
    """One PRD line at T = t_ref: the two-level PRD oracle (pinned on its
    own), through MALI sweeps and a V-cycle with its coarse-grid entry."""
    (atm2, atom2), (ml_atm, ml_atom) = _two_level_pair(0.9)
    p2 = O.TwoLevelProblem(atm2, atom2, n_grids=2)
    pm = O.MultiLevelProblem(ml_atm, ml_atom, n_grids=2)
    n2, nm = p2.zero_radiation(2), pm.zero_radiation(2)
    for _ in range(4):
        n2, c2 = p2.mali_sweep(2, n2)
        nm, cm = pm.mali_sweep(2, nm)
        assert abs(cm - c2) < 1e-12
    assert O.max_rel_error(nm, n2) < 1e-12
    params = dict(nu_fmg=4, nu0=4, nu1=2, nu2=2, nu3=32)
    n2, c2 = p2.fas_cycle(n2, False, params)
    nm, cm = pm.fas_cycle(nm, False, params)
    assert O.max_rel_error(nm, n2) < 1e-12 and abs(cm - c2) < 1e-12


def _ml_prd_box(gamma=1.0, nx=8, nz=17, line_freq=7):
    atom = synth.hydrogen_like_atom(line_freq=line_freq, cont_freq=4, seed=2, gamma_prd=gamma)
    atm = synth.chromosphere(nx, nx, nz, atom, seed=2, ground_collisions=1e-3)
    return atm, atom


def test_ml_prd_table_follows_the_continuous_kernel():
    """At every node the matrix is c_a R0(x_a, x_b) c_b with R0 the kernel
    erfc(max(|x|, |x'|)/d)/(2 d^2) at the node's Doppler width; on a fine
    grid the symmetric factors c tend to 1 (the kernel's marginal is the
    node's profile), so a wrong width scaling would show; the discrete
    marginals are the profile exactly."""
    special = pytest.importorskip("scipy.special")
    atm, atom = _ml_prd_box(line_freq=41)
    p = O.MultiLevelProblem(atm, atom)
    ti = p.prd_lines[0]
    R, wq, phi = p.prd_tables(1, ti)
    x = np.array([p.freqs[f][2] for f in p.line_freqs[ti]])
    d = np.sqrt(atm.T.reshape(-1) / atom.t_ref)
    assert d.min() < 0.95 and d.max() > 1.2
    ax = np.abs(x)
    R0 = 0.5 * special.erfc(np.maximum(ax[:, None], ax[None, :])[None] / d[:, None, None]) \
        / d[:, None, None] ** 2
    cc = R / R0                                    # c_a c_b
    c = np.sqrt(np.einsum("vaa->va", cc))
    assert np.allclose(cc, c[:, :, None] * c[:, None, :], rtol=1e-12)
    # inside |x| <= 3 (the grid ends at 4, where truncation of the kernel
    # shows): 4e-3 here, against 0.15 with R0 scaled by 1/d instead of 1/d^2
    # and 12 without the width
    assert np.max(np.abs(c[:, ax <= 3.0] - 1.0)) < 1e-2
    assert np.allclose(np.einsum("vab,va->vb", R, wq), phi, rtol=1e-12)


def test_ml_prd_ratio_conserves_photons_and_reduces_to_crd():
    atm, atom = _ml_prd_box()
    p = O.MultiLevelProblem(atm, atom)
    n = p.zero_radiation(1)
    terms, _ = p.transition_terms(1, n)
    rng = np.random.default_rng(3)
    p.jbg[1] = np.exp(rng.normal(size=p.jbg[1].shape))
    rho = p.prd_ratios(1, n, terms)
    assert set(rho) == set(p.prd_lines) and len(rho) == 2    # both resonance lines
    for ti, r in rho.items():
        _, wq, phi = p.prd_tables(1, ti)
        assert np.allclose(np.sum(wq * phi * r.T, axis=1), 1.0, rtol=0, atol=1e-13)
        assert np.max(np.abs(r - 1.0)) > 1e-3
    # a field flat across each line: rho = 1
    for ti, fs in p.line_freqs.items():
        p.jbg[1][fs] = p.jbg[1][fs[0]]
    for r in p.prd_ratios(1, n, terms).values():
        assert np.max(np.abs(r - 1.0)) < 1e-13
    # vanishing coherence takes the CRD path
    atm2, atom0 = _ml_prd_box(gamma=0.0)
    atm3, atom_eps = _ml_prd_box(gamma=1e-14)
    q0, q1 = O.MultiLevelProblem(atm2, atom0), O.MultiLevelProblem(atm3, atom_eps)
    m0, m1 = q0.zero_radiation(1), q1.zero_radiation(1)
    for _ in range(3):
        m0, _ = q0.mali_sweep(1, m0)
        m1, _ = q1.mali_sweep(1, m1)
    assert O.max_rel_error(m1, m0) < 1e-12


def test_ml_prd_conservation_multigrid_and_effect():
    atm, atom = _ml_prd_box(nx=4, nz=9)
    p = O.MultiLevelProblem(atm, atom, n_grids=2)
    n = p.zero_radiation(2)
    for _ in range(3):
        n, _ = p.mali_sweep(2, n)
        assert np.allclose(n.sum(axis=0), atm.n_tot, rtol=1e-13)
        assert np.all(n > 0)
    params = dict(nu_fmg=8, nu0=10, nu1=2, nu2=4, nu3=16)
    n_mali, _ = O.mali_solve(O.MultiLevelProblem(atm, atom, n_grids=2), 1e-11)
    n_fas, _ = O.fas_solve(O.MultiLevelProblem(atm, atom, n_grids=2), 1e-10, params)
    n_fmg, _ = O.fmg_solve(O.MultiLevelProblem(atm, atom, n_grids=2), 1e-10, params)
    assert O.max_rel_error(n_fas, n_mali) < 1e-8
    assert O.max_rel_error(n_fmg, n_mali) < 1e-8
    _, crd_atom = _ml_prd_box(gamma=0.0, nx=4, nz=9)
    n_crd, _ = O.mali_solve(O.MultiLevelProblem(atm, crd_atom, n_grids=2), 1e-11)
    assert O.max_rel_error(n_crd, n_mali) > 1e-4


def test_ml_prd_in_a_flow_with_background_scattering():
    """In a flow the PRD lines keep their comoving field apart from the
    observer-frame field that background scattering reads: zero flow equals
    the static path, MALI stays positive, FAS meets MALI."""
    atom = synth.hydrogen_like_atom(line_freq=7, cont_freq=4, seed=2, gamma_prd=1.0)
    atm = synth.chromosphere(4, 4, 9, atom, seed=2, ground_collisions=1e-3, scattering=1.0)
    ps = O.MultiLevelProblem(atm, atom)
    ns = ps.zero_radiation(1)
    atm.vel = np.zeros((3,) + atm.shape)
    pm = O.MultiLevelProblem(atm, atom)
    nm = pm.zero_radiation(1)
    for _ in range(3):
        ns, _ = ps.mali_sweep(1, ns)
        nm, _ = pm.mali_sweep(1, nm)
    assert O.max_rel_error(nm, ns) < 1e-10
    assert set(pm.jcm[1]) == set(pm.prd_lines) and not ps.jcm[1]
    vatm = synth.chromosphere(4, 4, 9, atom, seed=2, ground_collisions=1e-2, scattering=1.0,
                              velocity=1.0)
    p = O.MultiLevelProblem(vatm, atom, n_grids=2)
    n = p.zero_radiation(2)
    for _ in range(3):
        n, _ = p.mali_sweep(2, n)
        assert np.allclose(n.sum(axis=0), vatm.n_tot, rtol=1e-13)
        assert np.all(n > 0)
    params = dict(nu_fmg=8, nu0=10, nu1=2, nu2=4, nu3=16)
    n_mali, _ = O.mali_solve(O.MultiLevelProblem(vatm, atom, n_grids=2), 1e-11)
    n_fas, _ = O.fas_solve(O.MultiLevelProblem(vatm, atom, n_grids=2), 1e-10, params)
    assert O.max_rel_error(n_fas, n_mali) < 1e-8


def test_ml_prd_with_background_scattering_shares_the_lagged_field():
    """PRD lines and background scattering read the same lagged field; the
    start Lambda-iterates it (scattering), conservation holds and FAS meets
    MALI."""
    atom = synth.hydrogen_like_atom(line_freq=7, cont_freq=4, seed=2, gamma_prd=1.0)
    atm = synth.chromosphere(4, 4, 9, atom, seed=2, ground_collisions=1e-3, scattering=1.0)
    p = O.MultiLevelProblem(atm, atom, n_grids=2)
    assert p.scatter and p.prd_lines and p.lagged
    n = p.zero_radiation(2)
    assert np.any(p.jbg[2] > 0)          # the start's Lambda-iteration
    for _ in range(3):
        n, _ = p.mali_sweep(2, n)
        assert np.allclose(n.sum(axis=0), atm.n_tot, rtol=1e-13)
    params = dict(nu_fmg=8, nu0=10, nu1=2, nu2=4, nu3=16)
    n_mali, _ = O.mali_solve(O.MultiLevelProblem(atm, atom, n_grids=2), 1e-11)
    n_fas, _ = O.fas_solve(O.MultiLevelProblem(atm, atom, n_grids=2), 1e-10, params)
    assert O.max_rel_error(n_fas, n_mali) < 1e-8


def test_ml_damped_prd_reduces_to_two_level_damped_prd():
    """One damped PRD line at T = t_ref: the two-level oracle with R_II-A and
    the Voigt profile, through MALI sweeps and a V-cycle."""
    a, g = 0.05, 1.0
    atom2 = synth.TwoLevelAtom(gamma_prd=g, a_damp=a, n_freq=9, x_max=4.0)
    atm2, atom2 = synth.stratified_two_level(4, 4, 9, eps=1e-2, sigma=0.3, seed=4, atom=atom2)
    line = synth.Line(0, 1, 1.0, atom2.a_ul, atom2.kappa, atom2.n_freq, atom2.x_max, a, g)
    ml_atom = synth.MultiLevelAtom(g=np.array([1.0, 1.0]), theta=np.array([0.0, atom2.theta]),
                                   theta_ref=atom2.theta, lines=[line], continua=[],
                                   t_ref=5000.0)
    c = np.zeros((2, 2) + atm2.shape)
    c[1, 0] = atm2.c_ul
    c[0, 1] = atm2.c_ul * np.exp(-atom2.theta / atm2.T)
    ml_atm = synth.MultiLevelAtmosphere(atm2.nx, atm2.ny, atm2.nz, atm2.dx, atm2.dy, atm2.z,
                                        atm2.T, atm2.n_tot, np.zeros(atm2.shape), c,
                                        np.zeros((2,) + atm2.shape))
    p2 = O.TwoLevelProblem(atm2, atom2, n_grids=2)
    pm = O.MultiLevelProblem(ml_atm, ml_atom, n_grids=2)
    n2, nm = p2.zero_radiation(2), pm.zero_radiation(2)
    for _ in range(3):
        n2, c2 = p2.mali_sweep(2, n2)
        nm, cm = pm.mali_sweep(2, nm)
        assert abs(cm - c2) < 1e-12
    params = dict(nu_fmg=4, nu0=4, nu1=2, nu2=2, nu3=32)
    n2, _ = p2.fas_cycle(n2, False, params)
    nm, _ = pm.fas_cycle(nm, False, params)
    assert O.max_rel_error(nm, n2) < 1e-12


def test_ml_damped_prd_table_follows_the_continuous_kernel():
    """At nodes of different Doppler widths d the damped table is
    c_a R0(x_a, x_b) c_b with R0 = R_II-A(x/d, x'/d; a/d)/d^2; inside the grid
    the symmetric factors stay near 1 (1 % here, where the Lorentz wings are
    cut at 6 Doppler widths; 15 % or more with a wrong width scaling) and
    the discrete marginals are the node's Voigt profile."""
    a = 0.05
    atom = synth.hydrogen_like_atom(line_freq=31, cont_freq=3, seed=2, gamma_prd=1.0,
                                    a_damp=a, x_max=6.0)
    atm = synth.chromosphere(1, 1, 3, atom, seed=2, ground_collisions=1e-3)
    p = O.MultiLevelProblem(atm, atom)
    ti = p.prd_lines[0]
    R, wq, phi = p.prd_tables(1, ti)
    x = np.array([p.freqs[f][2] for f in p.line_freqs[ti]])
    d = np.sqrt(atm.T.reshape(-1) / atom.t_ref)
    assert d.min() < 0.95 and d.max() > 1.3
    kernel = lambda i, j, dv: O.redistribution_r2a(x[i] / dv, x[j] / dv, a / dv) / dv ** 2
    inner = np.flatnonzero(np.abs(x) <= 3.0)
    for v, dv in enumerate(d):
        c = {i: math.sqrt(R[v, i, i] / kernel(i, i, dv)) for i in inner}
        assert max(abs(ci - 1.0) for ci in c.values()) < 3e-2
        for i, j in ((inner[0], inner[-1]), (inner[2], inner[len(inner) // 2])):
            assert abs(R[v, i, j] / (c[i] * c[j] * kernel(i, j, dv)) - 1.0) < 1e-12
    assert np.allclose(np.einsum("vab,va->vb", R, wq), phi, rtol=1e-12)


def test_ml_prd_in_a_flow_reduces_to_two_level_moving_prd():
    """One PRD line at T = t_ref in a flow: the two-level oracle with
    comoving-frame redistribution (itself pinned by its zero-flow and
    uniform-flow limits), through MALI sweeps and a V-cycle."""
    (atm2, atom2), (ml_atm, ml_atom) = _two_level_pair(0.9, nx=4, nz=9)
    vatm, _ = synth.stratified_two_level(4, 4, 9, eps=1e-2, sigma=0.3, seed=4, atom=atom2,
                                         velocity=1.0)
    atm2.vel = vatm.vel
    ml_atm.vel = vatm.vel.copy()
    p2 = O.TwoLevelProblem(atm2, atom2, n_grids=2)
    pm = O.MultiLevelProblem(ml_atm, ml_atom, n_grids=2)
    n2, nm = p2.zero_radiation(2), pm.zero_radiation(2)
    for _ in range(3):
        n2, c2 = p2.mali_sweep(2, n2)
        nm, cm = pm.mali_sweep(2, nm)
        assert abs(cm - c2) < 1e-12
    params = dict(nu_fmg=4, nu0=4, nu1=2, nu2=2, nu3=32)
    n2, _ = p2.fas_cycle(n2, False, params)
    nm, _ = pm.fas_cycle(nm, False, params)
    assert O.max_rel_error(nm, n2) < 1e-12


def test_ml_prd_in_a_flow_zero_flow_conservation_and_fas():
    atm, atom = _ml_prd_box(nx=4, nz=9)
    ps = O.MultiLevelProblem(atm, atom)
    ns = ps.zero_radiation(1)
    atm.vel = np.zeros((3,) + atm.shape)
    pm = O.MultiLevelProblem(atm, atom)
    nm = pm.zero_radiation(1)
    for _ in range(3):
        ns, _ = ps.mali_sweep(1, ns)
        nm, _ = pm.mali_sweep(1, nm)
    assert O.max_rel_error(nm, ns) < 1e-10
    vatm = synth.chromosphere(4, 4, 9, atom, seed=2, ground_collisions=1e-3, velocity=1.0)
    p = O.MultiLevelProblem(vatm, atom, n_grids=2)
    n = p.zero_radiation(2)
    for _ in range(3):
        n, _ = p.mali_sweep(2, n)
        assert np.allclose(n.sum(axis=0), vatm.n_tot, rtol=1e-13)
        assert np.all(n > 0)
    params = dict(nu_fmg=8, nu0=10, nu1=2, nu2=4, nu3=16)
    n_mali, _ = O.mali_solve(O.MultiLevelProblem(vatm, atom, n_grids=2), 1e-11)
    n_fas, _ = O.fas_solve(O.MultiLevelProblem(vatm, atom, n_grids=2), 1e-10, params)
    assert O.max_rel_error(n_fas, n_mali) < 1e-8
