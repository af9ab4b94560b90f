"""Pins of the CPU oracle against closed forms, invariants and library routines.

None of these compares the oracle with itself: each checks it against a
result fixed by the mathematics (exact transfer solutions that the linear short
characteristics must reproduce, the LTE limit, the sqrt(eps) law, a dense
solve of the discrete Lambda operator, scipy's own interpolators and
convolution) so that a dropped term, a swapped weight, a wrong sign of an
upwind shift or a transposed index fails at least one test.
"""

import math

import numpy as np
import pytest

from oracle import mg3d_oracle as O
from paper_1701_01607_gb300 import synth


# ---------------------------------------------------------------- quadrature

def test_a4_moments():
    mu, w = O.a4_quadrature()
    assert mu.shape == (24, 3)
    assert np.allclose(np.sum(mu * mu, axis=1), 1.0, atol=1e-15)
    assert abs(w.sum() - 1.0) < 1e-15
    for i in range(3):
        assert abs(np.sum(w * mu[:, i])) < 1e-15
        assert abs(np.sum(w * mu[:, i] ** 2) - 1.0 / 3.0) < 1e-15
        # the A4 parameter is fixed by integrating mu^4 exactly
        assert abs(np.sum(w * mu[:, i] ** 4) - 0.2) < 1e-15
        for j in range(3):
            if i != j:
                assert abs(np.sum(w * mu[:, i] * mu[:, j])) < 1e-15
    # the value commonly tabulated for the 24-direction level-symmetric set
    assert abs(np.min(np.abs(mu)) - 0.3500212) < 1e-7
    assert abs(np.max(np.abs(mu)) - 0.8688903) < 1e-7
    assert np.all(mu[:12, 2] > 0) and np.all(mu[12:, 2] < 0)


def test_frequency_grid_normalised_and_symmetric():
    x, phi, wphi = O.frequency_grid(9, 3.0)
    assert abs(wphi.sum() - 1.0) < 1e-15
    assert np.allclose(x, -x[::-1])
    assert np.allclose(wphi, wphi[::-1])
    assert abs(x[1] - x[0] - 0.75) < 1e-15
    # trapezoid: interior weights equal, end weights half
    w = wphi / phi
    assert np.allclose(w[1:-1], w[1]) and abs(w[0] - 0.5 * w[1]) < 1e-15


# --------------------------------------------------- formal solution, exact

def _slab(nz=9, ny=4, nx=4, z=None):
    if z is None:
        z = np.cumsum(np.r_[0.0, np.linspace(0.3, 1.7, nz - 1)])   # non-uniform
    return z, nx, ny


def test_fs_constant_source_matches_closed_form():
    """Constant chi and S: I = S + (I_in - S) exp(-tau_path) for every ray."""
    z, nx, ny = _slab()
    nz = len(z)
    chi0, S0, Ib, It = 0.7, 2.5, 4.0, 0.5
    mu, wr = O.a4_quadrature()
    chi = np.full((1, nz, ny, nx), chi0)
    _, _, _, I = O.formal_solution_raw(z, 1.0, 1.0, mu, wr, chi, S0, 1.0, Ib, It, True)
    for r in range(24):
        mz = mu[r, 2]
        if mz > 0:
            path = (z - z[0]) / mz
            exact = S0 + (Ib - S0) * np.exp(-chi0 * path)
        else:
            path = (z[-1] - z) / abs(mz)
            exact = S0 + (It - S0) * np.exp(-chi0 * path)
        got = I[r, 0, :, 2, 1]
        assert np.allclose(got, exact, rtol=1e-13, atol=1e-13), r


def test_fs_linear_source_matches_closed_form():
    """S linear in height and chi constant: the linear SC step is exact.

    Up ray at height z_k entering at z_0 with I_b, path optical depth
    T = chi (z_k - z_0)/mu, S = a + b z:
        I = I_b e^-T + (a + b z_k)(1 - e^-T) - (b mu/chi)(1 - e^-T (1 + T)).
    A swap of w_0 and w_up, or a wrong sign in either, fails this.
    """
    z, nx, ny = _slab(nz=11)
    nz = len(z)
    chi0, a, b, Ib, It = 1.3, 0.4, 0.9, 3.0, 0.2
    mu, wr = O.a4_quadrature()
    chi = np.full((1, nz, ny, nx), chi0)
    S = np.broadcast_to((a + b * z)[None, :, None, None], chi.shape)
    _, _, _, I = O.formal_solution_raw(z, 1.0, 1.0, mu, wr, chi, S, 1.0, Ib, It, True)
    for r in range(24):
        mz = abs(mu[r, 2])
        if mu[r, 2] > 0:
            T = chi0 * (z - z[0]) / mz
            exact = (Ib * np.exp(-T) + (a + b * z) * (1 - np.exp(-T))
                     - (b * mz / chi0) * (1 - np.exp(-T) * (1 + T)))
        else:
            # going down, S decreases along the path: slope -b per unit height
            T = chi0 * (z[-1] - z) / mz
            exact = (It * np.exp(-T) + (a + b * z) * (1 - np.exp(-T))
                     + (b * mz / chi0) * (1 - np.exp(-T) * (1 + T)))
        assert np.allclose(I[r, 0, :, 1, 2], exact, rtol=1e-12, atol=1e-13), r


def test_fs_horizontal_transport_of_a_pattern():
    """Pure absorption of a random bottom pattern along the (a, a, b) rays.

    With dz = (b/a) dx each step moves those rays exactly one cell in x and y,
    so bilinear interpolation is exact and the pattern must arrive shifted by
    k cells (periodically) and attenuated by exp(-chi k dz / b).
    """
    mu, wr = O.a4_quadrature()
    a = np.min(np.abs(mu))
    b = np.max(np.abs(mu))
    nx = ny = 8
    nz = 7
    z = np.arange(nz) * (b / a)
    rng = np.random.default_rng(5)
    Ib = rng.uniform(0.5, 2.0, size=(1, ny, nx))
    chi0 = 0.05
    chi = np.full((1, nz, ny, nx), chi0)
    _, _, _, I = O.formal_solution_raw(z, 1.0, 1.0, mu, wr, chi, 0.0, 1.0, Ib, 0.0, True)
    checked = 0
    for r in range(12):
        mx, my, mz = mu[r]
        if abs(abs(mz) - b) > 1e-12:
            continue
        sx, sy = int(round(np.sign(mx))), int(round(np.sign(my)))
        for k in range(nz):
            expect = np.roll(Ib[0], shift=(k * sy, k * sx), axis=(0, 1))
            expect = expect * np.exp(-chi0 * (z[k] - z[0]) / mz)
            assert np.allclose(I[r, 0, k], expect, rtol=1e-12, atol=1e-14), (r, k)
        checked += 1
    assert checked == 4


def test_homogeneous_3d_equals_plane_parallel_closed_form():
    """Horizontally homogeneous 3D box, exponential opacity, constant S.

    With S constant the transfer solution along any ray is
    I = S + (I_in - S) exp(-tau_path) for the discrete trapezoid optical depth,
    independent of x and y.  Every column must equal it.
    """
    nz = 17
    z = np.linspace(0, 8.0, nz)
    mu, wr = O.a4_quadrature()
    chi_z = 5.0 * np.exp(-z / 1.5)
    chi = np.broadcast_to(chi_z[None, :, None, None], (2, nz, 4, 4)).copy()
    chi[1] *= 0.3
    S0, Ib = 1.7, 2.9
    _, _, _, I = O.formal_solution_raw(z, 1.0, 1.0, mu, wr, chi, S0, 0.5, Ib, 0.0, True)
    dtau_z = 0.5 * (chi_z[1:] + chi_z[:-1]) * np.diff(z)
    tau_from_bottom = np.r_[0.0, np.cumsum(dtau_z)]
    tau_from_top = tau_from_bottom[-1] - tau_from_bottom
    for f, scale in ((0, 1.0), (1, 0.3)):
        for r in range(24):
            mz = mu[r, 2]
            if mz > 0:
                exact = S0 + (Ib - S0) * np.exp(-scale * tau_from_bottom / mz)
            else:
                exact = S0 + (0.0 - S0) * np.exp(-scale * tau_from_top / abs(mz))
            col = I[r, f]
            assert np.allclose(col, exact[:, None, None], rtol=1e-12, atol=1e-14)


# --------------------------------------------- two-level physics and MALI

def _small_problem(nx=4, nz=9, eps=1e-2, n_grids=1, tau_bottom=1e3, sigma=0.0, seed=3):
    atm, atom = synth.stratified_two_level(nx, nx, nz, eps=eps, tau_bottom=tau_bottom,
                                           sigma=sigma, seed=seed)
    return O.TwoLevelProblem(atm, atom, n_grids=n_grids), atm, atom


def test_zero_radiation_start_closed_form():
    prob, atm, atom = _small_problem()
    n = prob.zero_radiation(1)
    ratio = n[1] / n[0]
    c_lu = atm.c_ul * atom.g_ratio * np.exp(-atom.theta / atm.T)
    assert np.allclose(ratio, c_lu / (atom.a_ul + atm.c_ul), rtol=1e-14)
    assert np.allclose(n.sum(axis=0), atm.n_tot, rtol=1e-14)


def test_lte_limit_one_sweep():
    """eps -> 1 (collisions dominate): one sweep gives Boltzmann populations."""
    prob, atm, atom = _small_problem()
    lev = prob.levels[1]
    lev.c_ul[:] = 1e12 * atom.a_ul
    n = prob.zero_radiation(1)
    n, _ = prob.mali_sweep(1, n)
    boltz = atom.g_ratio * np.exp(-atom.theta / atm.T)
    assert np.allclose(n[1] / n[0], boltz, rtol=1e-11)
    S = n[1] / (atom.g_ratio * n[0] - n[1])
    assert np.allclose(S, prob.planck(atm.T), rtol=1e-11)


def test_mali_sweep_equals_source_function_form():
    """The population-form update equals S = ((1-eps) Jeff + eps B)/(1-(1-eps) Lambda*)."""
    prob, atm, atom = _small_problem(nx=4, nz=9, eps=3e-2)
    n0 = prob.zero_radiation(1)
    n0, _ = prob.mali_sweep(1, n0)
    _, Jeff, U = prob.formal_solution(1, n0)
    n1, _ = prob.mali_sweep(1, n0)
    epsp = atm.c_ul * (-np.expm1(-atom.theta / atm.T)) / atom.a_ul
    eps = epsp / (1 + epsp)
    B = prob.planck(atm.T)
    lam = 1.0 - U
    S_expect = ((1 - eps) * Jeff + eps * B) / (1 - (1 - eps) * lam)
    S_got = n1[1] / (atom.g_ratio * n1[0] - n1[1])
    assert np.allclose(S_got, S_expect, rtol=1e-12)


def test_conservation_every_sweep():
    prob, atm, _ = _small_problem(sigma=0.3)
    n = prob.zero_radiation(1)
    for _ in range(4):
        n, _ = prob.mali_sweep(1, n)
        assert np.allclose(n.sum(axis=0), atm.n_tot, rtol=1e-14, atol=0)


def test_dense_lambda_solve_matches_converged_mali():
    """Converged MALI equals the direct solve of the discrete problem.

    At the converged populations the opacity is frozen; the Lambda operator is
    built column by column (unit source at one node, no incoming radiation),
    the boundary term by a run with S = 0, and
        (I - diag(1-eps) Lambda) S = eps B + (1 - eps) J_bc
    is solved by LU.  The diagonal of Lambda must also equal 1 - U.
    """
    prob, atm, atom = _small_problem(nx=2, nz=9, eps=5e-2, tau_bottom=1e2, sigma=0.2)
    lev = prob.levels[1]
    n = prob.zero_radiation(1)
    for _ in range(400):
        n, C = prob.mali_sweep(1, n)
        if C < 1e-13:
            break
    assert C < 1e-12
    chi, S = prob.opacity_source(lev, n)
    nf = chi.shape[0]
    shape = lev.shape
    nvox = S.size
    chi4 = chi.reshape((nf,) + shape)
    wphi = prob.wphi[:, None, None, None]
    zeros_bc = np.zeros((nf, lev.ny, lev.nx))
    Lam = np.empty((nvox, nvox))
    for j in range(nvox):
        e = np.zeros(nvox)
        e[j] = 1.0
        Jb, _, _ = O.formal_solution_raw(lev.z, lev.dx, lev.dy, prob.mu, prob.wray, chi4,
                                         e.reshape(shape)[None], wphi, zeros_bc, zeros_bc)
        Lam[:, j] = Jb.reshape(-1)
    Ib = np.broadcast_to(prob.planck(lev.T[0])[None], (nf, lev.ny, lev.nx))
    Jbc, _, U = O.formal_solution_raw(lev.z, lev.dx, lev.dy, prob.mu, prob.wray, chi4,
                                      np.zeros((1,) + shape), wphi, Ib, zeros_bc)
    assert np.allclose(np.diag(Lam), 1.0 - U.reshape(-1), rtol=1e-13, atol=1e-15)
    epsp = (lev.c_ul * (-np.expm1(-atom.theta / lev.T)) / atom.a_ul).reshape(-1)
    eps = epsp / (1 + epsp)
    B = prob.planck(lev.T).reshape(-1)
    A = np.eye(nvox) - (1 - eps)[:, None] * Lam
    S_direct = np.linalg.solve(A, eps * B + (1 - eps) * Jbc.reshape(-1))
    assert np.allclose(S, S_direct, rtol=1e-10)


def test_sqrt_eps_law_under_refinement():
    """Isothermal, no incident radiation: S(0) -> sqrt(eps) B as the grid refines.

    The top node sits at line-centre tau = 1e-4.  The error of the surface
    source function must fall monotonically with resolution (points per
    decade of tau) and be below 2 % at 16 points per decade.
    """
    eps = 1e-2
    decades = 7  # tau from 1e-4 to 1e3
    errs = []
    for ppd in (2, 4, 8, 16):
        nz = ppd * decades + 1
        if nz % 2 == 0:
            nz += 1
        atm, atom = synth.stratified_two_level(2, 2, nz, eps=eps, tau_bottom=1e3)
        prob = O.TwoLevelProblem(atm, atom, n_grids=1)
        n = prob.zero_radiation(1)
        for _ in range(5000):
            n, C = prob.mali_sweep(1, n)
            if C < 1e-9:
                break
        S = n[1] / (atom.g_ratio * n[0] - n[1])
        errs.append(abs(S[-1, 0, 0] / prob.planck(5000.0) / math.sqrt(eps) - 1.0))
    assert all(b < a for a, b in zip(errs, errs[1:])), errs
    assert errs[-1] < 0.02, errs


# ------------------------------------------------------- grid transfer

def test_restriction_identities_and_scipy():
    from scipy import ndimage
    rng = np.random.default_rng(0)
    f = rng.uniform(1, 2, size=(9, 8, 8))
    c = O.restrict_fw(f)
    assert c.shape == (5, 4, 4)
    assert np.allclose(O.restrict_fw(np.full((9, 8, 8), 3.25)), 3.25, rtol=1e-15)
    # interior coarse planes equal a 3x3x3 convolution with the (1/4,1/2,1/4)^3
    # kernel, periodic in x and y, sampled at even nodes
    w1 = np.array([0.25, 0.5, 0.25])
    kern = w1[:, None, None] * w1[None, :, None] * w1[None, None, :]
    conv = ndimage.convolve(f, kern, mode="wrap")
    assert np.allclose(c[1:-1], conv[2:-2:2, ::2, ::2], rtol=1e-14)
    # boundary planes: injection in z, (1/4,1/2,1/4)^2 in x, y
    k2 = w1[:, None] * w1[None, :]
    for K, kf in ((0, 0), (4, 8)):
        plane = ndimage.convolve(f[kf], k2, mode="wrap")[::2, ::2]
        assert np.allclose(c[K], plane, rtol=1e-14)
    # a z-independent field keeps its horizontal sum up to the factor 4
    g = np.broadcast_to(rng.uniform(size=(1, 8, 8)), (9, 8, 8))
    assert np.allclose(O.restrict_fw(g).sum(axis=(1, 2)), g[0].sum() / 4.0, rtol=1e-14)


def test_prolongation_matches_scipy_trilinear():
    from scipy.interpolate import RegularGridInterpolator
    rng = np.random.default_rng(1)
    nzc, nyc, nxc = 5, 4, 6
    z_fine = np.cumsum(np.r_[0.0, rng.uniform(0.5, 1.5, size=2 * nzc - 2)])
    zc = z_fine[::2]
    ac = rng.uniform(-1, 1, size=(nzc, nyc, nxc))
    fine = O.prolong_trilinear(ac, z_fine)
    assert fine.shape == (2 * nzc - 1, 2 * nyc, 2 * nxc)
    # periodic padding in x and y for the library interpolator
    pad = np.concatenate([ac, ac[:, :1, :]], axis=1)
    pad = np.concatenate([pad, pad[:, :, :1]], axis=2)
    interp = RegularGridInterpolator((zc, np.arange(nyc + 1) * 2.0, np.arange(nxc + 1) * 2.0),
                                     pad, method="linear")
    Z, Y, X = np.meshgrid(z_fine, np.arange(2 * nyc) * 1.0, np.arange(2 * nxc) * 1.0,
                          indexing="ij")
    ref = interp(np.stack([Z, Y, X], axis=-1))
    assert np.allclose(fine, ref, rtol=1e-13, atol=1e-14)
    # exact for fields linear in height
    lin = 2.0 + 0.5 * zc[:, None, None] + 0 * ac
    assert np.allclose(O.prolong_trilinear(lin, z_fine),
                       (2.0 + 0.5 * z_fine)[:, None, None], rtol=1e-14)


# ------------------------------------------------------ multigrid

PARAMS = dict(nu_fmg=16, nu0=0, nu1=2, nu2=2, nu3=32)


def test_fas_fixed_point_invariance():
    """A V-cycle leaves a converged solution unchanged: R(r) = 0, e = 0."""
    prob, atm, atom = _small_problem(nx=8, nz=17, eps=1e-2, n_grids=3, sigma=0.3)
    n = prob.zero_radiation(3)
    for _ in range(3000):
        n, C = prob.mali_sweep(3, n)
        if C < 1e-14:
            break
    assert C < 1e-13
    n2, C2 = prob.fas_cycle(n, False, PARAMS)
    assert C2 < 1e-11


def test_mali_fas_fmg_same_solution():
    """MALI, FAS and FMG converged tightly reach the same discrete solution, and
    the V-cycle contracts the correction faster per cycle than MALI per sweep."""
    prob, atm, atom = _small_problem(nx=8, nz=17, eps=1e-2, n_grids=3, sigma=0.3)
    h_mali, h_fas = [], []
    n_mali, _ = O.mali_solve(prob, 1e-11, history=h_mali)
    prob2 = O.TwoLevelProblem(atm, atom, n_grids=3)
    n_fas, cyc = O.fas_solve(prob2, 1e-11, PARAMS, history=h_fas)
    prob3 = O.TwoLevelProblem(atm, atom, n_grids=3)
    n_fmg, cyc2 = O.fmg_solve(prob3, 1e-11, PARAMS)
    assert O.max_rel_error(n_fas, n_mali) < 1e-8
    assert O.max_rel_error(n_fmg, n_mali) < 1e-8
    rho_mali = h_mali[-1] / h_mali[-2]
    rho_fas = h_fas[-1] / h_fas[-2]
    assert rho_fas < 0.5 and rho_fas < rho_mali, (rho_fas, rho_mali)


def test_half_weighting_and_injection():
    from scipy import ndimage
    rng = np.random.default_rng(4)
    f = rng.uniform(1, 2, size=(2, 9, 8, 6))
    inj = O.restrict_inj(f)
    assert np.array_equal(inj, f[:, ::2, ::2, ::2])
    hw = O.restrict_hw(f)
    assert np.allclose(O.restrict_hw(np.full((9, 8, 6), 2.5)), 2.5, rtol=1e-15)
    k3 = np.zeros((3, 3, 3))
    k3[1, 1, 1] = 0.5
    for (a, b, c) in ((0, 1, 1), (2, 1, 1), (1, 0, 1), (1, 2, 1), (1, 1, 0), (1, 1, 2)):
        k3[a, b, c] = 1.0 / 12.0
    for comp in range(2):
        conv = ndimage.convolve(f[comp], k3, mode="wrap")
        assert np.allclose(hw[comp, 1:-1], conv[2:-2:2, ::2, ::2], rtol=1e-14)
        k2 = np.zeros((3, 3))
        k2[1, 1] = 0.5
        k2[0, 1] = k2[2, 1] = k2[1, 0] = k2[1, 2] = 0.125
        for K, kf in ((0, 0), (4, 8)):
            plane = ndimage.convolve(f[comp, kf], k2, mode="wrap")[::2, ::2]
            assert np.allclose(hw[comp, K], plane, rtol=1e-14)


def test_fas_converges_with_each_restriction():
    """All three restrictions give a convergent FAS on a smooth problem with
    the same fixed point (the restriction changes only the path)."""
    atm, atom = synth.stratified_two_level(8, 8, 17, eps=1e-2, sigma=0.3, seed=9)
    sols = []
    for mode in (0, 1, 2):
        prob = O.TwoLevelProblem(atm, atom, n_grids=3, restriction=mode)
        n, cyc = O.fas_solve(prob, 1e-10, dict(nu_fmg=8, nu0=0, nu1=2, nu2=2, nu3=32))
        sols.append(n)
    for n in sols[1:]:
        assert O.max_rel_error(n, sols[0]) < 1e-7


def _mali_history(nz, eps=1e-3, nx=4):
    atm, atom = synth.stratified_two_level(nx, nx, nz, eps=eps, sigma=0.3, seed=3)
    n_inf, it = O.mali_solve(O.TwoLevelProblem(atm, atom), 1e-14)
    p = O.TwoLevelProblem(atm, atom)
    n = p.zero_radiation(1)
    C, E = [], []
    for _ in range(it):
        n, c = p.mali_sweep(1, n)
        C.append(c)
        E.append(O.max_rel_error(n, n_inf))
    return np.array(C), np.array(E)


def test_mali_error_estimate_of_eq13_and_spectral_radius():
    """In the asymptotic linear regime the true error follows
    E_i = rho/(1 - rho) C_i with rho estimated as C_(i+1)/C_i (Eq. 13 and the
    estimate after it), and that rho is the operational spectral radius
    E_(i+1)/E_i (Eq. 12); one-grid MALI's spectral radius grows as the grid
    is refined (Sec. 4.13)."""
    radii = []
    for nz in (17, 33):
        C, E = _mali_history(nz)
        sel = (C[:-1] < 1e-4) & (C[:-1] > 1e-9)
        assert sel.sum() >= 10
        rho_c = C[1:] / C[:-1]
        rho_e = E[1:] / E[:-1]
        est = rho_c / (1.0 - rho_c) * C[:-1]
        assert np.max(np.abs(est[sel] / E[:-1][sel] - 1.0)) < 1e-3
        assert np.max(np.abs(rho_c[sel] / rho_e[sel] - 1.0)) < 1e-3
        radii.append(float(np.median(rho_c[sel])))
    assert 0.5 < radii[0] < radii[1] < 1.0


def test_multigrid_spectral_radius_nearly_independent_of_grid_spacing():
    """Sec. 4.13: unlike one-grid MALI, whose spectral radius grows as the
    grid is refined (so its iterations per decade of error roughly double
    from 17 to 33 nodes per column), the V-cycle's stays nearly constant when
    a grid is added over the same coarsest grid."""
    params = dict(nu_fmg=4, nu0=4, nu1=2, nu2=2, nu3=32)
    per_decade = {}
    for nz, ng in ((17, 2), (33, 3)):
        atm, atom = synth.stratified_two_level(4, 4, nz, eps=1e-3, sigma=0.3, seed=3)
        n_inf, _ = O.fas_solve(O.TwoLevelProblem(atm, atom, n_grids=ng), 1e-13, params)
        p = O.TwoLevelProblem(atm, atom, n_grids=ng)
        n = p.zero_radiation(ng)
        E = []
        for cyc in range(6):
            n, _ = p.fas_cycle(n, cyc == 0, params)
            E.append(O.max_rel_error(n, n_inf))
        rho = float(np.median(np.array(E[2:]) / np.array(E[1:-1])))
        assert rho < 0.35
        per_decade[nz] = -1.0 / math.log10(rho)
    C17, _ = _mali_history(17)
    C33, _ = _mali_history(33)
    mali = {nz: -1.0 / math.log10(float(np.median((C[1:] / C[:-1])[(C[:-1] < 1e-4) &
                                                                       (C[:-1] > 1e-9)])))
            for nz, C in ((17, C17), (33, C33))}
    assert mali[33] / mali[17] > 2.0
    assert per_decade[33] / per_decade[17] < 1.5


def test_zero_radiation_start_gives_a_smoother_error_than_lte():
    """Sec. 4.11: after the first MALI sweeps the error left by the
    zero-radiation start is smoother than the one left by an LTE start; the
    smoothing number of Sec. 4.11, the largest second difference of
    (n_i - n_inf)/n_inf (here along z, x and y), is several times smaller."""
    atm, atom = synth.stratified_two_level(4, 4, 33, eps=1e-3, sigma=0.3, seed=3)
    n_inf, _ = O.mali_solve(O.TwoLevelProblem(atm, atom), 1e-13)

    def smoothing_number(n):
        e = (n - n_inf) / n_inf
        d2 = np.abs(e[:, 2:] - 2.0 * e[:, 1:-1] + e[:, :-2]).max()
        for ax in (2, 3):
            d2 = max(d2, np.abs(np.roll(e, 1, ax) - 2.0 * e + np.roll(e, -1, ax)).max())
        return d2

    r = atom.g_ratio * np.exp(-atom.theta / atm.T)
    starts = {"zero": O.TwoLevelProblem(atm, atom).zero_radiation(1),
              "lte": np.stack([atm.n_tot / (1.0 + r), atm.n_tot * r / (1.0 + r)])}
    hist = {}
    for name, n in starts.items():
        p = O.TwoLevelProblem(atm, atom)
        hist[name] = []
        for _ in range(8):
            n, _ = p.mali_sweep(1, n)
            hist[name].append(smoothing_number(n))
    ratio = np.array(hist["lte"]) / np.array(hist["zero"])
    assert np.all(ratio[1:] > 3.0), ratio


def test_threaded_formal_solution_equals_the_serial_loop():
    """The all-cores timing entry (rays on several host threads, partial sums
    added in ray order) computes the serial loop's Jbar, Jeff and U up to the
    association of the sums."""
    atm, atom = synth.stratified_two_level(8, 8, 17, eps=1e-3, sigma=0.3, seed=12)
    p = O.TwoLevelProblem(atm, atom)
    n = p.zero_radiation(1)
    serial = p.formal_solution(1, n)
    p.threads = 4
    threaded = p.formal_solution(1, n)
    for a, b in zip(threaded, serial):
        assert float(np.max(np.abs(a - b) / np.abs(b))) < 1e-13
