"""Pins of the oracle's cubic Hermite operators (Sec. 3 and Sec. 4.5).

The monotone cubic Hermite interpolant with Fritsch-Butland slopes is what
scipy's PchipInterpolator implements, so the slopes, the 1D interpolant, the
successive-pass 3D prolongation and the 2D upwind interpolation of the short
characteristics are each compared with scipy applied pass by pass.  Closed
forms (exact transport at whole-cell offsets, horizontally homogeneous
columns, linear data) and the range property of monotone interpolation pin
the rest.
"""

import numpy as np
import pytest

from oracle import mg3d_oracle as O
from paper_1701_01607_gb300 import synth

interpolate = pytest.importorskip("scipy.interpolate")

PARAMS = dict(nu_fmg=4, nu0=4, nu1=2, nu2=2, nu3=32)


# ------------------------------------------------------------- 1D slopes

def test_slopes_match_scipy_pchip_nonuniform():
    rng = np.random.default_rng(11)
    for n in (2, 3, 5, 17):
        x = np.cumsum(rng.uniform(0.2, 2.0, n))
        # monotone stretches, extrema, a flat run and a sign change
        y = rng.normal(size=(4, n))
        if n >= 5:
            y[1, 1:3] = y[1, 1]
            y[2] = np.sort(y[2])
            y[3] = -y[3] ** 2
        d = O.pchip_slopes(y, np.diff(x), periodic=False)
        ref = interpolate.PchipInterpolator(x, y, axis=-1).derivative()(x)
        assert np.allclose(d, ref, rtol=1e-13, atol=1e-13), n


def test_hermite_eval_matches_scipy_between_nodes():
    rng = np.random.default_rng(12)
    x = np.cumsum(rng.uniform(0.3, 1.5, 9))
    y = rng.uniform(-1, 3, 9)
    d = O.pchip_slopes(y, np.diff(x), periodic=False)
    spl = interpolate.PchipInterpolator(x, y)
    for i in range(8):
        for t in (0.0, 0.17, 0.5, 0.9):
            h = x[i + 1] - x[i]
            got = O.hermite_eval(y[i], y[i + 1], d[i], d[i + 1], h, t)
            assert abs(got - spl(x[i] + t * h)) < 1e-13


def test_periodic_slopes_equal_pchip_on_tiled_row():
    rng = np.random.default_rng(13)
    n = 8
    y = rng.uniform(0, 2, n)
    d = O.pchip_slopes(y, np.ones(n), periodic=True)
    xt = np.arange(3 * n, dtype=float)
    ref = interpolate.PchipInterpolator(xt, np.tile(y, 3)).derivative()(xt[n:2 * n])
    assert np.allclose(d, ref, rtol=1e-13, atol=1e-14)


# --------------------------------------------------- 3D prolongation (Sec. 4.5)

def _scipy_prolong(ac, z_fine):
    """x (periodic), then y (periodic), then z: scipy PCHIP along each axis."""
    nzc, nyc, nxc = ac.shape[-3:]
    xs = np.arange(3 * nxc, dtype=float)
    a = interpolate.PchipInterpolator(xs, np.concatenate([ac] * 3, axis=-1), axis=-1)(
        nxc + np.arange(2 * nxc) / 2.0)
    ys = np.arange(3 * nyc, dtype=float)
    a = interpolate.PchipInterpolator(ys, np.concatenate([a] * 3, axis=-2), axis=-2)(
        nyc + np.arange(2 * nyc) / 2.0)
    return interpolate.PchipInterpolator(z_fine[::2], a, axis=-3)(z_fine)


def test_prolong_hermite_matches_scipy_passes():
    rng = np.random.default_rng(14)
    z = np.cumsum(np.r_[0.0, rng.uniform(0.5, 1.5, 16)])       # 17 fine planes
    ac = np.exp(rng.normal(size=(2, 9, 4, 6)))
    got = O.prolong_hermite(ac, z)
    assert got.shape == (2, 17, 8, 12)
    assert np.allclose(got, _scipy_prolong(ac, z), rtol=1e-13, atol=1e-14)


def test_prolong_hermite_stays_in_cell_range_and_keeps_nodes():
    """Each pass keeps values between the two coarse values of the interval,
    so a fine value lies within its 2 x 2 x 2 coarse cell (no new extrema, no
    negative populations from positive ones); coincident nodes are exact."""
    rng = np.random.default_rng(15)
    z = np.cumsum(np.r_[0.0, rng.uniform(0.2, 2.0, 12)])
    ac = np.exp(3.0 * rng.normal(size=(7, 5, 5)))
    f = O.prolong_hermite(ac, z)
    nzc, nyc, nxc = ac.shape
    assert np.array_equal(f[::2, ::2, ::2], ac)
    for k in range(f.shape[0]):
        ks = {k // 2, min((k + 1) // 2, nzc - 1)}
        for j in range(f.shape[1]):
            js = {j // 2 % nyc, (j + 1) // 2 % nyc}
            for i in range(f.shape[2]):
                is_ = {i // 2 % nxc, (i + 1) // 2 % nxc}
                cell = ac[np.ix_(sorted(ks), sorted(js), sorted(is_))]
                assert cell.min() * (1 - 1e-14) <= f[k, j, i] <= cell.max() * (1 + 1e-14)


def test_prolong_hermite_exact_on_linear_z_and_constants():
    z = np.array([0.0, 0.4, 1.0, 1.9, 3.0, 3.2, 4.5, 5.0, 7.0])
    zc = z[::2]
    ac = np.broadcast_to((2.0 + 0.7 * zc)[:, None, None], (5, 3, 4)).copy()
    f = O.prolong_hermite(ac, z)
    assert np.allclose(f, (2.0 + 0.7 * z)[:, None, None], rtol=1e-14)
    assert np.allclose(O.prolong_hermite(np.full((5, 3, 4), 3.25), z), 3.25, rtol=1e-15)


# ------------------------------------------- upwind interpolation (Sec. 3)

def test_sc_hermite_one_step_is_scipy_bicubic():
    """With chi = 0 and S = 0 one step carries the bottom pattern unchanged
    to the upwind point, so plane 1 holds the 2D interpolant of the bottom
    plane: x pass on the rows, then the y pass, each a periodic PCHIP."""
    mu, wr = O.a4_quadrature()
    nx, ny = 8, 6
    rng = np.random.default_rng(16)
    Ib = rng.uniform(0.2, 3.0, size=(1, ny, nx))
    z = np.array([0.0, 0.7])
    chi = np.zeros((1, 2, ny, nx))
    for interp in (0, 1):
        _, _, _, I = O.formal_solution_raw(z, 1.3, 0.9, mu, wr, chi, 0.0, 1.0, Ib, 0.0, True,
                                           interp=interp)
        tiled = np.tile(Ib[0], (3, 3))
        xs, ys = np.arange(3 * nx, dtype=float), np.arange(3 * ny, dtype=float)
        for r in range(12):
            s = 0.7 / mu[r, 2]
            xu = nx + np.arange(nx) - s * mu[r, 0] / 1.3
            yu = ny + np.arange(ny) - s * mu[r, 1] / 0.9
            if interp:
                rows = interpolate.PchipInterpolator(xs, tiled, axis=1)(xu)     # [3ny, nx]
                ref = np.empty((ny, nx))
                for i in range(nx):
                    ref[:, i] = interpolate.PchipInterpolator(ys, rows[:, i])(yu)
            else:
                ref = interpolate.RegularGridInterpolator((ys, xs), tiled)(
                    np.stack(np.meshgrid(yu, xu, indexing="ij"), axis=-1))
            assert np.allclose(I[r, 0, 1], ref, rtol=1e-13, atol=1e-14), (interp, r)


def test_sc_hermite_transport_at_whole_cells_is_exact():
    """dz = (b/a) dx moves the (a, a, b) rays one whole cell per step: the
    Hermite interpolant returns node values there, so the pattern arrives
    shifted and attenuated exactly."""
    mu, wr = O.a4_quadrature()
    a, b = np.min(np.abs(mu)), np.max(np.abs(mu))
    nx = ny = 8
    nz = 7
    z = np.arange(nz) * (b / a)
    Ib = np.random.default_rng(5).uniform(0.5, 2.0, size=(1, ny, nx))
    chi = np.full((1, nz, ny, nx), 0.05)
    _, _, _, I = O.formal_solution_raw(z, 1.0, 1.0, mu, wr, chi, 0.0, 1.0, Ib, 0.0, True,
                                       interp=1)
    checked = 0
    for r in range(12):
        mx, my, mz = mu[r]
        if abs(mz - b) > 1e-12:
            continue
        sx, sy = int(round(np.sign(mx))), int(round(np.sign(my)))
        for k in range(nz):
            expect = np.roll(Ib[0], shift=(k * sy, k * sx), axis=(0, 1))
            expect = expect * np.exp(-0.05 * z[k] / mz)
            assert np.allclose(I[r, 0, k], expect, rtol=1e-12, atol=1e-14)
        checked += 1
    assert checked == 4


def test_sc_hermite_homogeneous_equals_closed_form():
    """Horizontally homogeneous planes: any interpolation returns the plane
    value, and the columns follow I = S + (I_in - S) exp(-tau) exactly."""
    nz = 17
    z = np.linspace(0, 8.0, nz)
    mu, wr = O.a4_quadrature()
    chi_z = 5.0 * np.exp(-z / 1.5)
    chi = np.broadcast_to(chi_z[None, :, None, None], (1, nz, 4, 4)).copy()
    S0, Ib = 1.7, 2.9
    _, _, _, I = O.formal_solution_raw(z, 1.0, 1.0, mu, wr, chi, S0, 1.0, Ib, 0.0, True,
                                       interp=1)
    tau_b = np.r_[0.0, np.cumsum(0.5 * (chi_z[1:] + chi_z[:-1]) * np.diff(z))]
    for r in range(24):
        mz = mu[r, 2]
        exact = (S0 + (Ib - S0) * np.exp(-tau_b / mz) if mz > 0
                 else S0 - S0 * np.exp(-(tau_b[-1] - tau_b) / abs(mz)))
        assert np.allclose(I[r, 0], exact[:, None, None], rtol=1e-12, atol=1e-14)


def _advect_error(n, interp):
    """Transport (chi = 0) of sin(2 pi x/n) sin(2 pi y/n) over n steps of 0.3
    cells along the (a, a, b) rays; max error at the top against the exact
    shifted pattern."""
    mu, wr = O.a4_quadrature()
    a, b = np.min(np.abs(mu)), np.max(np.abs(mu))
    dz = 0.3 * b / a
    z = np.arange(n + 1) * dz
    xx = np.arange(n)
    pat = lambda x, y: 1.5 + 0.5 * np.sin(2 * np.pi * x / n)[None, :] * \
        np.sin(2 * np.pi * y / n)[:, None]
    Ib = pat(xx, xx)[None]
    chi = np.zeros((1, n + 1, n, n))
    _, _, _, I = O.formal_solution_raw(z, 1.0, 1.0, mu, wr, chi, 0.0, 1.0, Ib, 0.0, True,
                                       interp=interp)
    err = 0.0
    for r in range(12):
        mx, my, mz = mu[r]
        if abs(mz - b) > 1e-12:
            continue
        shift = 0.3 * n
        exact = pat(xx - np.sign(mx) * shift, xx - np.sign(my) * shift)
        err = max(err, np.max(np.abs(I[r, 0, n] - exact)))
    return err


def test_sc_hermite_advects_smooth_pattern_more_accurately():
    """Linear interpolation damps a resolved mode by O(h^2) per step, so over
    the n steps of a fixed shift its error falls as O(h); the monotone cubic
    Hermite interpolant (slopes limited to zero at the extrema) has the same
    order here but stays about three times closer to the exact shifted
    pattern (measured: 0.35-0.38 of the linear error at 16 and 32 cells per
    wavelength)."""
    el16, eh16 = _advect_error(16, 0), _advect_error(16, 1)
    el32, eh32 = _advect_error(32, 0), _advect_error(32, 1)
    assert eh16 < 0.45 * el16, (eh16, el16)
    assert eh32 < 0.45 * el32, (eh32, el32)
    assert el16 / el32 > 1.6 and eh16 / eh32 > 1.4, (el16 / el32, eh16 / eh32)


# ------------------------------------- iterations with the Hermite operators

def _problem(n_grids, nx=8, nz=17, eps=1e-2, **kw):
    atm, atom = synth.stratified_two_level(nx, nx, nz, eps=eps, tau_bottom=1e3, sigma=0.3,
                                           seed=3)
    return O.TwoLevelProblem(atm, atom, n_grids=n_grids, **kw), atm, atom


def test_hermite_fas_fixed_point_and_conservation():
    """Hermite upwind interpolation and Hermite prolongation: populations are
    conserved in every sweep and a V-cycle leaves a converged solution
    unchanged (the interpolated correction of zero is zero)."""
    prob, atm, atom = _problem(3, eps=0.1, interpolation=1, sc_interp=1)
    n = prob.zero_radiation(3)
    for it in range(3000):
        n, C = prob.mali_sweep(3, n)
        if it < 3:
            assert np.max(np.abs(n.sum(axis=0) / atm.n_tot - 1.0)) < 1e-13
        if C < 1e-14:
            break
    assert C < 1e-13
    _, C2 = prob.fas_cycle(n, False, PARAMS)
    assert C2 < 1e-11


def test_hermite_mali_fas_fmg_same_solution():
    """With Hermite upwind interpolation MALI, FAS and FMG (Hermite or
    trilinear prolongation) converge to one discrete solution, which differs
    from the linear scheme's by the discretisation difference only."""
    kw = dict(nx=4, nz=9, eps=3e-2)
    prob, atm, atom = _problem(3, sc_interp=1, **kw)
    n_mali, _ = O.mali_solve(prob, 1e-11)
    out = []
    for interp in (0, 1):
        p2 = O.TwoLevelProblem(atm, atom, n_grids=3, interpolation=interp, sc_interp=1)
        out.append(O.fas_solve(p2, 1e-11, PARAMS)[0])
    p3 = O.TwoLevelProblem(atm, atom, n_grids=3, interpolation=1, sc_interp=1)
    out.append(O.fmg_solve(p3, 1e-11, PARAMS)[0])
    for n in out:
        assert O.max_rel_error(n, n_mali) < 1e-8
    n_lin, _ = O.mali_solve(_problem(3, **kw)[0], 1e-11)
    d = O.max_rel_error(n_lin, n_mali)
    assert 1e-6 < d < 0.2, d


def test_hermite_multilevel_conservation_and_agreement():
    """The multi-level atom with both Hermite operators: particle conservation
    in every sweep, and MALI and 2-grid FAS reach the same populations."""
    atom = synth.hydrogen_like_atom(line_freq=5, cont_freq=3, seed=2)
    atm = synth.chromosphere(4, 4, 9, atom, seed=2)
    p = O.MultiLevelProblem(atm, atom, n_grids=2, interpolation=1, sc_interp=1)
    n = p.zero_radiation(2)
    for _ in range(3):
        n, _ = p.mali_sweep(2, n)
        assert np.max(np.abs(n.sum(axis=0) / atm.n_tot - 1.0)) < 1e-13
    n_fas, _ = O.fas_solve(p, 1e-10, PARAMS, max_cycles=60)
    p1 = O.MultiLevelProblem(atm, atom, n_grids=1, sc_interp=1)
    n_mali, _ = O.mali_solve(p1, 1e-11)
    assert O.max_rel_error(n_fas, n_mali) < 1e-8
