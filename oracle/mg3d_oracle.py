"""CPU oracle for the multigrid non-LTE 3D radiative-transfer hot path (FP64).

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
CPU-baseline / reference legs of ``bench.py`` may import this module.  It shares
no code with the CUDA library: the formal solution is the plain C loop nest in
``oracle/fs_oracle.c`` and everything else is written out here in numpy.  The
only thing both sides consume in common is the seeded input generator
``paper_1701_01607_gb300.synth`` (atmosphere arrays and atom parameters).

What each function follows in the paper (Bjorgen & Leenaarts 2017):

* ``a4_quadrature``     -- the 24-direction Carlson A4 set (Sec. 3).  The paper
  does not print its values.  Reading: three directions per octant, the
  permutations of (a, a, b) with 2a^2 + b^2 = 1 and equal weights 1/24; ``a``
  is fixed by integrating mu^4 exactly, 2a^4 + b^4 = 3/5 (a = 0.3500212).
* ``frequency_grid``    -- CRD Doppler profile sampled at equidistant offsets
  with trapezoid weights, renormalised so that sum(w phi) = 1 (reading; the
  paper only states CRD).
* ``formal_solution``   -- short characteristics with linear or Hermite-spline
  upwind interpolation (Sec. 3) accumulating Jbar, Jeff = Jbar - Lambda* S and
  U = 1 - Lambda*.
* ``rate_matrix`` / ``W`` -- statistical equilibrium (Eq. 2) with the first
  rate equation replaced by particle conservation (Eq. 3), so that
  W(n) = f with f = (n_tot, 0, ..., 0) (Eq. 4 and the f vector after it).
  Radiative rates carry the diagonal-operator preconditioning of Rybicki &
  Hummer (1991) that MALI uses (Sec. 2.1, Sec. 3).
* ``mali_sweep``        -- one MALI (Jacobi) iteration; ``max_rel_change`` is
  C_i of Sec. 3.3.
* ``restrict_fw``       -- full-weighting restriction (Sec. 4.4), 27 points.
* ``prolong_trilinear`` -- trilinear interpolation (Sec. 4.5).
* ``prolong_hermite``   -- monotone cubic Hermite interpolation, the paper's
  other interpolation operator (Sec. 4.5), as successive 1D passes x, y, z.
* ``vcycle``            -- FAS V-cycle, Eqs. 5-11 and the recursion of Sec. 2.2
  with nu_1 pre-, nu_2 post-smoothing, nu_3 coarse iterations, nu_0 in the
  first cycle (Sec. 4.12) and the 10 % fix for negative populations (Sec. 4.10).
* ``fmg_solve``         -- full multigrid (Sec. 2.3, Fig. 1).
* ``MultiLevelProblem`` -- the multi-level atom (Eqs. 2-4 with lines, continua
  and a grey background, Sec. 3.2), with optional background coherent
  scattering whose field is lagged, Lambda-iterated at the zero-radiation
  start and on each coarse-grid entry, and held on coarse grids (Sec. 4.8).
* ``formal_solution_moving`` -- moving atmospheres (both atom kinds): the
  profile seen along ray r shifted by mu_r . u and renormalised per node and
  ray (the paper's Bifrost atmospheres move; Sec. 3.1, Sec. 6).
* ``prd_matrix`` / ``formal_solution_prd`` -- partial redistribution for the
  two-level atom (the next step of Sec. 6): angle-averaged Doppler
  redistribution mixed with CRD, S_f = rho_f S from the lagged field; in a
  flow (``_formal_solution_moving_prd``) the redistribution happens in each
  node's comoving frame and each ray reads rho at its shifted offsets.
* ``MultiLevelProblem.prd_ratios`` / ``prd_tables`` -- partial redistribution
  of multi-level lines, the two-level reading generalised: R_I-A at each
  node's Doppler width, f_rad from the plain lagged rates into the upper
  level, the emissivity and the transition's share of chi scaled by rho.
* ``line_profile`` / ``ml_line_profile`` -- Doppler or, with damping, Voigt
  profiles (the paper's atoms have damped lines); a multi-level line's
  damping parameter scales as 1/d with the node's Doppler width d.

Readings where the paper is silent (the same readings hold on the GPU path):
full weighting at the fixed z boundaries injects in z; n_before of Eq. 10 is
R(n^k) as it enters level k-1; the negative fix applies per (level, node)
whenever n_old (1 + I(e)) <= 0; W(n) on the right of Eq. 9 is evaluated in
the preconditioned form Gamma(Jeff(n), U(n)) n, which equals the unpreconditioned
rates at n by algebra.

Parity pins: quadrature moments, closed-form slab intensities, the LTE limit,
the sqrt(eps) law, horizontally homogeneous 3D = plane-parallel closed form,
the dense Lambda-matrix solve, FAS fixed-point invariance, agreement of MALI,
FAS and FMG, transfer-operator identities and particle conservation (see
tests/test_oracle_*.py).
"""

from __future__ import annotations

import ctypes
import dataclasses
import math
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_BUILD = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_BUILD, "liboracle.so")
_lib = None


def build(force: bool = False) -> str:
    """Compile oracle/fs_oracle.c into oracle/_build/liboracle.so (plain gcc,
    with OpenMP for the all-cores timing entry when the compiler has it)."""
    src = os.path.join(_HERE, "fs_oracle.c")
    if (not force and os.path.exists(_LIB_PATH)
            and os.path.getmtime(_LIB_PATH) >= os.path.getmtime(src)):
        return _LIB_PATH
    os.makedirs(_BUILD, exist_ok=True)
    tmp = _LIB_PATH + f".tmp{os.getpid()}"
    base = ["gcc", "-O2", "-std=c99", "-shared", "-fPIC", "-o", tmp, src, "-lm"]
    try:
        subprocess.check_call(base + ["-fopenmp"], stderr=subprocess.DEVNULL)
    except subprocess.CalledProcessError:
        subprocess.check_call(base)
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _load():
    global _lib
    if _lib is None:
        lib = ctypes.CDLL(build())
        d = ctypes.POINTER(ctypes.c_double)
        lib.orc_formal_solution.restype = ctypes.c_int
        lib.orc_formal_solution.argtypes = [
            ctypes.c_long, ctypes.c_long, ctypes.c_long, ctypes.c_double, ctypes.c_double,
            d, ctypes.c_long, d, d, ctypes.c_long, d, d, d, d, d, d, d, d, d, ctypes.c_int]
        lib.orc_formal_solution_threads.restype = ctypes.c_int
        lib.orc_formal_solution_threads.argtypes = [
            ctypes.c_long, ctypes.c_long, ctypes.c_long, ctypes.c_double, ctypes.c_double,
            d, ctypes.c_long, d, d, ctypes.c_long, d, d, d, d, d, d, d, d, ctypes.c_int,
            ctypes.c_int]
        lib.orc_max_threads.restype = ctypes.c_int
        lib.orc_max_threads.argtypes = []
        lib.orc_formal_solution_nu.restype = ctypes.c_int
        lib.orc_formal_solution_nu.argtypes = [
            ctypes.c_long, ctypes.c_long, ctypes.c_long, ctypes.c_double, ctypes.c_double,
            d, ctypes.c_long, d, d, ctypes.c_long, d, d, d, d, d, d, d, d, d, ctypes.c_int]
        _lib = lib
    return _lib


def max_threads() -> int:
    """Host threads the oracle's OpenMP runtime offers (1 without OpenMP)."""
    return int(_load().orc_max_threads())


def _ptr(a):
    if a is None:
        return None
    assert a.dtype == np.float64 and a.flags["C_CONTIGUOUS"]
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


# --------------------------------------------------------------------------
# Angle and frequency quadrature
# --------------------------------------------------------------------------

def a4_quadrature(a: float | None = None):
    """Carlson A4 set: 24 unit vectors and weights (Sec. 3).

    Three directions per octant, the permutations of (a, a, b) with
    2a^2 + b^2 = 1.  By default a^2 is the root of 6a^4 - 4a^2 + 2/5 = 0
    (from 2a^4 + b^4 = 3/5) that keeps b real.  Rays 0-11 point up (mu_z > 0).
    """
    if a is None:
        a = math.sqrt((4.0 - math.sqrt(6.4)) / 12.0)
    b = math.sqrt(1.0 - 2.0 * a * a)
    dirs = []
    for sz in (1.0, -1.0):
        for sy in (1.0, -1.0):
            for sx in (1.0, -1.0):
                for (cx, cy, cz) in ((b, a, a), (a, b, a), (a, a, b)):
                    dirs.append((sx * cx, sy * cy, sz * cz))
    mu = np.array(dirs, dtype=np.float64)
    w = np.full(len(dirs), 1.0 / len(dirs))
    return mu, w


def line_profile(x, a: float = 0.0):
    """phi(x) per unit Doppler width: exp(-x^2)/sqrt(pi), or for damping
    a > 0 the Voigt profile H(a, x)/sqrt(pi), H(a, x) = Re w(x + i a) with w
    the Faddeeva function."""
    x = np.asarray(x, dtype=np.float64)
    if a > 0.0:
        from scipy.special import wofz
        return wofz(x + 1j * a).real / math.sqrt(math.pi)
    return np.exp(-x * x) / math.sqrt(math.pi)


def ml_line_profile(x, d, a: float = 0.0):
    """A multi-level line's profile per unit reference Doppler width at
    offset x (reference widths) at a node whose Doppler width is d reference
    widths: phi(x/d; a/d)/d with phi = ``line_profile``.  The damping width
    does not scale with temperature, so the node's damping parameter is a/d
    (a given at t_ref)."""
    x = np.asarray(x, dtype=np.float64)
    d = np.asarray(d, dtype=np.float64)
    if a > 0.0:
        from scipy.special import wofz
        return wofz(x / d + 1j * (a / d)).real / (math.sqrt(math.pi) * d)
    return np.exp(-(x / d) ** 2) / (math.sqrt(math.pi) * d)


def frequency_grid(n_freq: int, x_max: float, a_damp: float = 0.0):
    """Frequency grid: offsets x, profile phi(x) (``line_profile``), weights.

    The weights are the trapezoid rule on equidistant x in [-x_max, x_max],
    scaled so that sum_nu w phi = 1 exactly (with damping this renormalises
    the Lorentzian wings cut at x_max).  Returns (x, phi, wphi) with
    wphi = w * phi.
    """
    if n_freq == 1:
        x = np.zeros(1)
        phi = line_profile(x, a_damp)
        w = np.ones(1)
    else:
        x = np.linspace(-x_max, x_max, n_freq)
        h = x[1] - x[0]
        w = np.full(n_freq, h)
        w[0] *= 0.5
        w[-1] *= 0.5
        phi = line_profile(x, a_damp)
    wphi = w * phi
    wphi = wphi / wphi.sum()
    return x, phi, wphi


def formal_solution_raw(z, dx, dy, mu, wray, chi, S, wphi, I_bottom, I_top,
                        want_intensity=False, interp=0):
    """Formal solution for given chi, S [nfreq, nz, ny, nx] (Sec. 3).

    ``wphi`` [nfreq, nz, ny, nx] weights the frequency sum; ``I_bottom`` and
    ``I_top`` [nfreq, ny, nx] are the entering intensities; ``interp`` picks
    the upwind interpolation (0 bilinear, 1 monotone cubic Hermite).  Returns
    (Jbar, Jeff, U) [nz, ny, nx] and, if asked, I [nrays, nfreq, nz, ny, nx].
    """
    chi = np.ascontiguousarray(chi, dtype=np.float64)
    nf, nz, ny, nx = chi.shape
    S = np.ascontiguousarray(np.broadcast_to(S, chi.shape), dtype=np.float64)
    wphi = np.ascontiguousarray(np.broadcast_to(wphi, chi.shape), dtype=np.float64)
    Ib = np.ascontiguousarray(np.broadcast_to(I_bottom, (nf, ny, nx)), dtype=np.float64)
    It = np.ascontiguousarray(np.broadcast_to(I_top, (nf, ny, nx)), dtype=np.float64)
    mu = np.ascontiguousarray(mu, dtype=np.float64)
    wray = np.ascontiguousarray(wray, dtype=np.float64)
    z = np.ascontiguousarray(z, dtype=np.float64)
    Jbar = np.empty((nz, ny, nx))
    Jeff = np.empty((nz, ny, nx))
    U = np.empty((nz, ny, nx))
    I = np.empty((len(wray), nf, nz, ny, nx)) if want_intensity else None
    rc = _load().orc_formal_solution(nx, ny, nz, float(dx), float(dy), _ptr(z), len(wray),
                                     _ptr(mu), _ptr(wray), nf, _ptr(chi), _ptr(S),
                                     _ptr(wphi), _ptr(Ib), _ptr(It), _ptr(Jbar), _ptr(Jeff),
                                     _ptr(U), _ptr(I), int(interp))
    if rc != 0:
        raise RuntimeError("oracle formal solution failed")
    if want_intensity:
        return Jbar, Jeff, U, I
    return Jbar, Jeff, U


def read_shifted(v, y, x, outside):
    """v [nf, nvox] given on the equidistant frequency grid x [nf], read at
    offsets y [nf, nvox] by linear interpolation; beyond the grid the edge
    value (outside None) or the constant ``outside``."""
    nf = len(x)
    if nf == 1:
        return v.copy()
    h = x[1] - x[0]
    p = (y - x[0]) / h
    i = np.clip(np.floor(p).astype(np.int64), 0, nf - 2)
    t = np.clip(p - i, 0.0, 1.0)
    out = (1.0 - t) * np.take_along_axis(v, i, axis=0) + t * np.take_along_axis(v, i + 1, axis=0)
    # the end nodes belong to the grid even where rounding puts p a hair
    # outside [0, nf - 1] (a spacing such as 8/6 is not exact)
    lo, hi = p < -1e-9, p > nf - 1 + 1e-9
    if outside is None:
        return np.where(lo, v[:1], np.where(hi, v[-1:], out))
    return np.where(lo | hi, outside, out)


# --------------------------------------------------------------------------
# One grid level
# --------------------------------------------------------------------------

@dataclasses.dataclass
class Level:
    nx: int
    ny: int
    nz: int
    dx: float
    dy: float
    z: np.ndarray
    T: np.ndarray
    n_tot: np.ndarray
    c_ul: np.ndarray
    vel: np.ndarray | None = None   # [3, nz, ny, nx] in Doppler widths

    @property
    def shape(self):
        return (self.nz, self.ny, self.nx)


class TwoLevelProblem:
    """The problem W(n) = f on a hierarchy of grids (finest = index ``n_grids``).

    ``levels[k]`` for k = 1 (coarsest) .. n_grids (finest), as in the paper.
    Populations are arrays [2, nz, ny, nx]: index 0 lower, 1 upper level.
    """

    def __init__(self, atm, atom, n_grids: int = 1, quad_a: float | None = None,
                 restriction: int = 0, interpolation: int = 0, sc_interp: int = 0):
        self.atom = atom
        self.n_grids = n_grids
        self.restriction = restriction
        self.interpolation = interpolation
        self.sc_interp = sc_interp
        # host threads of the static two-level formal solution (1: the plain
        # serial loop; more: rays in parallel, for timing on all cores)
        self.threads = 1
        self.mu, self.wray = a4_quadrature(quad_a)
        self.a_damp = float(getattr(atom, "a_damp", 0.0))
        self.x, self.phi, self.wphi = frequency_grid(atom.n_freq, atom.x_max, self.a_damp)
        vel = getattr(atm, "vel", None)
        fine = Level(atm.nx, atm.ny, atm.nz, atm.dx, atm.dy, np.asarray(atm.z, float),
                     np.asarray(atm.T, float), np.asarray(atm.n_tot, float),
                     np.asarray(atm.c_ul, float),
                     None if vel is None else np.asarray(vel, float))
        self.levels = {n_grids: fine}
        for k in range(n_grids - 1, 0, -1):
            self.levels[k] = coarsen_level(self.levels[k + 1])
        self.fs_count = {k: 0 for k in self.levels}
        self.sweep_count = {k: 0 for k in self.levels}
        self.negatives = 0
        # partial redistribution: the lagged mean intensity per frequency and
        # grid, and the discrete redistribution matrix
        self.gamma = float(getattr(atom, "gamma_prd", 0.0))
        self.prd = self.gamma > 0.0
        nf = len(self.x)
        self.jnu = {k: np.zeros((nf, lev.nx * lev.ny * lev.nz)) for k, lev in self.levels.items()}
        self.wq = self.wphi / self.phi
        self.R = prd_matrix(self.x, self.wq, self.phi, self.a_damp) if self.prd else None
        self.top = n_grids
        self._force_bg = False

    # ---- the lagged radiation field (partial redistribution) ----
    def updates_background(self, k: int) -> bool:
        """Whether a formal solution on grid k replaces the grid's lagged
        field by its own mean intensity: on the grid being solved always; on
        a coarser grid only in the Lambda-iteration that starts it (see the
        multi-level class)."""
        return self.prd and (k == self.top or self._force_bg)

    def lambda_iteration(self, k: int, n):
        self._force_bg = True
        try:
            self.formal_solution(k, n)
        finally:
            self._force_bg = False

    def prd_profile_ratio(self, k: int):
        """rho_f = psi_f/phi_f at every node from the lagged field J_f:
        rho = 1 + gamma f_rad (sum_f' w_f' R(f', f) J_f' / (phi_f Jbar) - 1),
        with Jbar = sum w phi J and f_rad = B_lu Jbar/(B_lu Jbar + C_lu), the
        radiative share of the upward transitions (equal at statistical
        equilibrium to n_l B_lu Jbar/(n_u P_u)); rho = 1 where Jbar = 0."""
        lev = self.levels[k]
        J = self.jnu[k]
        Jbar = self.wphi @ J
        g, A = self.atom.g_ratio, self.atom.a_ul
        c_lu = lev.c_ul.reshape(-1) * g * np.exp(-self.atom.theta / lev.T.reshape(-1))
        frad = g * A * Jbar / (g * A * Jbar + c_lu)
        Af = (self.R * self.wq[:, None]).T @ J                   # [nf, nvox]
        with np.errstate(divide="ignore", invalid="ignore"):
            ratio = np.where(Jbar > 0, Af / (self.phi[:, None] * Jbar[None, :]), 1.0)
        return 1.0 + self.gamma * frad[None, :] * (ratio - 1.0)

    def formal_solution_prd(self, k: int, n):
        """Formal solution with partial redistribution: S_f = rho_f S with S
        the CRD source function of the populations and rho_f from the lagged
        field; the MALI sums Jeff = sum w phi (I - w0 rho S) and
        U = sum w phi (1 - w0 rho) treat S as new and rho as fixed."""
        lev = self.levels[k]
        chi, S = self.opacity_source(lev, n)
        rho = self.prd_profile_ratio(k)
        Sf = rho * S[None, :]
        nf = len(self.phi)
        shp = (nf,) + lev.shape
        Ib = self.planck(lev.T[0]).reshape(1, lev.ny, lev.nx)
        Jx, Ux, Jm = formal_solution_nu_raw(lev.z, lev.dx, lev.dy, self.mu, self.wray,
                                            chi.reshape(shp), Sf.reshape(shp), Sf.reshape(shp),
                                            rho.reshape(shp), Ib, 0.0, want_j=True,
                                            interp=self.sc_interp)
        Jx, Ux, Jm = (a.reshape(nf, -1) for a in (Jx, Ux, Jm))
        if self.updates_background(k):
            self.jnu[k] = Jm
        self.fs_count[k] += 1
        return ((self.wphi @ Jm).reshape(lev.shape), (self.wphi @ Jx).reshape(lev.shape),
                (self.wphi @ Ux).reshape(lev.shape))

    # ---- opacity and source function (Eq. 1, CRD two-level atom) ----
    def planck(self, T):
        """B(T) at line centre in units of 2 h nu0^3/c^2."""
        return 1.0 / np.expm1(self.atom.theta / T)

    def opacity_source(self, lev: Level, n):
        """chi_nu [nfreq, nvox] and S [nvox] from populations.

        chi_nu = kappa (n_l g_u/g_l - n_u) phi(x_nu);  S = n_u/(n_l g_u/g_l - n_u),
        the ratio of line emissivity n_u A_ul to line opacity, with
        B_lu = (g_u/g_l) B_ul and B_ul = A_ul in these intensity units.
        """
        g = self.atom.g_ratio
        nl = n[0].reshape(-1)
        nu = n[1].reshape(-1)
        diff = nl * g - nu
        chi = self.atom.kappa * diff[None, :] * self.phi[:, None]
        S = nu / diff
        return chi, S

    def formal_solution(self, k: int, n):
        """One formal solution on level k with populations n: (Jbar, Jeff, U)."""
        lev = self.levels[k]
        if lev.vel is not None:
            return self.formal_solution_moving(k, n)
        if self.prd:
            return self.formal_solution_prd(k, n)
        nvox = lev.nx * lev.ny * lev.nz
        nf = len(self.phi)
        chi, S = self.opacity_source(lev, n)
        chi = np.ascontiguousarray(chi)
        Sf = np.ascontiguousarray(np.broadcast_to(S[None, :], (nf, nvox)))
        wphi = np.ascontiguousarray(np.broadcast_to(self.wphi[:, None], (nf, nvox)))
        Ib = np.ascontiguousarray(np.broadcast_to(
            self.planck(lev.T[0]).reshape(1, -1), (nf, lev.nx * lev.ny)))
        It = np.zeros((nf, lev.nx * lev.ny))
        Jbar = np.empty(nvox)
        Jeff = np.empty(nvox)
        U = np.empty(nvox)
        mu = np.ascontiguousarray(self.mu)
        if self.threads > 1:
            # rays on several host threads (timing the oracle on all cores)
            rc = _load().orc_formal_solution_threads(
                lev.nx, lev.ny, lev.nz, lev.dx, lev.dy, _ptr(np.ascontiguousarray(lev.z)),
                len(self.wray), _ptr(mu), _ptr(self.wray), nf, _ptr(chi), _ptr(Sf),
                _ptr(wphi), _ptr(Ib), _ptr(It), _ptr(Jbar), _ptr(Jeff), _ptr(U),
                int(self.sc_interp), int(self.threads))
        else:
            rc = _load().orc_formal_solution(
                lev.nx, lev.ny, lev.nz, lev.dx, lev.dy, _ptr(np.ascontiguousarray(lev.z)),
                len(self.wray), _ptr(mu), _ptr(self.wray), nf, _ptr(chi), _ptr(Sf),
                _ptr(wphi), _ptr(Ib), _ptr(It), _ptr(Jbar), _ptr(Jeff), _ptr(U), None,
                int(self.sc_interp))
        if rc != 0:
            raise RuntimeError("oracle formal solution failed")
        self.fs_count[k] += 1
        return (Jbar.reshape(lev.shape), Jeff.reshape(lev.shape), U.reshape(lev.shape))

    def formal_solution_moving(self, k: int, n):
        """Formal solution in a moving atmosphere (CRD; the paper's Bifrost
        atmospheres move).  Reading: along ray r the line profile at a node
        is Doppler-shifted by the projected velocity, phi(x_nu - mu_r . u)
        with u in Doppler widths, and the frequency weights w_nu phi are
        renormalised per node and ray to sum to 1, so that Jbar stays a
        profile average.  Opacity and weights then depend on the ray: each
        ray is solved on its own by the C loop nest and the sums are added.
        """
        lev = self.levels[k]
        nvox = lev.nx * lev.ny * lev.nz
        nf = len(self.phi)
        g = self.atom.g_ratio
        nl = n[0].reshape(-1)
        nu = n[1].reshape(-1)
        diff = nl * g - nu
        chi0 = self.atom.kappa * diff
        S = np.ascontiguousarray(np.broadcast_to((nu / diff)[None, :], (nf, nvox)))
        wq = self.wphi / self.phi          # the frequency quadrature weights
        u = lev.vel.reshape(3, -1)
        if self.prd:
            return self._formal_solution_moving_prd(k, lev, chi0, nu / diff, u)
        Ib = np.ascontiguousarray(np.broadcast_to(
            self.planck(lev.T[0]).reshape(1, -1), (nf, lev.nx * lev.ny)))
        It = np.zeros((nf, lev.nx * lev.ny))
        Jbar = np.zeros(nvox)
        Jeff = np.zeros(nvox)
        U = np.zeros(nvox)
        z = np.ascontiguousarray(lev.z)
        for r in range(len(self.wray)):
            ur = self.mu[r] @ u                                   # [nvox]
            prof = line_profile(self.x[:, None] - ur[None, :], self.a_damp)
            wphi = wq[:, None] * prof
            wphi = np.ascontiguousarray(wphi / wphi.sum(axis=0))
            chi = np.ascontiguousarray(chi0[None, :] * prof)
            jb, je, uu = (np.empty(nvox) for _ in range(3))
            mu1 = np.ascontiguousarray(self.mu[r:r + 1])
            w1 = np.ascontiguousarray(self.wray[r:r + 1])
            rc = _load().orc_formal_solution(
                lev.nx, lev.ny, lev.nz, lev.dx, lev.dy, _ptr(z), 1, _ptr(mu1), _ptr(w1), nf,
                _ptr(chi), _ptr(S), _ptr(wphi), _ptr(Ib), _ptr(It), _ptr(jb), _ptr(je),
                _ptr(uu), None, int(self.sc_interp))
            if rc != 0:
                raise RuntimeError("oracle formal solution failed")
            Jbar += jb
            Jeff += je
            U += uu
        self.fs_count[k] += 1
        return (Jbar.reshape(lev.shape), Jeff.reshape(lev.shape), U.reshape(lev.shape))

    def _shifted(self, v, y, outside):
        """``read_shifted`` on this atom's frequency grid."""
        return read_shifted(v, y, self.x, outside)

    def _formal_solution_moving_prd(self, k: int, lev, chi0, S, u):
        """Partial redistribution in a flow (reading: redistribution in each
        node's comoving frame, the hybrid treatment of Leenaarts, Pereira &
        Uitenbroek 2012).  Along ray r the shift is s = mu_r . u.  The lagged
        field is the comoving mean intensity J_cm(y) = sum_r w_r I_r(y + s),
        I_r read at observer offset y + s by linear interpolation in
        frequency (edge value beyond the grid); rho_cm follows from it as in
        the static case, and the emission of ray r at observer offset x has
        the ratio rho_cm(x - s) (1 beyond the grid), scaled per node and ray
        so that the emission profile keeps sum_f w phi rho = 1 on the ray's
        renormalised weights (photon conservation, exact in the static
        case; without it the local operator overshoots where a shifted line
        meets the grid's edge, and MALI loses positivity).  Opacity and the
        renormalised weights are those of the moving CRD solution; the MALI
        sums treat rho as fixed, as in the static case."""
        nvox = lev.nx * lev.ny * lev.nz
        nf = len(self.phi)
        wq = self.wphi / self.phi
        rho_cm = self.prd_profile_ratio(k)
        shp = (nf,) + lev.shape
        Ib = self.planck(lev.T[0]).reshape(1, lev.ny, lev.nx)
        Jbar, Jeff, U = (np.zeros(nvox) for _ in range(3))
        Jcm = np.zeros((nf, nvox))
        for r in range(len(self.wray)):
            ur = self.mu[r] @ u
            xs = self.x[:, None] - ur[None, :]                      # comoving offsets
            prof = line_profile(xs, self.a_damp)
            wphi = wq[:, None] * prof
            wphi = wphi / wphi.sum(axis=0)
            chi = chi0[None, :] * prof
            rho = self._shifted(rho_cm, xs, 1.0)
            # photons conserved per node and ray: sum_f w phi rho = 1 on the
            # ray's renormalised weights, as in the static case
            rho = rho / np.sum(wphi * rho, axis=0)[None, :]
            Sf = rho * S[None, :]
            Jx, Ux, Jm = formal_solution_nu_raw(lev.z, lev.dx, lev.dy, self.mu[r:r + 1],
                                                self.wray[r:r + 1], chi.reshape(shp),
                                                Sf.reshape(shp), Sf.reshape(shp),
                                                rho.reshape(shp), Ib, 0.0, want_j=True,
                                                interp=self.sc_interp)
            Jx, Ux, Jm = (a.reshape(nf, -1) for a in (Jx, Ux, Jm))
            Jbar += np.sum(wphi * Jm, axis=0)
            Jeff += np.sum(wphi * Jx, axis=0)
            U += np.sum(wphi * Ux, axis=0)
            I_r = Jm / self.wray[r]
            Jcm += self.wray[r] * self._shifted(I_r, self.x[:, None] + ur[None, :], None)
        if self.updates_background(k):
            self.jnu[k] = Jcm
        self.fs_count[k] += 1
        return Jbar.reshape(lev.shape), Jeff.reshape(lev.shape), U.reshape(lev.shape)

    # ---- statistical equilibrium (Eqs. 2-4) ----
    def rate_matrix(self, k: int, Jeff, U):
        """Matrix M [nvox, 2, 2] with W(n) = M n (rows: conservation, level u).

        Row 0 is particle conservation (Eq. 3).  Row 1 is the rate equation of
        the upper level in the sign convention of Eq. 2: n_u sum P_uj - sum n_j P_ju.
        Preconditioned radiative rates (Rybicki & Hummer 1991):
            P_lu = B_lu Jeff + C_lu,   P_ul = A_ul U + B_ul Jeff + C_ul,
        with U = 1 - Lambda*.  For Jeff = Jbar - Lambda* S(n) evaluated at the
        same n these equal the plain rates B_lu Jbar + C_lu and A_ul + B_ul
        Jbar + C_ul applied to n.
        """
        lev = self.levels[k]
        A = self.atom.a_ul
        g = self.atom.g_ratio
        c_ul = lev.c_ul.reshape(-1)
        c_lu = c_ul * g * np.exp(-self.atom.theta / lev.T.reshape(-1))
        je = Jeff.reshape(-1)
        uu = U.reshape(-1)
        P_lu = g * A * je + c_lu
        P_ul = A * uu + A * je + c_ul
        M = np.empty((je.size, 2, 2))
        M[:, 0, 0] = 1.0
        M[:, 0, 1] = 1.0
        M[:, 1, 0] = -P_lu
        M[:, 1, 1] = P_ul
        return M

    def default_rhs(self, k: int):
        lev = self.levels[k]
        f = np.zeros((2,) + lev.shape)
        f[0] = lev.n_tot
        return f

    def apply(self, M, n):
        nv = n.reshape(n.shape[0], -1).T             # [nvox, N]
        out = np.einsum("vij,vj->vi", M, nv)
        return out.T.reshape(n.shape)

    def solve(self, M, f):
        fv = f.reshape(f.shape[0], -1).T[:, :, None]
        x = np.linalg.solve(M, fv)[:, :, 0]
        return x.T.reshape(f.shape)

    def W(self, k: int, n):
        """W^k_*(n): rates from an extra formal solution with n (Eq. 5)."""
        _, Jeff, U = self.formal_solution(k, n)
        return self.apply(self.rate_matrix(k, Jeff, U), n)

    def zero_radiation(self, k: int):
        """Populations from statistical equilibrium with J = 0 (Sec. 4.11);
        with partial redistribution the lagged field starts at zero, so the
        first formal solution sees rho = 1 (CRD)."""
        lev = self.levels[k]
        zeros = np.zeros(lev.shape)
        ones = np.ones(lev.shape)
        if self.prd:
            self.jnu[k] = np.zeros_like(self.jnu[k])
        return self.solve(self.rate_matrix(k, zeros, ones), self.default_rhs(k))

    def mali_sweep(self, k: int, n, f=None):
        """One MALI iteration on level k solving W(n) = f; returns (n_new, C)."""
        if f is None:
            f = self.default_rhs(k)
        _, Jeff, U = self.formal_solution(k, n)
        n_new = self.solve(self.rate_matrix(k, Jeff, U), f)
        self.sweep_count[k] += 1
        return n_new, max_rel_change(n_new, n)

    # ---- multigrid (Secs. 2.2-2.3) ----
    def restrict(self, k_fine: int, a):
        """Restriction of populations and residuals: full weighting (the
        paper's choice) unless half weighting or injection was selected; the
        atmosphere is always full-weighted (Sec. 4.7)."""
        if getattr(self, "restriction", 0) == 1:
            return restrict_hw(a)
        if getattr(self, "restriction", 0) == 2:
            return restrict_inj(a)
        return restrict_fw(a)

    def prolong(self, k_fine: int, a_coarse):
        """Interpolation operator (Sec. 4.5): trilinear, or monotone cubic
        Hermite when ``interpolation`` is 1."""
        if self.interpolation == 1:
            return prolong_hermite(a_coarse, self.levels[k_fine].z)
        return prolong_trilinear(a_coarse, self.levels[k_fine].z)

    def vcycle(self, k: int, n: dict, f: dict, first: bool, params):
        """One FAS V-cycle from level k down to level 1; updates n[k] in place."""
        nu_pre = params["nu0"] if (first and k == self.n_grids) else params["nu1"]
        for _ in range(nu_pre):
            n[k], _ = self.mali_sweep(k, n[k], f[k])
        # residual with an extra formal solution (Eq. 5)
        r = f[k] - self.W(k, n[k])
        # coarse-grid equation (Eq. 9)
        n[k - 1] = self.restrict(k, n[k])
        self.coarse_entry(k, n[k - 1])
        n_before = n[k - 1].copy()
        f[k - 1] = self.restrict(k, r) + self.W(k - 1, n[k - 1])
        if k - 1 == 1:
            for _ in range(params["nu3"]):
                n[1], _ = self.mali_sweep(1, n[1], f[1])
        else:
            self.vcycle(k - 1, n, f, False, params)
        # relative correction (Eq. 10) and its interpolation (Eq. 11)
        e = (n[k - 1] - n_before) / n_before
        n_old = n[k]
        n_new = n_old * (1.0 + self.prolong(k, e))
        bad = n_new <= 0.0
        self.negatives += int(bad.sum())
        n_new[bad] = 0.1 * n_old[bad]
        n[k] = n_new
        for _ in range(params["nu2"]):
            n[k], _ = self.mali_sweep(k, n[k], f[k])

    def coarse_entry(self, k: int, n_coarse):
        """A V-cycle enters grid k-1 from k: with partial redistribution the
        lagged field of k, full-weighted, then one Lambda-iteration; the
        field stays fixed on grid k-1 until the cycle leaves it."""
        if self.prd:
            jf = self.jnu[k].reshape((-1,) + self.levels[k].shape)
            self.jnu[k - 1] = restrict_fw(jf).reshape(jf.shape[0], -1)
            self.lambda_iteration(k - 1, n_coarse)

    def fmg_prolong(self, k: int):
        """FMG moves the full approximation from grid k-1 to k, and the
        lagged field of partial redistribution with it."""
        if self.prd:
            jc = self.jnu[k - 1].reshape((-1,) + self.levels[k - 1].shape)
            self.jnu[k] = self.prolong(k, jc).reshape(jc.shape[0], -1)

    def fas_cycle(self, n_fine, first: bool, params):
        L = self.n_grids
        self.top = L
        n = {L: n_fine.copy()}
        f = {L: self.default_rhs(L)}
        self.vcycle(L, n, f, first, params)
        return n[L], max_rel_change(n[L], n_fine)


def max_rel_change(n_new, n_old):
    """C = max |n_new - n_old| / |n_new| over all levels and nodes (Sec. 3.3)."""
    return float(np.max(np.abs(n_new - n_old) / np.abs(n_new)))


def max_rel_error(n, n_ref):
    """E_inf = max |n - n_ref| / |n_ref| (Sec. 3.3)."""
    return float(np.max(np.abs(n - n_ref) / np.abs(n_ref)))


# --------------------------------------------------------------------------
# Grid transfer (Sec. 4.1, 4.4-4.7)
# --------------------------------------------------------------------------

def restrict_hw(a):
    """Half weighting of [..., nz, ny, nx] onto every second node (Sec. 4.4).

    Coarse node (K, J, I) on fine node (2K, 2J, 2I) takes 1/2 of the centre
    and 1/12 of each of its six axis neighbours (x, y periodic).  On the two
    fixed boundary planes only the plane itself is used: 1/2 of the centre
    and 1/8 of each of its four in-plane neighbours.  (Reading: the paper
    calls half weighting an average of the node and its six neighbours
    without giving weights; these are the standard half-weighting ones.)
    """
    a = np.asarray(a, dtype=np.float64)
    nz, ny, nx = a.shape[-3:]
    if nz % 2 != 1 or ny % 2 or nx % 2:
        raise ValueError("grid does not coarsen")
    nzc = (nz + 1) // 2
    zi = 2 * np.arange(nzc)
    c = a[..., zi, ::2, ::2]
    xm = np.roll(a, 1, axis=-1)[..., zi, ::2, ::2]
    xp = np.roll(a, -1, axis=-1)[..., zi, ::2, ::2]
    ym = np.roll(a, 1, axis=-2)[..., zi, ::2, ::2]
    yp = np.roll(a, -1, axis=-2)[..., zi, ::2, ::2]
    out = 0.5 * c + (xm + xp + ym + yp) / 12.0
    zm = a[..., np.clip(zi - 1, 0, nz - 1), ::2, ::2]
    zp = a[..., np.clip(zi + 1, 0, nz - 1), ::2, ::2]
    out += (zm + zp) / 12.0
    for K in (0, nzc - 1):
        out[..., K, :, :] = 0.5 * c[..., K, :, :] + (xm[..., K, :, :] + xp[..., K, :, :] +
                                                      ym[..., K, :, :] + yp[..., K, :, :]) / 8.0
    return out


def restrict_inj(a):
    """Injection (Sec. 4.4): the coarse node takes the fine node's value."""
    a = np.asarray(a, dtype=np.float64)
    return a[..., ::2, ::2, ::2].copy()


RESTRICTIONS = {0: None, 1: restrict_hw, 2: restrict_inj}


def restrict_fw(a):
    """Full weighting of [..., nz, ny, nx] onto every second node.

    Coarse node (K, J, I) sits on fine node (2K, 2J, 2I).  Its value is the
    sum over the 27 fine nodes (2K+c, 2J+b, 2I+a), a, b, c in {-1, 0, 1}, with
    weights w_a w_b w_c, w_0 = 1/2 and w_{+-1} = 1/4; x and y are periodic.  On
    the two fixed boundary planes (K = 0 and the top) the z stencil is the
    single fine plane 2K (weight 1): the boundary heights are kept.
    """
    a = np.asarray(a, dtype=np.float64)
    nz, ny, nx = a.shape[-3:]
    if nz % 2 != 1 or ny % 2 or nx % 2:
        raise ValueError("grid does not coarsen")
    nzc, nyc, nxc = (nz + 1) // 2, ny // 2, nx // 2
    wts = {-1: 0.25, 0: 0.5, 1: 0.25}
    out = np.zeros(a.shape[:-3] + (nzc, nyc, nxc))
    K = np.arange(nzc)
    interior = (K > 0) & (K < nzc - 1)
    for c in (-1, 0, 1):
        zi = np.clip(2 * K + c, 0, nz - 1)
        wz = np.where(interior, wts[c], 1.0 if c == 0 else 0.0)
        for b in (-1, 0, 1):
            yi = (2 * np.arange(nyc) + b) % ny
            for aa in (-1, 0, 1):
                xi = (2 * np.arange(nxc) + aa) % nx
                block = a[..., zi[:, None, None], yi[None, :, None], xi[None, None, :]]
                out += (wz[:, None, None] * wts[b] * wts[aa]) * block
    return out


def prolong_trilinear(ac, z_fine):
    """Trilinear interpolation of [..., nzc, nyc, nxc] onto the finer grid.

    Fine node i on an even index coincides with coarse node i/2; on an odd
    index it lies half-way (x, y: uniform spacing, periodic) or, in z, at the
    physical height z_fine[k] between the coarse planes at z_fine[k-1] and
    z_fine[k+1].  The value is the sum over the 8 surrounding coarse nodes of
    the product of the three 1D linear weights.
    """
    ac = np.asarray(ac, dtype=np.float64)
    nzc, nyc, nxc = ac.shape[-3:]
    nz, ny, nx = 2 * nzc - 1, 2 * nyc, 2 * nxc

    def axis_periodic(n, nc):
        i = np.arange(n)
        i0 = (i // 2) % nc
        i1 = np.where(i % 2 == 1, (i // 2 + 1) % nc, i0)
        w1 = np.where(i % 2 == 1, 0.5, 0.0)
        return i0, i1, 1.0 - w1, w1

    k = np.arange(nz)
    k0 = k // 2
    k1 = np.where(k % 2 == 1, k0 + 1, k0)
    zf = np.asarray(z_fine, dtype=np.float64)
    t = np.zeros(nz)
    odd = k % 2 == 1
    t[odd] = (zf[k[odd]] - zf[k[odd] - 1]) / (zf[k[odd] + 1] - zf[k[odd] - 1])
    zsets = ((k0, 1.0 - t), (k1, t))
    y0, y1, wy0, wy1 = axis_periodic(ny, nyc)
    x0, x1, wx0, wx1 = axis_periodic(nx, nxc)
    out = np.zeros(ac.shape[:-3] + (nz, ny, nx))
    for (zi, wz) in zsets:
        for (yi, wy) in ((y0, wy0), (y1, wy1)):
            for (xi, wx) in ((x0, wx0), (x1, wx1)):
                block = ac[..., zi[:, None, None], yi[None, :, None], xi[None, None, :]]
                out += (wz[:, None, None] * wy[None, :, None] * wx[None, None, :]) * block
    return out


def pchip_slopes(y, h, periodic: bool):
    """Node slopes of the monotone cubic Hermite interpolant along the last
    axis of ``y`` (Auer 2003; Fritsch & Butland 1984): with secants
    delta_i = (y_{i+1} - y_i)/h_i, an interior slope is the weighted harmonic
    mean (w1 + w2)/(w1/delta_{i-1} + w2/delta_i), w1 = 2h_i + h_{i-1},
    w2 = h_i + 2h_{i-1}, where both secants have the same strict sign, and 0
    otherwise.  ``periodic``: node n-1 is followed by node 0 at spacing h[-1]
    (every node is interior).  Otherwise the end slopes are the shape-
    preserving three-point ones: s = ((2h_0 + h_1) delta_0 - h_0 delta_1)/
    (h_0 + h_1), set to 0 if its sign differs from delta_0's and to 3 delta_0
    if delta_0 and delta_1 differ in sign and |s| > 3|delta_0| (the same at
    the far end); with two nodes the slope is the one secant.  ``h``: the
    n - 1 spacings (n when periodic)."""
    y = np.asarray(y, dtype=np.float64)
    h = np.asarray(h, dtype=np.float64)
    n = y.shape[-1]
    if periodic:
        delta = (np.roll(y, -1, axis=-1) - y) / h
        dm, dp = np.roll(delta, 1, axis=-1), delta
        hm, hp = np.roll(h, 1), h
    else:
        delta = np.diff(y, axis=-1) / h
        if n == 2:
            return np.concatenate([delta, delta], axis=-1)
        dm, dp = delta[..., :-1], delta[..., 1:]
        hm, hp = h[:-1], h[1:]
    w1, w2 = 2.0 * hp + hm, hp + 2.0 * hm
    same = ((dm > 0) & (dp > 0)) | ((dm < 0) & (dp < 0))
    with np.errstate(divide="ignore", invalid="ignore"):
        d = np.where(same, (w1 + w2) / (w1 / dm + w2 / dp), 0.0)
    if periodic:
        return d

    def end(d0, d1, h0, h1):
        s = ((2.0 * h0 + h1) * d0 - h0 * d1) / (h0 + h1)
        s = np.where(np.sign(s) != np.sign(d0), 0.0, s)
        return np.where((np.sign(d0) != np.sign(d1)) & (np.abs(s) > 3.0 * np.abs(d0)),
                        3.0 * d0, s)

    first = end(delta[..., 0], delta[..., 1], h[0], h[1])
    last = end(delta[..., -1], delta[..., -2], h[-1], h[-2])
    return np.concatenate([first[..., None], d, last[..., None]], axis=-1)


def hermite_eval(y0, y1, d0, d1, h, t):
    """Cubic Hermite on an interval of length h from end values y0, y1 and end
    slopes d0, d1, at fraction t."""
    t2, t3 = t * t, t * t * t
    return ((2 * t3 - 3 * t2 + 1) * y0 + (t3 - 2 * t2 + t) * h * d0
            + (-2 * t3 + 3 * t2) * y1 + (t3 - t2) * h * d1)


def _hermite_refine_axis(a, axis, periodic, xc, xf):
    """Monotone cubic Hermite of ``a`` along ``axis`` from nodes xc onto the
    finer nodes xf (xf[2i] = xc[i]; odd xf between two coarse nodes)."""
    a = np.moveaxis(np.asarray(a, dtype=np.float64), axis, -1)
    nc = a.shape[-1]
    if periodic:
        h = np.full(nc, xc[1] - xc[0] if nc > 1 else 1.0)
    else:
        h = np.diff(xc)
    d = pchip_slopes(a, h, periodic) if nc > 1 else np.zeros_like(a)
    nf = len(xf)
    out = np.empty(a.shape[:-1] + (nf,))
    out[..., 0::2] = a[..., : (nf + 1) // 2]
    i = np.arange(1, nf, 2)
    i0 = i // 2
    i1 = (i0 + 1) % nc
    hh = h[i0]
    t = (xf[i] - xc[i0]) / hh
    out[..., 1::2] = hermite_eval(a[..., i0], a[..., i1], d[..., i0], d[..., i1], hh, t)
    return np.moveaxis(out, -1, axis)


def prolong_hermite(ac, z_fine):
    """Monotone cubic Hermite interpolation of [..., nzc, nyc, nxc] onto the
    finer grid (Sec. 4.5, the alternative to trilinear interpolation).

    Reading: one-dimensional monotone Hermite passes (``pchip_slopes``),
    first along x (periodic, uniform), then along y (periodic, uniform), then
    along z at the physical heights (fixed ends); a fine node thus depends on
    the 4 x 4 x 4 coarse nodes around it.  Fine nodes on even indices keep
    the coarse value along that axis.  Each pass keeps a value between the
    two coarse values of its interval, so every fine value lies within the
    range of the 2 x 2 x 2 coarse nodes around it.
    """
    ac = np.asarray(ac, dtype=np.float64)
    nzc, nyc, nxc = ac.shape[-3:]
    nz, ny, nx = 2 * nzc - 1, 2 * nyc, 2 * nxc
    zf = np.asarray(z_fine, dtype=np.float64)
    a = _hermite_refine_axis(ac, -1, True, np.arange(nxc, dtype=float),
                             np.arange(nx) / 2.0)
    a = _hermite_refine_axis(a, -2, True, np.arange(nyc, dtype=float), np.arange(ny) / 2.0)
    return _hermite_refine_axis(a, -3, False, zf[::2], zf)


def redistribution_r2a(x, xp, a: float):
    """Hummer's angle-averaged R_II (upper level broadened, damping a > 0,
    coherent in the atom's frame, isotropic scattering), written as the
    average over the scattering angle g with weight sin(g)/2 of R_II(g):
        R_II-A(x, x') = (1/2pi) int_0^pi exp(-[(x - x')/(2 sin(g/2))]^2)
                        H(a / cos(g/2), (x + x')/(2 cos(g/2))) dg,
    H(a, v) = Re w(v + i a).  Its marginal is the Voigt profile; for a -> 0 it
    tends to erfc(max(|x|, |x'|))/2.  Unlike that limit it is not symmetric
    under x -> -x: far-wing photons stay in their wing."""
    from scipy.integrate import quad
    from scipy.special import wofz

    def f(g):
        s, c = math.sin(0.5 * g), math.cos(0.5 * g)
        if s <= 0.0 or c <= 0.0:
            return 0.0
        return (math.exp(-((x - xp) / (2.0 * s)) ** 2)
                * wofz((x + xp) / (2.0 * c) + 1j * a / c).real)

    return quad(f, 0.0, math.pi, epsabs=1e-15, epsrel=1e-13, limit=400)[0] / (2.0 * math.pi)


def prd_matrix(x, wq, phi, a_damp: float = 0.0, iters: int = 200):
    """Discrete angle-averaged redistribution matrix R[f', f] on the frequency
    grid: Hummer's R_I-A(x', x) = erfc(max(|x|, |x'|))/2 (pure Doppler
    redistribution; R_II-A for zero damping), or R_II-A with damping
    (``redistribution_r2a``), whose marginals are the line profile, scaled
    symmetrically, R = diag(c) R0 diag(c), so that the discrete marginals
    sum_f' wq_f' R[f', f] equal phi_f exactly (fixed-point iteration
    c <- sqrt(c phi / (R0^T (wq c)))).  Then a frequency-flat J gives rho = 1
    and the emission profile keeps sum w phi rho = 1."""
    from scipy.special import erfc
    x = np.asarray(x, dtype=np.float64)
    ax = np.abs(x)
    if a_damp > 0.0:
        n = len(x)
        R0 = np.empty((n, n))
        for i in range(n):
            for j in range(i, n):
                R0[i, j] = R0[j, i] = redistribution_r2a(x[i], x[j], a_damp)
    else:
        R0 = 0.5 * erfc(np.maximum(ax[:, None], ax[None, :]))
    c = np.ones(len(x))
    for _ in range(iters):
        c = np.sqrt(c * phi / (R0.T @ (wq * c)))
    return c[:, None] * R0 * c[None, :]


def coarsen_level(lev: Level) -> Level:
    """Atmosphere on the next coarser grid (Sec. 4.1, 4.7).

    The grid keeps every second node (z coordinates by dropping nodes, so the
    boundary heights stay fixed); T, n_tot and the collisional rate are
    carried over by full weighting, and so is the velocity field.
    """
    return Level(lev.nx // 2, lev.ny // 2, (lev.nz + 1) // 2, 2 * lev.dx, 2 * lev.dy,
                 lev.z[::2].copy(), restrict_fw(lev.T), restrict_fw(lev.n_tot),
                 restrict_fw(lev.c_ul), None if lev.vel is None else restrict_fw(lev.vel))


# --------------------------------------------------------------------------
# Drivers
# --------------------------------------------------------------------------

def mali_solve(prob: TwoLevelProblem, tol: float, max_iter: int = 100000, n0=None,
               history=None):
    """Plain MALI on the finest grid from the zero-radiation start."""
    L = prob.n_grids
    n = prob.zero_radiation(L) if n0 is None else n0.copy()
    for it in range(1, max_iter + 1):
        n, C = prob.mali_sweep(L, n)
        if history is not None:
            history.append(C)
        if not math.isfinite(C):
            raise FloatingPointError("MALI produced non-finite populations")
        if C < tol:
            return n, it
    raise RuntimeError("MALI did not converge")


def fas_solve(prob: TwoLevelProblem, tol: float, params, max_cycles: int = 1000,
              n0=None, history=None):
    """FAS V-cycles on the finest grid from the zero-radiation start."""
    L = prob.n_grids
    n = prob.zero_radiation(L) if n0 is None else n0.copy()
    for cyc in range(1, max_cycles + 1):
        n, C = prob.fas_cycle(n, cyc == 1, params)
        if history is not None:
            history.append(C)
        if not math.isfinite(C):
            raise FloatingPointError("FAS produced non-finite populations")
        if C < tol:
            return n, cyc
    raise RuntimeError("FAS did not converge")


def fmg_solve(prob: TwoLevelProblem, tol: float, params, max_cycles: int = 1000,
              history=None):
    """Full multigrid (Sec. 2.3): solve on level 1, interpolate the full
    approximation upward with one V-cycle per intermediate level, then
    regular V-cycles on the finest grid until C < tol."""
    L = prob.n_grids
    prob.top = 1          # the grid the current stage solves on
    n1 = prob.zero_radiation(1)
    for _ in range(params["nu_fmg"]):
        n1, _ = prob.mali_sweep(1, n1)
    n_k = n1
    for k in range(2, L + 1):
        prob.top = k
        n_k = prob.prolong(k, n_k)
        prob.fmg_prolong(k)
        if k < L:
            n = {k: n_k}
            f = {k: prob.default_rhs(k)}
            prob.vcycle(k, n, f, False, params)
            n_k = n[k]
    n = n_k
    for cyc in range(1, max_cycles + 1):
        n, C = prob.fas_cycle(n, cyc == 1, params)
        if history is not None:
            history.append(C)
        if not math.isfinite(C):
            raise FloatingPointError("FMG produced non-finite populations")
        if C < tol:
            return n, cyc
    raise RuntimeError("FMG did not converge")


# --------------------------------------------------------------------------
# Multi-level atom: lines, bound-free continua, grey background continuum
# --------------------------------------------------------------------------

@dataclasses.dataclass
class MLLevel:
    nx: int
    ny: int
    nz: int
    dx: float
    dy: float
    z: np.ndarray
    T: np.ndarray
    n_tot: np.ndarray
    chi_c: np.ndarray
    c: np.ndarray       # [N, N, nz, ny, nx]
    saha: np.ndarray    # [N, nz, ny, nx]
    sigma_c: np.ndarray  # background coherent scattering coefficient
    vel: np.ndarray | None = None   # [3, nz, ny, nx] in Doppler widths at t_ref

    @property
    def shape(self):
        return (self.nz, self.ny, self.nx)


def coarsen_ml_level(lev: MLLevel) -> MLLevel:
    """Coarser grid (Sec. 4.1, 4.7): every second node, full weighting of every
    atmospheric field (T, n_tot, background absorption and scattering,
    collisional rates, LTE ratios)."""
    return MLLevel(lev.nx // 2, lev.ny // 2, (lev.nz + 1) // 2, 2 * lev.dx, 2 * lev.dy,
                   lev.z[::2].copy(), restrict_fw(lev.T), restrict_fw(lev.n_tot),
                   restrict_fw(lev.chi_c), restrict_fw(lev.c), restrict_fw(lev.saha),
                   restrict_fw(lev.sigma_c), None if lev.vel is None else restrict_fw(lev.vel))


def formal_solution_nu_raw(z, dx, dy, mu, wray, chi, S, sl, fl, I_bottom, I_top,
                           want_j: bool = False, interp: int = 0):
    """Per-frequency angle sums Jx, Ux [nfreq, nz, ny, nx] (see fs_oracle.c),
    and with want_j also the mean intensity J = sum_r w_r I."""
    chi = np.ascontiguousarray(chi, dtype=np.float64)
    nf, nz, ny, nx = chi.shape
    arrs = [np.ascontiguousarray(np.broadcast_to(a, chi.shape), dtype=np.float64)
            for a in (S, sl, fl)]
    Ib = np.ascontiguousarray(np.broadcast_to(I_bottom, (nf, ny, nx)), dtype=np.float64)
    It = np.ascontiguousarray(np.broadcast_to(I_top, (nf, ny, nx)), dtype=np.float64)
    Jx = np.empty(chi.shape)
    Ux = np.empty(chi.shape)
    Jm = np.empty(chi.shape) if want_j else None
    rc = _load().orc_formal_solution_nu(nx, ny, nz, float(dx), float(dy),
                                        _ptr(np.ascontiguousarray(z, dtype=np.float64)),
                                        len(wray), _ptr(np.ascontiguousarray(mu)),
                                        _ptr(np.ascontiguousarray(wray)), nf, _ptr(chi),
                                        _ptr(arrs[0]), _ptr(arrs[1]), _ptr(arrs[2]), _ptr(Ib),
                                        _ptr(It), _ptr(Jx), _ptr(Ux), _ptr(Jm), int(interp))
    if rc != 0:
        raise RuntimeError("oracle formal solution failed")
    return (Jx, Ux, Jm) if want_j else (Jx, Ux)


def trapezoid_weights(x):
    w = np.zeros_like(x)
    if len(x) == 1:
        w[0] = 1.0
        return w
    d = np.diff(x)
    w[:-1] += 0.5 * d
    w[1:] += 0.5 * d
    return w


class MultiLevelProblem(TwoLevelProblem):
    """W(n) = f for an N-level atom (Eqs. 2-4) with lines, bound-free continua
    and a grey LTE background continuum, on a hierarchy of grids.

    Per frequency of transition t (lower l, upper u) and node:
        chi_t = n_l a - n_u b,   eta_t = n_u e        (line or bound-free)
        chi = chi_t + chi_c,     S = (eta_t + chi_c B_nu)/chi,
        sl = eta_t / chi,        fl = chi_t / chi.
    Lines: a = kappa (g_u/g_l) phi, b = kappa phi, e = kappa rho^3 phi with the
    Doppler profile phi(x) = exp(-(x/d)^2)/(sqrt(pi) d), d = sqrt(T/t_ref),
    or for a line with damping a (at t_ref) the Voigt profile
    H(a/d, x/d)/(sqrt(pi) d) (``ml_line_profile``).
    Bound-free (l -> continuum u): a = kappa y^-3, b = kappa y^-3 G E,
    e = kappa y^-3 G E (rho y)^3 with y = nu/nu_threshold, G = n_l*/n_u* and
    E = exp(-theta_ref rho y / T).  B_nu = (rho y)^3 / (exp(theta_ref rho y/T) - 1)
    (rho y -> rho for lines: one Planck value per line).
    With background coherent scattering (grey, isotropic, frequency-preserving
    coefficient sigma_c beside the absorption chi_c; Sec. 4.8):
        chi = chi_t + chi_c + sigma_c,
        S = (eta_t + chi_c B_nu + sigma_c J_nu) / chi,
    where J_nu is the mean intensity of the previous formal solution on the
    same grid (Lambda-iteration for the background; the preconditioning below
    treats only the transition's own emission as new).  Every formal solution
    stores its J_nu as the grid's background field; the zero-radiation start
    clears it and adds one Lambda-iteration; a V-cycle entering a coarser grid
    restricts it by full weighting, and FMG prolongs it with the populations
    (readings of Sec. 4.8, which restricts the field and runs one or two
    Lambda-iterations per coarse grid: here the coarse grid's own formal
    solutions, the first of them for the tau-correction, are those
    iterations).
    Preconditioned radiative rates (Rybicki & Hummer 1992, diagonal operator),
    with Jx = sum_r w_r (I - w0 sl), Ux = sum_r w_r (1 - w0 fl) per frequency:
        R_lu = sum_nu qa Jx,   R_ul = sum_nu (qe Ux + qb Jx),
    lines: qa = B_lu wphi, qb = B_ul wphi, qe = A_ul wphi (wphi: trapezoid x
    profile, normalised per node to sum 1; B_ul = A_ul/rho^3,
    B_lu = (g_u/g_l) B_ul); bound-free: qa = beta w_y y^-4, qb = qa G E,
    qe = qa G E (rho y)^3.
    """

    def __init__(self, atm, atom, n_grids: int = 1, quad_a: float | None = None,
                 restriction: int = 0, interpolation: int = 0, sc_interp: int = 0):
        self.atom = atom
        self.restriction = restriction
        self.interpolation = interpolation
        self.sc_interp = sc_interp
        self.N = atom.n_levels
        self.n_grids = n_grids
        self.mu, self.wray = a4_quadrature(quad_a)
        sigma = getattr(atm, "sigma_c", None)
        sigma = (np.zeros(np.shape(atm.T)) if sigma is None else np.asarray(sigma, float))
        vel = getattr(atm, "vel", None)
        fine = MLLevel(atm.nx, atm.ny, atm.nz, atm.dx, atm.dy, np.asarray(atm.z, float),
                       np.asarray(atm.T, float), np.asarray(atm.n_tot, float),
                       np.asarray(atm.chi_c, float), np.asarray(atm.c, float),
                       np.asarray(atm.saha, float), sigma,
                       None if vel is None else np.asarray(vel, float))
        self.scatter = bool(np.any(sigma > 0))
        self.levels = {n_grids: fine}
        for k in range(n_grids - 1, 0, -1):
            self.levels[k] = coarsen_ml_level(self.levels[k + 1])
        # frequency points: (kind, transition index, abscissa, weight)
        self.freqs = []
        for ti, ln in enumerate(atom.lines):
            x = np.linspace(-ln.x_max, ln.x_max, ln.n_freq) if ln.n_freq > 1 else np.zeros(1)
            for xv, wv in zip(x, trapezoid_weights(x)):
                self.freqs.append(("line", ti, float(xv), float(wv)))
        for ti, ct in enumerate(atom.continua):
            y = np.linspace(1.0, ct.y_max, ct.n_freq) if ct.n_freq > 1 else np.ones(1)
            for yv, wv in zip(y, trapezoid_weights(y)):
                self.freqs.append(("cont", ti, float(yv), float(wv)))
        self.line_freqs = {}
        for f, (kind, ti, xv, wv) in enumerate(self.freqs):
            if kind == "line":
                self.line_freqs.setdefault(ti, []).append(f)
        # partial redistribution of lines with a coherence fraction
        self.prd_lines = [ti for ti, ln in enumerate(atom.lines)
                          if getattr(ln, "gamma_prd", 0.0) > 0.0]
        self._prd_tables = {}
        # the lagged mean intensity per frequency serves background scattering
        # and partial redistribution alike
        self.lagged = self.scatter or bool(self.prd_lines)
        self.fs_count = {k: 0 for k in self.levels}
        self.sweep_count = {k: 0 for k in self.levels}
        self.negatives = 0
        nf = len(self.freqs)
        # background radiation field per grid, [nfreq, nvox]
        self.jbg = {k: np.zeros((nf, lev.nx * lev.ny * lev.nz)) for k, lev in self.levels.items()}
        # in a flow, PRD lines keep their comoving mean intensity apart from
        # the observer-frame field that background scattering reads
        self.jcm = {k: {} for k in self.levels}
        # the grid a solve or V-cycle currently treats as its finest: only its
        # formal solutions update its background field (see coarse_entry)
        self.top = n_grids
        self._force_bg = False

    def planck_rho(self, rho, T):
        return rho ** 3 / np.expm1(self.atom.theta_ref * rho / T)

    def transition_terms(self, k: int, n):
        """Per frequency: chi, S, sl, fl and the rate weights qa, qb, qe, all
        [nfreq, nvox], plus the bottom intensity [nfreq, nx*ny]."""
        lev = self.levels[k]
        at = self.atom
        T = lev.T.reshape(-1)
        nvox = T.size
        nf = len(self.freqs)
        out = {key: np.empty((nf, nvox)) for key in ("chi", "S", "sl", "fl", "qa", "qb", "qe")}
        Ib = np.empty((nf, lev.nx * lev.ny))
        chi_c = lev.chi_c.reshape(-1)
        sigma = lev.sigma_c.reshape(-1)
        nn = n.reshape(self.N, -1)
        # line profile normalisation per node and line
        d = np.sqrt(T / at.t_ref)
        norm = {}
        for (kind, ti, xv, wv) in self.freqs:
            if kind == "line":
                phi = ml_line_profile(xv, d, at.lines[ti].a_damp)
                norm[ti] = norm.get(ti, 0.0) + wv * phi
        for f, (kind, ti, xv, wv) in enumerate(self.freqs):
            if kind == "line":
                ln = at.lines[ti]
                lo, up = ln.lower, ln.upper
                phi = ml_line_profile(xv, d, ln.a_damp)
                gr = at.g[up] / at.g[lo]
                a = ln.kappa * gr * phi
                b = ln.kappa * phi
                e = ln.kappa * ln.rho ** 3 * phi
                B = self.planck_rho(ln.rho, T)
                wphi = wv * phi / norm[ti]
                b_ul = ln.a_ul / ln.rho ** 3
                out["qa"][f] = gr * b_ul * wphi
                out["qb"][f] = b_ul * wphi
                out["qe"][f] = ln.a_ul * wphi
                Ib[f] = self.planck_rho(ln.rho, lev.T[0].reshape(-1))
            else:
                ct = at.continua[ti]
                lo, up = ct.lower, self.N - 1
                G = lev.saha[lo].reshape(-1)
                E = np.exp(-at.theta_ref * ct.rho * xv / T)
                alpha = xv ** -3
                a = ct.kappa * alpha * np.ones_like(T)
                b = ct.kappa * alpha * G * E
                e = b * (ct.rho * xv) ** 3
                B = self.planck_rho(ct.rho * xv, T)
                qa = ct.beta * wv * xv ** -4
                out["qa"][f] = qa
                out["qb"][f] = qa * G * E
                out["qe"][f] = qa * G * E * (ct.rho * xv) ** 3
                Ib[f] = self.planck_rho(ct.rho * xv, lev.T[0].reshape(-1))
            chi_t = nn[lo] * a - nn[up] * b
            eta_t = nn[up] * e
            chi = chi_t + chi_c + sigma
            out["chi"][f] = chi
            out["S"][f] = (eta_t + chi_c * B + sigma * self.jbg[k][f]) / chi
            out["sl"][f] = eta_t / chi
            out["fl"][f] = chi_t / chi
        if self.prd_lines:
            # emission profile rho phi: the line emissivity, and with it the
            # transition's share of S, scales by rho; in the local operator
            # rho multiplies the transition's share of chi (the two-level
            # U = sum w phi (1 - w0 rho))
            for ti, rho in self.prd_ratios(k, n, out).items():
                for j, f in enumerate(self.line_freqs[ti]):
                    out["S"][f] += (rho[j] - 1.0) * out["sl"][f]
                    out["sl"][f] *= rho[j]
                    out["fl"][f] *= rho[j]
        return out, Ib

    # ---- partial redistribution of lines ----
    def prd_tables(self, k: int, ti: int):
        """For PRD line ti on grid k, per node: the redistribution matrix
        R[v, f', f] (R_I-A at the node's Doppler width d,
        R0(x', x) = erfc(max(|x|, |x'|)/d)/(2 d^2), or for a damped line
        R_II-A(x/d, x'/d; a/d)/d^2, scaled symmetrically so that its discrete
        marginals sum_f' wq R[f', f] are the node's profile, the fixed point
        of ``prd_matrix`` node by node), the normalised quadrature weights
        wq [v, f] and the profile phi [v, f]."""
        key = (k, ti)
        if key not in self._prd_tables:
            from scipy.special import erfc
            fs = self.line_freqs[ti]
            a = float(getattr(self.atom.lines[ti], "a_damp", 0.0))
            x = np.array([self.freqs[f][2] for f in fs])
            w = np.array([self.freqs[f][3] for f in fs])
            d = np.sqrt(self.levels[k].T.reshape(-1) / self.atom.t_ref)
            phi = ml_line_profile(x[None, :], d[:, None], a)
            wq = w[None, :] / (w[None, :] * phi).sum(axis=1)[:, None]
            ax = np.abs(x)
            dd = d[:, None, None]
            if a > 0.0:
                # one table per distinct Doppler width (the kernel is costly)
                R0 = np.empty((d.size, len(x), len(x)))
                cache = {}
                for v, dv in enumerate(d):
                    if dv not in cache:
                        t = np.empty((len(x), len(x)))
                        for i in range(len(x)):
                            for j in range(i, len(x)):
                                t[i, j] = t[j, i] = redistribution_r2a(
                                    x[i] / dv, x[j] / dv, a / dv) / dv ** 2
                        cache[dv] = t
                    R0[v] = cache[dv]
            else:
                R0 = 0.5 * erfc(np.maximum(ax[:, None], ax[None, :])[None, :, :] / dd) / dd ** 2
            c = np.ones_like(phi)
            for _ in range(200):
                c = np.sqrt(c * phi / np.einsum("vab,va->vb", R0, wq * c))
            self._prd_tables[key] = (c[:, :, None] * R0 * c[:, None, :], wq, phi)
        return self._prd_tables[key]

    def prd_ratios(self, k: int, n, terms):
        """rho_f = psi_f/phi_f for every PRD line at every node from the lagged
        field J_f (the two-level reading generalised):
            rho = 1 + gamma f_rad (sum_f' wq_f' R(f', f) J_f' / (phi_f Jbar) - 1),
        Jbar = sum wq phi J over the line, f_rad = n_l B_lu Jbar / sum_j n_j P_ju
        the radiative excitation's share of all transitions into the upper
        level (plain rates: the lagged J, no local operator, collisions);
        rho = 1 where Jbar = 0.  Returns {ti: rho [nf_line, nvox]}."""
        lev = self.levels[k]
        N = self.N
        nvox = lev.nx * lev.ny * lev.nz
        nn = n.reshape(N, -1)
        J = self.jbg[k]
        if self.jcm[k]:
            J = J.copy()
            for ti, jc in self.jcm[k].items():
                J[self.line_freqs[ti]] = jc
        P = lev.c.reshape(N, N, nvox).copy()
        for f, (kind, ti, xv, wv) in enumerate(self.freqs):
            if kind == "line":
                lo, up = self.atom.lines[ti].lower, self.atom.lines[ti].upper
            else:
                lo, up = self.atom.continua[ti].lower, N - 1
            P[lo, up] += terms["qa"][f] * J[f]
            P[up, lo] += terms["qe"][f] + terms["qb"][f] * J[f]
        out = {}
        for ti in self.prd_lines:
            ln = self.atom.lines[ti]
            fs = self.line_freqs[ti]
            R, wq, phi = self.prd_tables(k, ti)
            Jl = J[fs].T                                             # [nvox, nf_line]
            Jbar = np.sum(wq * phi * Jl, axis=1)
            excite = nn[ln.lower] * sum(terms["qa"][f] * J[f] for f in fs)
            inflow = sum(nn[j] * P[j, ln.upper] for j in range(N) if j != ln.upper)
            frad = excite / inflow
            Af = np.einsum("vab,va->vb", R, wq * Jl)
            with np.errstate(divide="ignore", invalid="ignore"):
                ratio = np.where(Jbar[:, None] > 0, Af / (phi * Jbar[:, None]), 1.0)
            out[ti] = (1.0 + ln.gamma_prd * frad[:, None] * (ratio - 1.0)).T
        return out

    def formal_solution(self, k: int, n):
        """Per-frequency (Jx, Ux) [nfreq, nz, ny, nx] and the rate weights; with
        background scattering the grid's background field becomes this
        solution's mean intensity."""
        lev = self.levels[k]
        if lev.vel is not None:
            return self.formal_solution_moving(k, n)
        terms, Ib = self.transition_terms(k, n)
        nf = len(self.freqs)
        shp = (nf,) + lev.shape
        res = formal_solution_nu_raw(lev.z, lev.dx, lev.dy, self.mu, self.wray,
                                     terms["chi"].reshape(shp), terms["S"].reshape(shp),
                                     terms["sl"].reshape(shp), terms["fl"].reshape(shp),
                                     Ib.reshape((nf, lev.ny, lev.nx)), 0.0,
                                     want_j=self.lagged, interp=self.sc_interp)
        Jx, Ux = res[0], res[1]
        if self.updates_background(k):
            self.jbg[k] = res[2].reshape(nf, -1)
        self.fs_count[k] += 1
        return Jx.reshape(nf, -1), Ux.reshape(nf, -1), terms

    def updates_background(self, k: int) -> bool:
        """Whether a formal solution on grid k replaces the grid's background
        field by its own mean intensity: on the grid being solved (the finest
        of the V-cycle, or of the FMG stage) always; on a coarser grid only in
        the Lambda-iteration that starts it, so that W on that grid is one
        operator from the tau-correction of Eq. 9 to the correction of Eq. 10
        (a converged fine solution then gets a zero correction)."""
        return self.lagged and (k == self.top or self._force_bg)

    def lambda_iteration(self, k: int, n):
        """One Lambda-iteration of the background field (Sec. 4.8): a formal
        solution with the populations held, whose mean intensity becomes the
        field."""
        self._force_bg = True
        try:
            self.formal_solution(k, n)
        finally:
            self._force_bg = False

    def coarse_entry(self, k: int, n_coarse):
        """Entering grid k-1 from k in a V-cycle (Sec. 4.8): the background
        field of k, full-weighted, then one Lambda-iteration with the
        restricted populations; the field then stays fixed on grid k-1
        until the cycle leaves it."""
        if self.lagged:
            fine = self.levels[k]
            jf = self.jbg[k].reshape((-1,) + fine.shape)
            self.jbg[k - 1] = restrict_fw(jf).reshape(jf.shape[0], -1)
            self.jcm[k - 1] = {ti: restrict_fw(jc.reshape((-1,) + fine.shape)).reshape(
                jc.shape[0], -1) for ti, jc in self.jcm[k].items()}
            self.lambda_iteration(k - 1, n_coarse)

    def fmg_prolong(self, k: int):
        """FMG moving the full approximation from grid k-1 to k: the
        background field moves with it (trilinear)."""
        if self.lagged:
            coarse = self.levels[k - 1]
            jc = self.jbg[k - 1].reshape((-1,) + coarse.shape)
            self.jbg[k] = self.prolong(k, jc).reshape(jc.shape[0], -1)
            self.jcm[k] = {ti: self.prolong(k, v.reshape((-1,) + coarse.shape)).reshape(
                v.shape[0], -1) for ti, v in self.jcm[k - 1].items()}

    def formal_solution_moving(self, k: int, n):
        """Formal solution in a moving atmosphere (the same reading as for the
        two-level atom): along ray r a line's profile at a node is
        phi((x - mu_r . u)/d)/(d sqrt(pi)), d the node's Doppler width in
        units of the one at t_ref, renormalised over the line's frequencies
        per node and ray; continua and the background do not shift.  Line
        opacity, emissivity and so chi, S and the transition shares depend
        on the ray, and so does the profile weight of the rates: each ray is
        solved on its own, and its angle sums enter the line sums weighted by
        its own profile weight.  Returned: those weighted sums with rate
        weights without the profile factor for lines (qa = g_u/g_l B_ul,
        qb = B_ul, qe = A_ul), and the plain sums with the usual weights for
        continua, so that the rates sum q J as in the static case."""
        lev = self.levels[k]
        at = self.atom
        terms, Ib = self.transition_terms(k, n)
        T = lev.T.reshape(-1)
        nvox = T.size
        nf = len(self.freqs)
        d = np.sqrt(T / at.t_ref)
        nn = n.reshape(self.N, -1)
        chi_c = lev.chi_c.reshape(-1)
        sigma = lev.sigma_c.reshape(-1)
        u = lev.vel.reshape(3, -1)
        Jw = np.zeros((nf, nvox))
        Uw = np.zeros((nf, nvox))
        Jm = np.zeros((nf, nvox))
        line_freqs = {}
        for f, (kind, ti, xv, wv) in enumerate(self.freqs):
            if kind == "line":
                line_freqs.setdefault(ti, []).append(f)
        shp = (nf,) + lev.shape
        # partial redistribution in the comoving frame (the two-level reading):
        # rho_cm per PRD line from the lagged comoving field, read by each ray
        # at its comoving offsets; the rays' intensities build the new field
        rho_cm = self.prd_ratios(k, n, terms) if self.prd_lines else {}
        xgrid = {ti: np.array([self.freqs[f][2] for f in line_freqs[ti]]) for ti in rho_cm}
        Jcm = {ti: np.zeros((len(line_freqs[ti]), nvox)) for ti in rho_cm}
        for r in range(len(self.wray)):
            ur = self.mu[r] @ u
            chi, S = terms["chi"].copy(), terms["S"].copy()
            sl, fl = terms["sl"].copy(), terms["fl"].copy()
            w = np.ones((nf, nvox))
            for ti, fs in line_freqs.items():
                ln = at.lines[ti]
                lo, up = ln.lower, ln.upper
                gr = at.g[up] / at.g[lo]
                B = self.planck_rho(ln.rho, T)
                phis = [ml_line_profile(self.freqs[f][2] - ur, d, ln.a_damp) for f in fs]
                norm = sum(self.freqs[f][3] * ph for f, ph in zip(fs, phis))
                if ti in rho_cm:
                    xl = xgrid[ti]
                    rho_r = read_shifted(rho_cm[ti], xl[:, None] - ur[None, :], xl, 1.0)
                    # photons conserved per node and ray (the two-level reading)
                    wl = np.array([self.freqs[f][3] for f in fs])[:, None] * np.array(phis) / norm
                    rho_r = rho_r / np.sum(wl * rho_r, axis=0)[None, :]
                else:
                    rho_r = np.ones((len(fs), nvox))
                for j, (f, ph) in enumerate(zip(fs, phis)):
                    chi_t = ln.kappa * ph * (nn[lo] * gr - nn[up])
                    eta_t = ln.kappa * ln.rho ** 3 * ph * nn[up] * rho_r[j]
                    chi[f] = chi_t + chi_c + sigma
                    S[f] = (eta_t + chi_c * B + sigma * self.jbg[k][f]) / chi[f]
                    sl[f] = eta_t / chi[f]
                    fl[f] = rho_r[j] * chi_t / chi[f]
                    w[f] = self.freqs[f][3] * ph / norm
            res = formal_solution_nu_raw(lev.z, lev.dx, lev.dy, self.mu[r:r + 1],
                                         self.wray[r:r + 1], chi.reshape(shp), S.reshape(shp),
                                         sl.reshape(shp), fl.reshape(shp),
                                         Ib.reshape((nf, lev.ny, lev.nx)), 0.0, want_j=True,
                                         interp=self.sc_interp)
            Jw += w * res[0].reshape(nf, -1)
            Uw += w * res[1].reshape(nf, -1)
            Jm += res[2].reshape(nf, -1)
            for ti in rho_cm:
                xl = xgrid[ti]
                I_r = res[2].reshape(nf, -1)[line_freqs[ti]] / self.wray[r]
                Jcm[ti] += self.wray[r] * read_shifted(I_r, xl[:, None] + ur[None, :], xl, None)
        for ti, fs in line_freqs.items():
            ln = at.lines[ti]
            gr = at.g[ln.upper] / at.g[ln.lower]
            b_ul = ln.a_ul / ln.rho ** 3
            for f in fs:
                terms["qa"][f] = gr * b_ul
                terms["qb"][f] = b_ul
                terms["qe"][f] = ln.a_ul
        if self.updates_background(k):
            self.jbg[k] = Jm
            self.jcm[k] = Jcm
        self.fs_count[k] += 1
        return Jw, Uw, terms

    def rate_matrix_from(self, k: int, Jx, Ux, terms):
        """M [nvox, N, N] with W(n) = M n: row 0 particle conservation (Eq. 3),
        row i the rate equation of level i in the sign convention of Eq. 2."""
        lev = self.levels[k]
        N = self.N
        nvox = lev.nx * lev.ny * lev.nz
        P = lev.c.reshape(N, N, nvox).copy()
        for f, (kind, ti, xv, wv) in enumerate(self.freqs):
            if kind == "line":
                lo, up = self.atom.lines[ti].lower, self.atom.lines[ti].upper
            else:
                lo, up = self.atom.continua[ti].lower, N - 1
            P[lo, up] += terms["qa"][f] * Jx[f]
            P[up, lo] += terms["qe"][f] * Ux[f] + terms["qb"][f] * Jx[f]
        M = np.zeros((nvox, N, N))
        M[:, 0, :] = 1.0
        for i in range(1, N):
            for j in range(N):
                if j == i:
                    M[:, i, i] = sum(P[i, jj] for jj in range(N) if jj != i)
                else:
                    M[:, i, j] = -P[j, i]
        return M

    def default_rhs(self, k: int):
        lev = self.levels[k]
        f = np.zeros((self.N,) + lev.shape)
        f[0] = lev.n_tot
        return f

    def W(self, k: int, n):
        Jx, Ux, terms = self.formal_solution(k, n)
        return self.apply(self.rate_matrix_from(k, Jx, Ux, terms), n)

    def zero_radiation(self, k: int):
        """Statistical equilibrium with J = 0 (Sec. 4.11): Jx = 0, Ux = 1."""
        lev = self.levels[k]
        nvox = lev.nx * lev.ny * lev.nz
        nf = len(self.freqs)
        n_any = np.ones((self.N,) + lev.shape)   # weights do not depend on n
        # only the rate weights are read; chi, S, sl and fl of these stand-in
        # populations go unused (and divide by zero where g_u = g_l)
        with np.errstate(divide="ignore", invalid="ignore"):
            terms, _ = self.transition_terms(k, n_any)
        M = self.rate_matrix_from(k, np.zeros((nf, nvox)), np.ones((nf, nvox)), terms)
        n = self.solve(M, self.default_rhs(k))
        if self.lagged:
            # the lagged field from nothing: cleared (rho = 1 for partial
            # redistribution); with background scattering one Lambda-iteration
            self.jbg[k] = np.zeros((nf, nvox))
            self.jcm[k] = {}
            if self.scatter:
                self.lambda_iteration(k, n)
        return n

    def mali_sweep(self, k: int, n, f=None):
        if f is None:
            f = self.default_rhs(k)
        Jx, Ux, terms = self.formal_solution(k, n)
        n_new = self.solve(self.rate_matrix_from(k, Jx, Ux, terms), f)
        self.sweep_count[k] += 1
        return n_new, max_rel_change(n_new, n)

    def lte_populations(self, k: int):
        """Saha-Boltzmann populations of the level's atmosphere (for checks)."""
        lev = self.levels[k]
        at = self.atom
        N = self.N
        rel = np.empty((N,) + lev.shape)
        rel[0] = 1.0
        for i in range(1, N - 1):
            rel[i] = at.g[i] / at.g[0] * np.exp(-(at.theta[i] - at.theta[0]) / lev.T)
        rel[N - 1] = 1.0 / lev.saha[0]          # n_c*/n_0*
        return rel / rel.sum(axis=0) * lev.n_tot
