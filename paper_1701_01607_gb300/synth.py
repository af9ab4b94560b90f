"""Seeded synthetic inputs: atmospheres and model-atom parameters.

This module builds the inputs that both the CUDA library and the CPU oracle
consume.  It holds none of the solver's arithmetic (no formal solution, no rate
equations, no grid transfer): only the recipe that turns a seed and a handful of
numbers into arrays.  The paper's own inputs (Bifrost snapshots, FAL-C, the
Carlsson & Leenaarts model atoms; Sec. 3.1-3.2) are not available, so these
synthetic stand-ins reproduce their structure instead:

* a static, isothermal two-level atom in complete redistribution, the
  redistribution every run of Sec. 3 uses;
* a vertically stratified number density chosen so that the LTE line-centre
  vertical optical depth runs log-linearly between two given values, which is
  the exponential atmosphere of a constant scale height;
* optional log-normal opacity perturbations from a Gaussian random field with a
  Kolmogorov-like spectrum, periodic in x and y (the horizontal boundaries of
  Sec. 4.2 are periodic);
* the collisional de-excitation rate chosen so that the two-level source
  function obeys S = (1 - eps) Jbar + eps B with a prescribed eps.

Units: lengths in grid cells of the finest grid (dx = dy = dz = 1 on a uniform
grid), rates in units of the Einstein A coefficient, intensities in units of
2 h nu0^3 / c^2.  Only the products chi * length and rate ratios enter the
problem, so this choice loses nothing.
"""

from __future__ import annotations

import dataclasses
import math

from typing import Optional

import numpy as np

H_PLANCK = 6.62607015e-34
C_LIGHT = 2.99792458e8
K_BOLTZ = 1.380649e-23


def theta_of_wavelength(lambda_m: float) -> float:
    """h nu0 / k in kelvin for a line at wavelength ``lambda_m`` (metres)."""
    return H_PLANCK * C_LIGHT / (lambda_m * K_BOLTZ)


@dataclasses.dataclass
class TwoLevelAtom:
    """Parameters of the two-level model atom (static, CRD, Doppler profile).

    ``kappa`` is the line opacity per unit lower-minus-upper population in
    inverse length at unit profile: the line opacity at normalised frequency
    offset x is kappa * (n_l g_u/g_l - n_u) * exp(-x^2)/sqrt(pi).
    """

    a_ul: float = 1.0
    g_ratio: float = 1.0          # g_u / g_l
    theta: float = theta_of_wavelength(500e-9)
    kappa: float = 1.0
    n_freq: int = 9
    x_max: float = 3.0
    gamma_prd: float = 0.0        # coherence fraction of partial redistribution (0: CRD)
    a_damp: float = 0.0           # damping (Voigt) parameter in Doppler widths (0: Doppler)


@dataclasses.dataclass
class Atmosphere:
    """A Cartesian atmosphere on nodes; arrays are C-ordered [z][y][x]."""

    nx: int
    ny: int
    nz: int
    dx: float
    dy: float
    z: np.ndarray        # [nz], increasing upward; z[0] is the bottom boundary
    T: np.ndarray        # [nz, ny, nx] kelvin
    n_tot: np.ndarray    # [nz, ny, nx] total number density of the atom
    c_ul: np.ndarray     # [nz, ny, nx] collisional de-excitation rate
    vel: Optional[np.ndarray] = None  # [3, nz, ny, nx] (x, y, z) velocity in
                                      # Doppler widths, or None (static)

    @property
    def shape(self):
        return (self.nz, self.ny, self.nx)


def collisional_rate_for_eps(eps, atom: TwoLevelAtom, T):
    """C_ul such that the two-level photon destruction probability is ``eps``.

    With eps' = C_ul (1 - exp(-theta/T)) / A_ul the source function of a
    two-level atom in CRD reads S = (Jbar + eps' B)/(1 + eps'), i.e. eps =
    eps'/(1 + eps').  Inverting gives C_ul = A_ul eps/(1-eps)/(1-exp(-theta/T)).
    ``eps`` may be 1 only through a large finite ratio; pass eps < 1.
    """
    eps = np.asarray(eps, dtype=np.float64)
    T = np.asarray(T, dtype=np.float64)
    ratio = eps / (1.0 - eps)
    return atom.a_ul * ratio / (-np.expm1(-atom.theta / T))


def gaussian_random_field(shape, seed: int, spectral_index: float = 11.0 / 3.0):
    """Unit-variance Gaussian random field, periodic in the last two axes.

    Seeded white noise is filtered in Fourier space by |k|^(-index/2), so that
    the power per mode falls as |k|^-index; index 11/3 gives a shell-integrated
    3D spectrum E(k) ~ k^-5/3.  The first axis (z) is generated on a domain of
    twice its length and cropped, so the field is not periodic vertically.
    """
    nz, ny, nx = shape
    big = (2 * nz, ny, nx)
    rng = np.random.default_rng(seed)
    noise = rng.standard_normal(big)
    kz = np.fft.fftfreq(big[0])[:, None, None]
    ky = np.fft.fftfreq(big[1])[None, :, None]
    kx = np.fft.fftfreq(big[2])[None, None, :]
    k2 = kx * kx + ky * ky + kz * kz
    amp = np.zeros_like(k2)
    nz_mask = k2 > 0
    amp[nz_mask] = k2[nz_mask] ** (-spectral_index / 4.0)
    field = np.fft.ifftn(np.fft.fftn(noise) * amp).real[:nz]
    field -= field.mean()
    std = field.std()
    if std > 0:
        field /= std
    return field


def stratified_two_level(nx: int, ny: int, nz: int, eps: float,
                         tau_top: float = 1e-4, tau_bottom: float = 1e4,
                         T: float = 5000.0, sigma: float = 0.0, seed: int = 0,
                         atom: TwoLevelAtom | None = None,
                         dx: float = 1.0, velocity: float = 0.0
                         ) -> tuple[Atmosphere, TwoLevelAtom]:
    """Isothermal, exponentially stratified box for the two-level atom.

    ``nz`` is the number of nodes (odd, so the grid coarsens with fixed
    vertical boundaries).  The heights are uniform with spacing ``dx``.  The
    number density is set so that, for LTE populations and no perturbation, the
    vertical line-centre optical depth measured from the top of an unbounded
    exponential atmosphere equals ``tau_top`` at the top node and
    ``tau_bottom`` at the bottom node.  ``sigma`` > 0 multiplies n_tot by the
    log-normal factor exp(sigma G - sigma^2/2) of a seeded Gaussian random
    field G.  ``velocity`` > 0 adds a velocity field whose three components
    are independent seeded Gaussian random fields (seeds seed+101..103) with
    that rms, in Doppler widths.
    """
    atom = atom or TwoLevelAtom()
    z = np.arange(nz, dtype=np.float64) * dx
    height = z[-1] - z[0]
    scale_height = height / math.log(tau_bottom / tau_top)
    tau = tau_top * np.exp((z[-1] - z) / scale_height)          # [nz]
    chi_lc = tau / scale_height                                 # line-centre opacity
    boltz = atom.g_ratio * math.exp(-atom.theta / T)            # n_u/n_l in LTE
    # LTE: n_l = n/(1+boltz), n_u = n boltz/(1+boltz); opacity factor is
    # n_l g_u/g_l - n_u = n_l (g_ratio - boltz) = n (g_ratio - boltz)/(1+boltz)
    per_n = atom.kappa * (atom.g_ratio - boltz) / (1.0 + boltz) / math.sqrt(math.pi)
    n_col = chi_lc / per_n
    n_tot = np.broadcast_to(n_col[:, None, None], (nz, ny, nx)).copy()
    if sigma > 0:
        g = gaussian_random_field((nz, ny, nx), seed)
        n_tot *= np.exp(sigma * g - 0.5 * sigma * sigma)
    Tarr = np.full((nz, ny, nx), float(T))
    c_ul = collisional_rate_for_eps(np.full((nz, ny, nx), eps), atom, Tarr)
    vel = None
    if velocity > 0:
        vel = np.stack([velocity * gaussian_random_field((nz, ny, nx), seed + 101 + c)
                        for c in range(3)])
    atm = Atmosphere(nx=nx, ny=ny, nz=nz, dx=dx, dy=dx, z=z, T=Tarr,
                     n_tot=n_tot, c_ul=np.ascontiguousarray(c_ul), vel=vel)
    return atm, atom


# Named workloads.  Grid sizes follow the even cell counts of the workload
# descriptions plus one node in z, so that nz = A 2^l + 1 (Sec. 4.2).
def box_16x16x33(seed: int = 0):
    """16x16x32 cells (33 nodes in z), eps=1e-3, tau 1e-4..1e4, T=5000 K."""
    return stratified_two_level(16, 16, 33, eps=1e-3, seed=seed)


def box_64x64x129_lognormal(seed: int = 1):
    """64x64x128 cells (129 nodes in z), eps=1e-4, log-normal sigma=0.3."""
    return stratified_two_level(64, 64, 129, eps=1e-4, sigma=0.3, seed=seed)


def stretched_heights(nz: int, d_mid: float, d_end: float, sharpness: float = 4.0):
    """Node heights [nz] whose spacing is d_mid at the middle of the column and
    grows smoothly (tanh^2 in the node index) to d_end at both ends, the
    pattern of the paper's Model 2 grid (fine in the middle, coarse at top and
    bottom).  z[0] = 0."""
    u = (np.arange(nz - 1) + 0.5) / (nz - 1) - 0.5
    t = np.tanh(sharpness * u) ** 2 / np.tanh(0.5 * sharpness) ** 2
    d = d_mid + (d_end - d_mid) * t
    return np.concatenate(([0.0], np.cumsum(d)))


def zero_populations_like(atm: Atmosphere, n_levels: int = 2):
    return np.zeros((n_levels,) + atm.shape)


# ---------------------------------------------------------------------------
# Multi-level atom (hydrogen-like, seeded) and a chromosphere-like atmosphere
# ---------------------------------------------------------------------------

@dataclasses.dataclass
class Line:
    lower: int
    upper: int
    rho: float          # nu / nu_ref
    a_ul: float         # Einstein A (rate units)
    kappa: float        # opacity per unit (n_l g_u/g_l - n_u) at unit profile
    n_freq: int
    x_max: float        # half width in reference Doppler widths
    a_damp: float = 0.0  # damping parameter at t_ref (0: Doppler profile)
    gamma_prd: float = 0.0  # coherence fraction of partial redistribution (0: CRD)


@dataclasses.dataclass
class Continuum:
    lower: int          # bound level; the upper level is the continuum level
    rho: float          # threshold nu / nu_ref
    beta: float         # photoionisation rate per unit J at threshold (rate units)
    kappa: float        # opacity per unit population at threshold (1/length)
    n_freq: int
    y_max: float        # frequencies nu/nu_threshold in [1, y_max]


@dataclasses.dataclass
class MultiLevelAtom:
    """N levels (the last may be a continuum), lines and bound-free continua.

    theta[i] is the energy of level i over k (K), measured from level 0;
    theta_ref = h nu_ref / k.  Intensities are in units of 2 h nu_ref^3/c^2,
    so B_ul = A_ul / rho^3 and B_lu = (g_u/g_l) B_ul for a line.
    """
    g: np.ndarray
    theta: np.ndarray
    theta_ref: float
    lines: list
    continua: list
    t_ref: float = 5000.0   # Doppler widths scale as sqrt(T / t_ref)

    @property
    def n_levels(self):
        return len(self.g)


@dataclasses.dataclass
class MultiLevelAtmosphere:
    """Cartesian atmosphere for a multi-level atom; arrays [nz][ny][nx].

    c[i, j] is the collisional rate from level i to level j (i != j);
    saha[i] is the LTE ratio n_i*/n_c* of bound level i to the continuum
    level (used by bound-free transitions); chi_c is the grey background
    absorption, whose source function is the Planck function; sigma_c (None
    for none) is a grey background coherent-scattering coefficient.
    """
    nx: int
    ny: int
    nz: int
    dx: float
    dy: float
    z: np.ndarray
    T: np.ndarray
    n_tot: np.ndarray
    chi_c: np.ndarray
    c: np.ndarray        # [N, N, nz, ny, nx]
    saha: np.ndarray     # [N, nz, ny, nx] (0 for levels without a continuum)
    sigma_c: Optional[np.ndarray] = None
    vel: Optional[np.ndarray] = None   # [3, nz, ny, nx] (x, y, z) velocity in units of
                                       # the Doppler width at t_ref, or None (static)

    @property
    def shape(self):
        return (self.nz, self.ny, self.nx)


def hydrogen_like_atom(n_bound: int = 5, line_freq: int = 100, cont_freq: int = 20,
                       seed: int = 2, theta_ref: float = 40000.0, x_max: float = 4.0,
                       y_max: float = 2.5, kappa_line: float = 10.0,
                       kappa_cont: float = 1e-3, beta_cont: float = 0.05,
                       jitter: float = 0.2, a_damp: float = 0.0,
                       gamma_prd: float = 0.0) -> MultiLevelAtom:
    """A seeded hydrogen-like atom: n_bound bound levels plus a continuum.

    Level n (1-based) has g = 2 n^2 and energy theta_ref (1 - 1/n^2)/(3/4)
    (so that the 1-2 line has h nu/k = theta_ref); the continuum sits at
    theta_ref/(3/4).  Lines 1-2, 2-3, ..., (n_bound-1)-n_bound and 1-3 with
    Kramers-like oscillator strengths; one bound-free continuum per bound
    level with a nu^-3 cross-section.  Strengths carry a seeded +-jitter.
    a_damp > 0 gives every line that damping parameter at t_ref (Voigt
    profiles), gamma_prd > 0 the resonance lines (lower level 0) that
    coherence fraction of partial redistribution; neither draws random
    numbers, so the seeded strengths do not change with them.
    """
    rng = np.random.default_rng(seed)
    n = np.arange(1, n_bound + 1, dtype=np.float64)
    g = np.r_[2.0 * n * n, 1.0]
    theta_ion = theta_ref / 0.75
    theta = np.r_[theta_ion * (1.0 - 1.0 / (n * n)), theta_ion]

    def jit():
        return 1.0 + jitter * (2.0 * rng.random() - 1.0)

    pairs = [(i, i + 1) for i in range(n_bound - 1)] + ([(0, 2)] if n_bound >= 3 else [])

    def kramers_f(nlo, nup):
        # Kramers' oscillator strength ~ 1/(l^5 u^3 (1/l^2 - 1/u^2)^3), scaled to
        # the hydrogen Lyman-alpha value 0.4162 for the 1-2 line
        raw = lambda a, b: 1.0 / (a ** 5 * b ** 3 * (1.0 / a ** 2 - 1.0 / b ** 2) ** 3)
        return 0.4162 * raw(nlo, nup) / raw(1.0, 2.0)

    f12 = kramers_f(1.0, 2.0)
    lines = []
    for (lo, up) in pairs:
        nlo, nup = lo + 1.0, up + 1.0
        rho = (1.0 / nlo ** 2 - 1.0 / nup ** 2) / 0.75
        f_lu = kramers_f(nlo, nup)
        # A_ul ~ f_lu (g_l/g_u) nu^2, in units where the 1-2 line has A = 1
        a_ul = (f_lu / f12) * (g[lo] / g[up]) / (g[0] / g[1]) * rho ** 2
        lines.append(Line(lo, up, rho, a_ul * jit(), kappa_line * (f_lu / f12) * jit(),
                          line_freq, x_max, a_damp, gamma_prd if lo == 0 else 0.0))
    continua = []
    for lo in range(n_bound):
        rho = (theta_ion - theta[lo]) / theta_ref
        continua.append(Continuum(lo, rho, beta_cont * (lo + 1) * jit(),
                                  kappa_cont * (lo + 1) * jit(), cont_freq, y_max))
    return MultiLevelAtom(g=g, theta=theta, theta_ref=theta_ref, lines=lines,
                          continua=continua)


def chromosphere(nx: int, ny: int, nz: int, atom: MultiLevelAtom, seed: int = 2,
                 t_min: float = 4000.0, t_max: float = 10000.0, scale_heights: float = 8.0,
                 n_bottom: float = 1e4, sigma_t: float = 0.1, ionisation: float = 1e-3,
                 saha_scale: float = 10.0, c_strength: float = 1e-2, chi_c0: float = 1e-2,
                 dx: float = 1.0, z=None, ground_collisions: float = 1.0,
                 scattering: float = 0.0, velocity: float = 0.0) -> MultiLevelAtmosphere:
    """Chromosphere-like box: T rises from t_min to t_max with height (with
    seeded 3D perturbations of relative size sigma_t), the density falls by
    e^scale_heights from bottom to top; electron density = ionisation x
    density; collisional rates from a van Regemorter-like n_e T^-1/2 law with
    seeded strengths and detailed balance; Saha-like LTE ratios
    saha_i = saha_scale n_e T^-3/2 (g_i/g_c) exp(theta_ion_i / T).  With the
    default strengths no line or continuum is inverted at the zero-radiation
    start (ten times weaker collisions make the upper lines mase).
    ground_collisions scales the collisions out of the ground level only, so
    that the resonance lines can be made scattering-dominated while the upper
    lines keep the collisions that prevent inversions.  scattering > 0 adds
    grey background coherent scattering sigma_c = scattering x chi_c.
    velocity > 0 adds a flow whose three components are independent seeded
    Gaussian random fields (seeds seed+101..103) with that rms, in Doppler
    widths at t_ref."""
    rng = np.random.default_rng(seed)
    if z is None:
        z = np.arange(nz, dtype=np.float64) * dx
    z = np.asarray(z, dtype=np.float64)
    h = (z - z[0]) / (z[-1] - z[0])
    T1 = t_min + (t_max - t_min) * h ** 2
    G = gaussian_random_field((nz, ny, nx), seed)
    T = T1[:, None, None] * (1.0 + sigma_t * np.tanh(G))
    rho = n_bottom * np.exp(-scale_heights * h)
    n_tot = np.broadcast_to(rho[:, None, None], (nz, ny, nx)).copy()
    n_e = ionisation * n_tot * (T / t_min)
    chi_c = chi_c0 * n_tot / n_bottom * (T / t_min) ** 2
    N = atom.n_levels
    c = np.zeros((N, N, nz, ny, nx))
    cont = N - 1
    saha = np.zeros((N, nz, ny, nx))
    for i in range(N - 1):
        th_ion = atom.theta[cont] - atom.theta[i]
        saha[i] = saha_scale * n_e * T ** -1.5 * (atom.g[i] / atom.g[cont]) * np.exp(th_ion / T)
    for i in range(N):
        for j in range(i + 1, N):
            s = c_strength * (1.0 + 0.2 * (2.0 * rng.random() - 1.0)) / (1.0 + (j - i))
            if i == 0:
                s *= ground_collisions
            down = s * n_e * (T / 5000.0) ** -0.5          # j -> i
            if j == cont:
                # detailed balance with the LTE ratio n_i*/n_c* = saha_i
                up = down / saha[i]
            else:
                up = down * (atom.g[j] / atom.g[i]) * np.exp(-(atom.theta[j] - atom.theta[i]) / T)
            c[j, i] = down
            c[i, j] = up
    sigma_c = scattering * chi_c if scattering > 0 else None
    vel = None
    if velocity > 0:
        vel = np.stack([velocity * gaussian_random_field((nz, ny, nx), seed + 101 + k)
                        for k in range(3)])
    return MultiLevelAtmosphere(nx=nx, ny=ny, nz=nz, dx=dx, dy=dx, z=z, T=T, n_tot=n_tot,
                                chi_c=chi_c, c=c, saha=saha, sigma_c=sigma_c, vel=vel)
