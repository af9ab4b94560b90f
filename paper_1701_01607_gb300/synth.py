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
                         dx: float = 1.0) -> tuple[Atmosphere, TwoLevelAtom]:
    """Isothermal, exponentially stratified box for the two-level atom.

    ``nz`` is the number of nodes (odd, so the grid coarsens with fixed
    vertical boundaries).  The heights are uniform with spacing ``dx``.  The
    number density is set so that, for LTE populations and no perturbation, the
    vertical line-centre optical depth measured from the top of an unbounded
    exponential atmosphere equals ``tau_top`` at the top node and
    ``tau_bottom`` at the bottom node.  ``sigma`` > 0 multiplies n_tot by the
    log-normal factor exp(sigma G - sigma^2/2) of a seeded Gaussian random
    field G.
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
    atm = Atmosphere(nx=nx, ny=ny, nz=nz, dx=dx, dy=dx, z=z, T=Tarr,
                     n_tot=n_tot, c_ul=np.ascontiguousarray(c_ul))
    return atm, atom


# Named workloads.  Grid sizes follow the even cell counts of the workload
# descriptions plus one node in z, so that nz = A 2^l + 1 (Sec. 4.2).
def box_16x16x33(seed: int = 0):
    """16x16x32 cells (33 nodes in z), eps=1e-3, tau 1e-4..1e4, T=5000 K."""
    return stratified_two_level(16, 16, 33, eps=1e-3, seed=seed)


def box_64x64x129_lognormal(seed: int = 1):
    """64x64x128 cells (129 nodes in z), eps=1e-4, log-normal sigma=0.3."""
    return stratified_two_level(64, 64, 129, eps=1e-4, sigma=0.3, seed=seed)


def zero_populations_like(atm: Atmosphere, n_levels: int = 2):
    return np.zeros((n_levels,) + atm.shape)
