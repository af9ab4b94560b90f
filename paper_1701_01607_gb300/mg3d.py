"""Thin ctypes binding of the C ABI in include/mg3d.h (same names).

Only argument marshalling lives here: every step of the solver runs in the
CUDA library.  Loading fails loudly if the library has not been built; there
is no CPU fallback.
"""

from __future__ import annotations

import ctypes
import os

import numpy as np

from . import build as _build

MG3D_OK = 0
MG3D_E_ARG = -1
MG3D_E_GRID = -2
MG3D_E_CUDA = -3
MG3D_E_OOM = -4
MG3D_E_DIVERGED = -5
MG3D_E_MAXITER = -6
MG3D_E_STATE = -8
MG3D_MAX_GRIDS = 8
MG3D_PREC_F64 = 0
MG3D_PREC_F32 = 1
MG3D_RESTRICT_FULL = 0
MG3D_RESTRICT_HALF = 1
MG3D_RESTRICT_INJECT = 2
MG3D_INTERP_LINEAR = 0
MG3D_INTERP_HERMITE = 1
MG3D_NOALLOC_MAX_NODES = 65536
MG3D_NOALLOC_MAX_NZ = 1024
MG3D_NOALLOC_MAX_FREQ = 64

_D = ctypes.POINTER(ctypes.c_double)


class mg3d_atmosphere(ctypes.Structure):
    _fields_ = [("nx", ctypes.c_int), ("ny", ctypes.c_int), ("nz", ctypes.c_int),
                ("dx", ctypes.c_double), ("dy", ctypes.c_double),
                ("z", _D), ("T", _D), ("n_tot", _D), ("c_ul", _D), ("vel", _D)]


class mg3d_atom(ctypes.Structure):
    _fields_ = [("a_ul", ctypes.c_double), ("g_ratio", ctypes.c_double),
                ("theta", ctypes.c_double), ("kappa", ctypes.c_double),
                ("n_freq", ctypes.c_int), ("x_max", ctypes.c_double),
                ("gamma_prd", ctypes.c_double), ("a_damp", ctypes.c_double)]


class mg3d_quadrature(ctypes.Structure):
    _fields_ = [("a", ctypes.c_double)]


class mg3d_params(ctypes.Structure):
    _fields_ = [("n_grids", ctypes.c_int), ("nu_fmg", ctypes.c_int), ("nu0", ctypes.c_int),
                ("nu1", ctypes.c_int), ("nu2", ctypes.c_int), ("nu3", ctypes.c_int),
                ("fs_prec", ctypes.c_int), ("restriction", ctypes.c_int),
                ("ml_chunk", ctypes.c_int), ("interpolation", ctypes.c_int),
                ("sc_interp", ctypes.c_int)]


class mg3d_line(ctypes.Structure):
    _fields_ = [("lower", ctypes.c_int), ("upper", ctypes.c_int), ("rho", ctypes.c_double),
                ("a_ul", ctypes.c_double), ("kappa", ctypes.c_double), ("n_freq", ctypes.c_int),
                ("x_max", ctypes.c_double), ("a_damp", ctypes.c_double),
                ("gamma_prd", ctypes.c_double)]


class mg3d_continuum(ctypes.Structure):
    _fields_ = [("lower", ctypes.c_int), ("rho", ctypes.c_double), ("beta", ctypes.c_double),
                ("kappa", ctypes.c_double), ("n_freq", ctypes.c_int), ("y_max", ctypes.c_double)]


class mg3d_ml_atom(ctypes.Structure):
    _fields_ = [("n_levels", ctypes.c_int), ("g", _D), ("theta", _D),
                ("theta_ref", ctypes.c_double), ("t_ref", ctypes.c_double),
                ("n_lines", ctypes.c_int), ("lines", ctypes.POINTER(mg3d_line)),
                ("n_continua", ctypes.c_int), ("continua", ctypes.POINTER(mg3d_continuum))]


class mg3d_ml_atmosphere(ctypes.Structure):
    _fields_ = [("nx", ctypes.c_int), ("ny", ctypes.c_int), ("nz", ctypes.c_int),
                ("dx", ctypes.c_double), ("dy", ctypes.c_double), ("z", _D), ("T", _D),
                ("n_tot", _D), ("chi_c", _D), ("c", _D), ("saha", _D), ("sigma_c", _D),
                ("vel", _D)]


class mg3d_stats(ctypes.Structure):
    _fields_ = [("iterations", ctypes.c_int),
                ("sweeps", ctypes.c_int * (MG3D_MAX_GRIDS + 1)),
                ("formal_solutions", ctypes.c_int * (MG3D_MAX_GRIDS + 1)),
                ("last_change", ctypes.c_double), ("negatives", ctypes.c_longlong),
                ("seconds", ctypes.c_double), ("fine_fs_equivalents", ctypes.c_double)]


class mg3d_counters(ctypes.Structure):
    _fields_ = [("kernel_launches", ctypes.c_longlong), ("fs_launches", ctypes.c_longlong),
                ("fs_units", ctypes.c_double), ("fs_kernel_ms", ctypes.c_double),
                ("fs_timed_launches", ctypes.c_longlong),
                ("level_fs_launches", ctypes.c_longlong * (MG3D_MAX_GRIDS + 1)),
                ("level_fs_units", ctypes.c_double * (MG3D_MAX_GRIDS + 1)),
                ("level_fs_kernel_ms", ctypes.c_double * (MG3D_MAX_GRIDS + 1)),
                ("level_fs_timed_launches", ctypes.c_longlong * (MG3D_MAX_GRIDS + 1))]


_H = ctypes.c_void_p
_I = ctypes.c_int
_SIGNATURES = {
    "mg3d_last_error": (ctypes.c_char_p, []),
    "mg3d_create": (_I, [ctypes.POINTER(mg3d_atmosphere), ctypes.POINTER(mg3d_atom),
                         ctypes.POINTER(mg3d_quadrature), ctypes.POINTER(mg3d_params),
                         ctypes.POINTER(_H)]),
    "mg3d_create_ml": (_I, [ctypes.POINTER(mg3d_ml_atmosphere), ctypes.POINTER(mg3d_ml_atom),
                            ctypes.POINTER(mg3d_quadrature), ctypes.POINTER(mg3d_params),
                            ctypes.POINTER(_H)]),
    "mg3d_n_levels": (_I, [_H, ctypes.POINTER(_I), ctypes.POINTER(_I)]),
    "mg3d_formal_solve_ml": (_I, [_H, _I, _D, _D]),
    "mg3d_destroy": (_I, [_H]),
    "mg3d_batch_create": (_I, [_I, ctypes.POINTER(_H), ctypes.POINTER(_H)]),
    "mg3d_batch_destroy": (_I, [_H]),
    "mg3d_batch_fas_vcycle": (_I, [_H, _I, _D]),
    "mg3d_batch_fas_solve": (_I, [_H, ctypes.c_double, _I, ctypes.POINTER(mg3d_stats)]),
    "mg3d_batch_fmg_solve": (_I, [_H, ctypes.c_double, _I, ctypes.POINTER(mg3d_stats)]),
    "mg3d_batch_counters": (_I, [_H, ctypes.POINTER(ctypes.c_longlong),
                                 ctypes.POINTER(ctypes.c_double)]),
    "mg3d_set_stream": (_I, [_H, ctypes.c_void_p]),
    "mg3d_level_shape": (_I, [_H, _I, ctypes.POINTER(_I), ctypes.POINTER(_I),
                              ctypes.POINTER(_I)]),
    "mg3d_get_populations": (_I, [_H, _I, _D]),
    "mg3d_set_populations": (_I, [_H, _I, _D]),
    "mg3d_init_zero_radiation": (_I, [_H, _I]),
    "mg3d_formal_solve": (_I, [_H, _I, _D, _D]),
    "mg3d_mali_sweep": (_I, [_H, _I, _I, _D]),
    "mg3d_residual": (_I, [_H, _I, _D]),
    "mg3d_fas_vcycle": (_I, [_H, _I, _D]),
    "mg3d_mali_solve": (_I, [_H, ctypes.c_double, _I, ctypes.POINTER(mg3d_stats)]),
    "mg3d_fas_solve": (_I, [_H, ctypes.c_double, _I, ctypes.POINTER(mg3d_stats)]),
    "mg3d_fmg_solve": (_I, [_H, ctypes.c_double, _I, ctypes.POINTER(mg3d_stats)]),
    "mg3d_restrict": (_I, [_H, _I, _I, _D, _D]),
    "mg3d_prolong": (_I, [_H, _I, _I, _D, _D]),
    "mg3d_set_fs_config": (_I, [_H, _I, _I, _I, _I, _I, _I]),
    "mg3d_get_fs_config": (_I, [_H, _I, ctypes.POINTER(_I), ctypes.POINTER(_I),
                                ctypes.POINTER(_I), ctypes.POINTER(_I), ctypes.POINTER(_I)]),
    "mg3d_set_ml_chunk": (_I, [_H, _I]),
    "mg3d_get_ml_chunk": (_I, [_H, ctypes.POINTER(_I)]),
    "mg3d_set_ml_shape": (_I, [_H, _I, _I, _I, _I]),
    "mg3d_set_ml_shape_ex": (_I, [_H, _I, _I, _I, _I, _I, _I]),
    "mg3d_get_ml_shape_ex": (_I, [_H, _I, ctypes.POINTER(_I), ctypes.POINTER(_I),
                                 ctypes.POINTER(_I), ctypes.POINTER(_I), ctypes.POINTER(_I)]),
    "mg3d_get_ml_shape": (_I, [_H, _I, ctypes.POINTER(_I), ctypes.POINTER(_I),
                               ctypes.POINTER(_I)]),
    "mg3d_get_fs_occupancy": (_I, [_H, _I, _I, _I, _I, _I, _I, ctypes.POINTER(_I),
                                   ctypes.POINTER(ctypes.c_longlong)]),
    "mg3d_autotune": (_I, [_H, _I, ctypes.POINTER(_I), ctypes.POINTER(ctypes.c_double)]),
    "mg3d_check_exp": (_I, [_I, _D, _D]),
    "mg3d_probe_alu_peaks": (_I, [_I, _D]),
    "mg3d_fmg_stage": (_I, [_H, _I]),
    "mg3d_formal_solve_ex": (_I, [_H, _I, _I, _D, _D]),
    "mg3d_formal_solve_dev": (_I, [_H, _I, _I, ctypes.c_void_p, ctypes.c_void_p,
                                   ctypes.c_void_p]),
    "mg3d_get_populations_dev": (_I, [_H, _I, ctypes.c_void_p, ctypes.c_void_p]),
    "mg3d_set_populations_dev": (_I, [_H, _I, ctypes.c_void_p, ctypes.c_void_p]),
    "mg3d_check_profiles": (_I, [_I, ctypes.c_double, _D, _D, _D]),
    "mg3d_check_voigt": (_I, [_I, _D, _D, _D]),
    "mg3d_set_graphs": (_I, [_H, _I]),
    "mg3d_set_timing": (_I, [_H, _I]),
    "mg3d_get_counters": (_I, [_H, ctypes.POINTER(mg3d_counters)]),
    "mg3d_reset_counters": (_I, [_H]),
    "mg3d_formal_solve_noalloc": (_I, [_I, _I, _I, ctypes.c_double, ctypes.c_double,
                                       ctypes.c_void_p, ctypes.POINTER(mg3d_atom),
                                       ctypes.c_double, ctypes.c_void_p, ctypes.c_void_p,
                                       ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p,
                                       ctypes.c_void_p]),
}

_lib = None


def library_path() -> str:
    return _build.LIB


def load(build_if_missing: bool = False):
    """Load libmg3d.so; raise if it is missing (no fallback of any kind)."""
    global _lib
    if _lib is not None:
        return _lib
    path = library_path()
    if not os.path.exists(path):
        if not build_if_missing:
            raise RuntimeError(f"CUDA library not built: {path} (run __graft_entry__.build())")
        _build.build()
    lib = ctypes.CDLL(path)
    for name, (res, args) in _SIGNATURES.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    _lib = lib
    return lib


class MG3DError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"mg3d error {code}: {msg}")
        self.code = code


def _check(rc):
    if rc != MG3D_OK:
        raise MG3DError(rc, load().mg3d_last_error().decode())
    return rc


def _dptr(a):
    if a is None:
        return None
    if a.dtype != np.float64 or not a.flags["C_CONTIGUOUS"]:
        raise ValueError("expected a C-contiguous float64 array")
    return a.ctypes.data_as(_D)


# ---------------------------------------------------------------- same names

def mg3d_last_error() -> str:
    return load().mg3d_last_error().decode()


def mg3d_create(atm, atom, quad_a: float = 0.0, n_grids: int = 1, nu_fmg: int = 16,
                nu0: int = 0, nu1: int = 2, nu2: int = 2, nu3: int = 32,
                fs_prec: int = MG3D_PREC_F64, restriction: int = MG3D_RESTRICT_FULL,
                interpolation: int = MG3D_INTERP_LINEAR, sc_interp: int = MG3D_INTERP_LINEAR):
    """mg3d_create from a synth.Atmosphere and TwoLevelAtom; returns the handle.

    Variants: ``restriction`` (MG3D_RESTRICT_*), ``interpolation`` and
    ``sc_interp`` (MG3D_INTERP_LINEAR or _HERMITE), a velocity field in
    ``atm.vel`` ([3, nz, ny, nx] in Doppler widths) and partial redistribution
    through ``atom.gamma_prd``; the C header documents each."""
    lib = load()
    z = np.ascontiguousarray(atm.z, dtype=np.float64)
    T = np.ascontiguousarray(atm.T, dtype=np.float64)
    n_tot = np.ascontiguousarray(atm.n_tot, dtype=np.float64)
    c_ul = np.ascontiguousarray(atm.c_ul, dtype=np.float64)
    vel = getattr(atm, "vel", None)
    vel = None if vel is None else np.ascontiguousarray(vel, dtype=np.float64)
    a = mg3d_atmosphere(atm.nx, atm.ny, atm.nz, atm.dx, atm.dy, _dptr(z), _dptr(T),
                        _dptr(n_tot), _dptr(c_ul), _dptr(vel))
    at = mg3d_atom(atom.a_ul, atom.g_ratio, atom.theta, atom.kappa, atom.n_freq, atom.x_max,
                   getattr(atom, "gamma_prd", 0.0), getattr(atom, "a_damp", 0.0))
    q = mg3d_quadrature(quad_a)
    p = mg3d_params(n_grids, nu_fmg, nu0, nu1, nu2, nu3, fs_prec, restriction, 0, interpolation,
                    sc_interp)
    h = _H()
    _check(lib.mg3d_create(ctypes.byref(a), ctypes.byref(at), ctypes.byref(q),
                           ctypes.byref(p), ctypes.byref(h)))
    return h


def mg3d_create_ml(atm, atom, quad_a: float = 0.0, n_grids: int = 1, nu_fmg: int = 16,
                   nu0: int = 0, nu1: int = 2, nu2: int = 2, nu3: int = 32,
                   fs_prec: int = MG3D_PREC_F64, restriction: int = MG3D_RESTRICT_FULL,
                   ml_chunk: int = 0, interpolation: int = MG3D_INTERP_LINEAR,
                   sc_interp: int = MG3D_INTERP_LINEAR):
    """mg3d_create_ml from a synth.MultiLevelAtmosphere and MultiLevelAtom.

    Variants: ``restriction``, ``interpolation``, ``sc_interp`` as for
    mg3d_create, background scattering in ``atm.sigma_c`` and a velocity
    field in ``atm.vel`` (Doppler widths at the atom's t_ref); ``ml_chunk``
    sets the frequencies per chunk (0: automatic)."""
    lib = load()
    keep = {}

    def arr(name, a):
        keep[name] = np.ascontiguousarray(a, dtype=np.float64)
        return _dptr(keep[name])

    sigma = getattr(atm, "sigma_c", None)
    vel = getattr(atm, "vel", None)
    a = mg3d_ml_atmosphere(atm.nx, atm.ny, atm.nz, atm.dx, atm.dy, arr("z", atm.z),
                           arr("T", atm.T), arr("n", atm.n_tot), arr("cc", atm.chi_c),
                           arr("c", atm.c), arr("s", atm.saha),
                           arr("sg", sigma) if sigma is not None else None,
                           arr("v", vel) if vel is not None else None)
    lines = (mg3d_line * max(1, len(atom.lines)))(
        *[mg3d_line(l.lower, l.upper, l.rho, l.a_ul, l.kappa, l.n_freq, l.x_max,
                    getattr(l, "a_damp", 0.0), getattr(l, "gamma_prd", 0.0))
          for l in atom.lines])
    conts = (mg3d_continuum * max(1, len(atom.continua)))(
        *[mg3d_continuum(c.lower, c.rho, c.beta, c.kappa, c.n_freq, c.y_max)
          for c in atom.continua])
    at = mg3d_ml_atom(atom.n_levels, arr("g", atom.g), arr("th", atom.theta), atom.theta_ref,
                      atom.t_ref, len(atom.lines), lines, len(atom.continua), conts)
    q = mg3d_quadrature(quad_a)
    p = mg3d_params(n_grids, nu_fmg, nu0, nu1, nu2, nu3, fs_prec, restriction, ml_chunk,
                    interpolation, sc_interp)
    h = _H()
    _check(lib.mg3d_create_ml(ctypes.byref(a), ctypes.byref(at), ctypes.byref(q),
                              ctypes.byref(p), ctypes.byref(h)))
    return h


def mg3d_n_levels(h):
    n, f = _I(), _I()
    _check(load().mg3d_n_levels(h, ctypes.byref(n), ctypes.byref(f)))
    return n.value, f.value


def mg3d_formal_solve_ml(h, level: int):
    nx, ny, nz = mg3d_level_shape(h, level)
    _, nf = mg3d_n_levels(h)
    jx = np.empty((nf, nz, ny, nx))
    ux = np.empty((nf, nz, ny, nx))
    _check(load().mg3d_formal_solve_ml(h, level, _dptr(jx), _dptr(ux)))
    return jx, ux


def mg3d_destroy(h):
    return _check(load().mg3d_destroy(h))


def mg3d_set_stream(h, stream_ptr: int | None):
    return _check(load().mg3d_set_stream(h, ctypes.c_void_p(stream_ptr or 0)))


def mg3d_level_shape(h, level: int):
    nx, ny, nz = _I(), _I(), _I()
    _check(load().mg3d_level_shape(h, level, ctypes.byref(nx), ctypes.byref(ny),
                                   ctypes.byref(nz)))
    return nx.value, ny.value, nz.value


def mg3d_get_populations(h, level: int, out=None):
    nx, ny, nz = mg3d_level_shape(h, level)
    if out is None:
        out = np.empty((mg3d_n_levels(h)[0], nz, ny, nx))
    _check(load().mg3d_get_populations(h, level, _dptr(out)))
    return out


def mg3d_set_populations(h, level: int, n):
    n = np.ascontiguousarray(n, dtype=np.float64)
    return _check(load().mg3d_set_populations(h, level, _dptr(n)))


def mg3d_init_zero_radiation(h, level: int):
    return _check(load().mg3d_init_zero_radiation(h, level))


def mg3d_formal_solve(h, level: int, want: bool = True):
    nx, ny, nz = mg3d_level_shape(h, level)
    jeff = np.empty((nz, ny, nx)) if want else None
    u = np.empty((nz, ny, nx)) if want else None
    _check(load().mg3d_formal_solve(h, level, _dptr(jeff), _dptr(u)))
    return jeff, u


def mg3d_formal_solve_ex(h, level: int, prec: int, want: bool = True):
    """Formal solution in precision ``prec``; host outputs like mg3d_formal_solve."""
    nx, ny, nz = mg3d_level_shape(h, level)
    jeff = np.empty((nz, ny, nx)) if want else None
    u = np.empty((nz, ny, nx)) if want else None
    _check(load().mg3d_formal_solve_ex(h, level, prec, _dptr(jeff), _dptr(u)))
    return jeff, u


def mg3d_formal_solve_dev(h, level: int, prec: int, jeff_dev: int | None, u_dev: int | None,
                          stream_ptr: int | None = None):
    """Formal solution into device buffers (addresses, e.g. tensor.data_ptr()),
    ordered on the CUDA stream ``stream_ptr``; does not synchronise."""
    return _check(load().mg3d_formal_solve_dev(h, level, prec, ctypes.c_void_p(jeff_dev or 0),
                                               ctypes.c_void_p(u_dev or 0),
                                               ctypes.c_void_p(stream_ptr or 0)))


def mg3d_get_populations_dev(h, level: int, n_dev: int, stream_ptr: int | None = None):
    return _check(load().mg3d_get_populations_dev(h, level, ctypes.c_void_p(n_dev),
                                                  ctypes.c_void_p(stream_ptr or 0)))


def mg3d_set_populations_dev(h, level: int, n_dev: int, stream_ptr: int | None = None):
    return _check(load().mg3d_set_populations_dev(h, level, ctypes.c_void_p(n_dev),
                                                  ctypes.c_void_p(stream_ptr or 0)))


def mg3d_mali_sweep(h, level: int, n_sweeps: int = 1) -> float:
    c = ctypes.c_double()
    _check(load().mg3d_mali_sweep(h, level, n_sweeps, ctypes.byref(c)))
    return c.value


def mg3d_residual(h, level: int):
    nx, ny, nz = mg3d_level_shape(h, level)
    r = np.empty((mg3d_n_levels(h)[0], nz, ny, nx))
    _check(load().mg3d_residual(h, level, _dptr(r)))
    return r


def mg3d_fas_vcycle(h, is_first: bool = False) -> float:
    c = ctypes.c_double()
    _check(load().mg3d_fas_vcycle(h, int(bool(is_first)), ctypes.byref(c)))
    return c.value


def _stats_dict(st: mg3d_stats, n_grids: int):
    return {"iterations": st.iterations,
            "sweeps": {k: st.sweeps[k] for k in range(1, n_grids + 1)},
            "formal_solutions": {k: st.formal_solutions[k] for k in range(1, n_grids + 1)},
            "last_change": st.last_change, "negatives": st.negatives,
            "seconds": st.seconds, "fine_fs_equivalents": st.fine_fs_equivalents}


def _solve(fn, h, tol, cap, n_grids):
    st = mg3d_stats()
    _check(fn(h, tol, cap, ctypes.byref(st)))
    return _stats_dict(st, n_grids)


def mg3d_mali_solve(h, tol: float, max_sweeps: int = 100000, n_grids: int = 1):
    return _solve(load().mg3d_mali_solve, h, tol, max_sweeps, n_grids)


def mg3d_fas_solve(h, tol: float, max_cycles: int = 1000, n_grids: int = 1):
    return _solve(load().mg3d_fas_solve, h, tol, max_cycles, n_grids)


def mg3d_fmg_solve(h, tol: float, max_cycles: int = 1000, n_grids: int = 1):
    return _solve(load().mg3d_fmg_solve, h, tol, max_cycles, n_grids)


def mg3d_fmg_stage(h, stage: int):
    return _check(load().mg3d_fmg_stage(h, stage))


def mg3d_restrict(h, level_fine: int, fine):
    fine = np.ascontiguousarray(fine, dtype=np.float64)
    ncomp = fine.shape[0] if fine.ndim == 4 else 1
    nx, ny, nz = mg3d_level_shape(h, level_fine - 1)
    out = np.empty((ncomp, nz, ny, nx))
    _check(load().mg3d_restrict(h, level_fine, ncomp, _dptr(fine), _dptr(out)))
    return out if fine.ndim == 4 else out[0]


def mg3d_prolong(h, level_fine: int, coarse):
    coarse = np.ascontiguousarray(coarse, dtype=np.float64)
    ncomp = coarse.shape[0] if coarse.ndim == 4 else 1
    nx, ny, nz = mg3d_level_shape(h, level_fine)
    out = np.empty((ncomp, nz, ny, nx))
    _check(load().mg3d_prolong(h, level_fine, ncomp, _dptr(coarse), _dptr(out)))
    return out if coarse.ndim == 4 else out[0]


def mg3d_set_fs_config(h, level: int, freq_per_block: int, bands: int, threads: int = 256,
                       lean: int = 0, stage: int = 1):
    return _check(load().mg3d_set_fs_config(h, level, freq_per_block, bands, threads, lean,
                                            stage))


def mg3d_get_fs_config(h, level: int):
    """(freq_per_block, bands, threads, lean, stage) of a level's sweep."""
    v = [_I() for _ in range(5)]
    _check(load().mg3d_get_fs_config(h, level, *[ctypes.byref(x) for x in v]))
    return tuple(x.value for x in v)


def mg3d_set_ml_chunk(h, freq_per_chunk: int):
    """Frequencies per chunk of a multi-level formal solution (0: all)."""
    return _check(load().mg3d_set_ml_chunk(h, freq_per_chunk))


def mg3d_get_ml_chunk(h) -> int:
    c = _I()
    _check(load().mg3d_get_ml_chunk(h, ctypes.byref(c)))
    return c.value


def mg3d_set_ml_shape(h, level: int, bands: int, rays_per_block: int, threads: int = 256):
    return _check(load().mg3d_set_ml_shape(h, level, bands, rays_per_block, threads))


def mg3d_get_ml_shape(h, level: int):
    """(bands, rays_per_block, threads) of a level's multi-level sweep."""
    v = [_I() for _ in range(3)]
    _check(load().mg3d_get_ml_shape(h, level, *[ctypes.byref(x) for x in v]))
    return tuple(x.value for x in v)


def mg3d_set_ml_shape_ex(h, level: int, bands: int, rays_per_block: int, threads: int,
                         kind: int, freq_per_block: int = 1):
    return _check(load().mg3d_set_ml_shape_ex(h, level, bands, rays_per_block, threads, kind,
                                              freq_per_block))


def mg3d_get_ml_shape_ex(h, level: int):
    b, r, t, k, f = _I(), _I(), _I(), _I(), _I()
    _check(load().mg3d_get_ml_shape_ex(h, level, ctypes.byref(b), ctypes.byref(r),
                                       ctypes.byref(t), ctypes.byref(k), ctypes.byref(f)))
    return b.value, r.value, t.value, k.value, f.value


def mg3d_get_fs_occupancy(h, level: int, freq_per_block: int, bands: int, threads: int = 256,
                          lean: int = 0, stage: int = 1):
    """(clusters the GPU holds at once, dynamic shared memory bytes per block)."""
    n, smem = _I(), ctypes.c_longlong()
    _check(load().mg3d_get_fs_occupancy(h, level, freq_per_block, bands, threads, lean, stage,
                                        ctypes.byref(n), ctypes.byref(smem)))
    return n.value, smem.value


def mg3d_autotune(h, level: int = 0):
    n = _I()
    secs = ctypes.c_double()
    _check(load().mg3d_autotune(h, level, ctypes.byref(n), ctypes.byref(secs)))
    return {"evaluated": n.value, "seconds": secs.value}


def mg3d_probe_alu_peaks(reps: int = 3):
    """Measured peak rates (thread operations per second) of FP32 FMA, the ex2
    and rcp approximations and FP64 FMA on the current device."""
    out = np.empty(4)
    _check(load().mg3d_probe_alu_peaks(reps, _dptr(out)))
    return {"ffma": out[0], "ex2": out[1], "rcp": out[2], "dfma": out[3]}


def mg3d_check_exp(x):
    x = np.ascontiguousarray(x, dtype=np.float64)
    out = np.empty(2 * x.size)
    _check(load().mg3d_check_exp(x.size, _dptr(x), _dptr(out)))
    return out[0::2], out[1::2]


def mg3d_check_profiles(a: float, x, xp):
    """(H(a, x), R_II-A(x, xp)) as the library's host tables compute them."""
    x = np.ascontiguousarray(x, dtype=np.float64)
    xp = np.ascontiguousarray(np.broadcast_to(xp, x.shape), dtype=np.float64)
    out = np.empty(2 * x.size)
    _check(load().mg3d_check_profiles(x.size, float(a), _dptr(x), _dptr(xp), _dptr(out)))
    return out[0::2], out[1::2]


def mg3d_check_voigt(a, x):
    """H(a, x) by the library's rational Voigt function (host code)."""
    x = np.ascontiguousarray(x, dtype=np.float64)
    a = np.ascontiguousarray(np.broadcast_to(a, x.shape), dtype=np.float64)
    out = np.empty(x.size)
    _check(load().mg3d_check_voigt(x.size, _dptr(a), _dptr(x), _dptr(out)))
    return out.reshape(x.shape)


def mg3d_set_graphs(h, enable: bool):
    return _check(load().mg3d_set_graphs(h, int(bool(enable))))


def mg3d_set_timing(h, enable: bool):
    return _check(load().mg3d_set_timing(h, int(bool(enable))))


def mg3d_get_counters(h):
    c = mg3d_counters()
    _check(load().mg3d_get_counters(h, ctypes.byref(c)))
    lv = range(MG3D_MAX_GRIDS + 1)
    return {"kernel_launches": c.kernel_launches, "fs_launches": c.fs_launches,
            "fs_units": c.fs_units, "fs_kernel_ms": c.fs_kernel_ms,
            "fs_timed_launches": c.fs_timed_launches,
            "level_fs_launches": [c.level_fs_launches[k] for k in lv],
            "level_fs_units": [c.level_fs_units[k] for k in lv],
            "level_fs_kernel_ms": [c.level_fs_kernel_ms[k] for k in lv],
            "level_fs_timed_launches": [c.level_fs_timed_launches[k] for k in lv]}


def mg3d_reset_counters(h):
    return _check(load().mg3d_reset_counters(h))


def mg3d_formal_solve_noalloc(nx: int, ny: int, nz: int, dx: float, dy: float, z_dev: int,
                              atom, quad_a: float, chi0_dev: int, S_dev: int, bbot_dev: int,
                              jeff_dev: int, u_dev: int, stream_ptr: int | None = None) -> int:
    """Allocation-free formal solution on caller-owned device buffers.

    All buffer arguments are device addresses (e.g. a torch tensor's
    data_ptr()); returns the library's status code without raising, so that
    callers can inspect limit errors.
    """
    at = mg3d_atom(atom.a_ul, atom.g_ratio, atom.theta, atom.kappa, atom.n_freq, atom.x_max,
                   getattr(atom, "gamma_prd", 0.0), getattr(atom, "a_damp", 0.0))
    return load().mg3d_formal_solve_noalloc(nx, ny, nz, dx, dy, z_dev, ctypes.byref(at),
                                            quad_a, chi0_dev, S_dev, bbot_dev, jeff_dev,
                                            u_dev, stream_ptr)


# ------------------------------------------------------------------ batches

def mg3d_batch_create(handles):
    arr = (_H * len(handles))(*[h.value if isinstance(h, _H) else h for h in handles])
    b = _H()
    _check(load().mg3d_batch_create(len(handles), arr, ctypes.byref(b)))
    return b


def mg3d_batch_destroy(b):
    return _check(load().mg3d_batch_destroy(b))


def mg3d_batch_fas_vcycle(b, n: int, is_first: bool = False):
    c = np.empty(n)
    _check(load().mg3d_batch_fas_vcycle(b, int(bool(is_first)), _dptr(c)))
    return c


def _batch_solve(fn, b, n, tol, cap, n_grids):
    st = (mg3d_stats * n)()
    _check(fn(b, tol, cap, st))
    return [_stats_dict(st[i], n_grids) for i in range(n)]


def mg3d_batch_fas_solve(b, n: int, tol: float, max_cycles: int = 1000, n_grids: int = 1):
    return _batch_solve(load().mg3d_batch_fas_solve, b, n, tol, max_cycles, n_grids)


def mg3d_batch_fmg_solve(b, n: int, tol: float, max_cycles: int = 1000, n_grids: int = 1):
    return _batch_solve(load().mg3d_batch_fmg_solve, b, n, tol, max_cycles, n_grids)


def mg3d_batch_counters(b):
    l, u = ctypes.c_longlong(), ctypes.c_double()
    _check(load().mg3d_batch_counters(b, ctypes.byref(l), ctypes.byref(u)))
    return {"kernel_launches": l.value, "fs_units": u.value}
