"""GPU parity of moving atmospheres (two-level and multi-level atoms, CRD with
Doppler-shifted profiles) through the C ABI against the oracle."""

import numpy as np
import pytest

from oracle import mg3d_oracle as O
from paper_1701_01607_gb300 import mg3d as m
from paper_1701_01607_gb300 import synth

pytestmark = pytest.mark.gpu

PARAMS = dict(nu_fmg=16, nu0=0, nu1=2, nu2=2, nu3=32)
TOL_FS64 = 1e-12
TOL_POP64 = 1e-10


def rel(a, b):
    return float(np.max(np.abs(a - b) / np.abs(b)))


@pytest.fixture(scope="module", autouse=True)
def lib():
    m.load(build_if_missing=True)


def moving(nx, ny, nz, velocity=1.0, seed=11, eps=1e-3):
    return synth.stratified_two_level(nx, ny, nz, eps=eps, sigma=0.3, seed=seed,
                                      velocity=velocity)


def _fs_parity(atm, atom, tol, prec=m.MG3D_PREC_F64, config=None):
    h = m.mg3d_create(atm, atom, n_grids=1, fs_prec=prec, **PARAMS)
    try:
        if config is not None:
            m.mg3d_set_fs_config(h, 1, *config, 0)
            assert m.mg3d_get_fs_config(h, 1) == tuple(config) + (0,)
        jeff, u = m.mg3d_formal_solve(h, 1)
    finally:
        m.mg3d_destroy(h)
    prob = O.TwoLevelProblem(atm, atom)
    _, jo, uo = prob.formal_solution(1, prob.zero_radiation(1))
    assert rel(jeff, jo) < tol
    assert rel(u, uo) < tol
    return jeff


@pytest.mark.parametrize("shape", [(16, 16, 33), (12, 8, 17), (2, 2, 9), (1, 1, 3)])
def test_moving_formal_solution_fp64(shape):
    atm, atom = moving(*shape)
    _fs_parity(atm, atom, TOL_FS64)


@pytest.mark.parametrize("ng,bands,th,lean", [(1, 1, 128, 0), (9, 1, 128, 1), (4, 3, 128, 0),
                                              (2, 6, 64, 2), (3, 8, 128, 0), (5, 16, 32, 1)])
def test_moving_formal_solution_every_launch_shape(ng, bands, th, lean):
    """Ragged frequency groups and bands: the opacity planes, like the
    intensity planes, are read across the blocks of a cluster."""
    atm, atom = moving(16, 16, 17, seed=2)
    _fs_parity(atm, atom, TOL_FS64, config=(ng, bands, th, lean))


def test_moving_fp32_and_flow_matters():
    atm, atom = moving(16, 16, 33, velocity=1.5)
    j_move = _fs_parity(atm, atom, 1e-5, prec=m.MG3D_PREC_F32)
    atm.vel = None
    h = m.mg3d_create(atm, atom, n_grids=1, fs_prec=m.MG3D_PREC_F32, **PARAMS)
    try:
        j_static, _ = m.mg3d_formal_solve(h, 1)
    finally:
        m.mg3d_destroy(h)
    assert rel(j_move, j_static) > 1e-3


@pytest.mark.parametrize("n_grids", [2, 3])
def test_moving_mali_and_fas_vcycles_fp64(n_grids):
    atm, atom = moving(16, 16, 33, seed=5)
    h = m.mg3d_create(atm, atom, n_grids=n_grids, **PARAMS)
    prob = O.TwoLevelProblem(atm, atom, n_grids=n_grids)
    n = prob.zero_radiation(n_grids)
    try:
        for _ in range(2):
            c_gpu = m.mg3d_mali_sweep(h, n_grids, 1)
            n, c_orc = prob.mali_sweep(n_grids, n)
            assert abs(c_gpu - c_orc) <= 1e-8 * c_orc
        for _ in range(2):
            c_gpu = m.mg3d_fas_vcycle(h, False)
            n, c_orc = prob.fas_cycle(n, False, PARAMS)
            assert abs(c_gpu - c_orc) <= 1e-8 * c_orc
            assert rel(m.mg3d_get_populations(h, n_grids), n) < TOL_POP64
    finally:
        m.mg3d_destroy(h)


def test_moving_fmg_and_autotune_fp64():
    atm, atom = moving(16, 16, 33, seed=6)
    h = m.mg3d_create(atm, atom, n_grids=3, **PARAMS)
    try:
        with pytest.raises(m.MG3DError, match="unstaged"):
            m.mg3d_set_fs_config(h, 3, 3, 2, 128, 0, 1)
        m.mg3d_autotune(h)
        assert all(m.mg3d_get_fs_config(h, k)[4] == 0 for k in (1, 2, 3))
        st = m.mg3d_fmg_solve(h, 1e-3, n_grids=3)
        n_fmg = m.mg3d_get_populations(h, 3)
    finally:
        m.mg3d_destroy(h)
    prob = O.TwoLevelProblem(atm, atom, n_grids=3)
    n_f, cyc = O.fmg_solve(prob, 1e-3, PARAMS)
    assert st["iterations"] == cyc
    assert rel(n_fmg, n_f) < TOL_POP64


def test_moving_refusals():
    atm, atom = moving(8, 8, 17)
    with pytest.raises(m.MG3DError, match="linear upwind"):
        m.mg3d_create(atm, atom, n_grids=1, sc_interp=m.MG3D_INTERP_HERMITE, **PARAMS)
    h = m.mg3d_create(atm, atom, n_grids=2, **PARAMS)
    try:
        with pytest.raises(m.MG3DError, match="moving"):
            m.mg3d_batch_create([h])
    finally:
        m.mg3d_destroy(h)


# ----------------------------------------------------------- multi-level atom

def moving_ml(nx=8, ny=8, nz=17, velocity=1.0, scattering=0.0, seed=2):
    atom = synth.hydrogen_like_atom(line_freq=7, cont_freq=4, seed=seed)
    atm = synth.chromosphere(nx, ny, nz, atom, seed=seed, velocity=velocity,
                             scattering=scattering)
    return atm, atom


def per_freq_err(got, ref):
    nf = ref.shape[0]
    err = np.max(np.abs(got.reshape(nf, -1) - ref), axis=1) / np.max(np.abs(ref), axis=1)
    return float(np.max(err))


@pytest.mark.parametrize("shape,rpb,bands,chunk", [((8, 8, 17), 12, 1, 0), ((8, 8, 17), 3, 4, 11),
                                                   ((12, 8, 9), 6, 8, 0), ((2, 2, 5), 12, 2, 7)])
def test_moving_ml_formal_solution_and_mali_fp64(shape, rpb, bands, chunk):
    """Profile-weighted angle sums per frequency, then two MALI sweeps, with
    ray groups, bands of one or two rows and chunks that split lines."""
    atm, atom = moving_ml(*shape)
    p = O.MultiLevelProblem(atm, atom)
    n0 = p.zero_radiation(1)
    Jo, Uo, _ = p.formal_solution(1, n0)
    n1, _ = p.mali_sweep(1, n0)
    n2, _ = p.mali_sweep(1, n1)
    h = m.mg3d_create_ml(atm, atom, n_grids=1, ml_chunk=chunk)
    try:
        m.mg3d_set_ml_shape(h, 1, bands, rpb, 64)
        jx, ux = m.mg3d_formal_solve_ml(h, 1)
        assert per_freq_err(jx, Jo) < 1e-11 and per_freq_err(ux, Uo) < 1e-11
        m.mg3d_mali_sweep(h, 1, 2)
        assert rel(m.mg3d_get_populations(h, 1), n2) < TOL_POP64
    finally:
        m.mg3d_destroy(h)


def test_moving_ml_fas_fmg_with_scattering_fp64():
    """Flow and background scattering through 2-grid V-cycles and FMG: the
    coarse background field is restricted, Lambda-iterated once and then
    held (the oracle's reading)."""
    atm, atom = moving_ml(16, 16, 33, scattering=1.0)
    ml = dict(nu_fmg=8, nu0=4, nu1=2, nu2=2, nu3=16)
    h = m.mg3d_create_ml(atm, atom, n_grids=2, **ml)
    p = O.MultiLevelProblem(atm, atom, n_grids=2)
    n = p.zero_radiation(2)
    try:
        for cyc in range(2):
            c_gpu = m.mg3d_fas_vcycle(h, cyc == 0)
            n, c_orc = p.fas_cycle(n, cyc == 0, ml)
            assert abs(c_gpu - c_orc) <= 1e-6 * c_orc
            assert rel(m.mg3d_get_populations(h, 2), n) < TOL_POP64
        st = m.mg3d_fmg_solve(h, 1e-6, n_grids=2)
        n_gpu = m.mg3d_get_populations(h, 2)
    finally:
        m.mg3d_destroy(h)
    p2 = O.MultiLevelProblem(atm, atom, n_grids=2)
    n_o, cyc = O.fmg_solve(p2, 1e-6, ml)
    assert st["iterations"] == cyc
    assert rel(n_gpu, n_o) < TOL_POP64


def test_moving_ml_fp32_autotuned_and_refusals():
    atm, atom = moving_ml()
    h = m.mg3d_create_ml(atm, atom, n_grids=1, fs_prec=m.MG3D_PREC_F32)
    p = O.MultiLevelProblem(atm, atom)
    n = p.zero_radiation(1)
    Jo, Uo, _ = p.formal_solution(1, n)
    try:
        m.mg3d_autotune(h)
        jx, ux = m.mg3d_formal_solve_ml(h, 1)
        assert per_freq_err(jx, Jo) < 1e-5 and per_freq_err(ux, Uo) < 1e-5
        m.mg3d_mali_sweep(h, 1, 4)
        for _ in range(4):
            n, _ = p.mali_sweep(1, n)
        assert rel(m.mg3d_get_populations(h, 1), n) < 1e-4
    finally:
        m.mg3d_destroy(h)
    with pytest.raises(m.MG3DError, match="linear upwind"):
        m.mg3d_create_ml(atm, atom, n_grids=1, sc_interp=m.MG3D_INTERP_HERMITE)
