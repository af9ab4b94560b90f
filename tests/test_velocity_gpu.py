"""GPU parity of moving atmospheres (two-level atom, CRD with Doppler-shifted
profiles) through the C ABI against the oracle."""

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
