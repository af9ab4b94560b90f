"""GPU parity of partial redistribution (two-level atom) through the C ABI
against the oracle.  The lagged mean intensity is internal state, so parity
is checked through iterations: MALI sweeps (the first sees CRD), formal
solutions after them, V-cycles and FMG."""

import numpy as np
import pytest

from oracle import mg3d_oracle as O
from paper_1701_01607_gb300 import mg3d as m
from paper_1701_01607_gb300 import synth

pytestmark = pytest.mark.gpu

PARAMS = dict(nu_fmg=16, nu0=0, nu1=2, nu2=2, nu3=32)
TOL_POP64 = 1e-10


def rel(a, b):
    return float(np.max(np.abs(a - b) / np.abs(b)))


@pytest.fixture(scope="module", autouse=True)
def lib():
    m.load(build_if_missing=True)


def prd_box(nx=16, ny=16, nz=33, gamma=0.9, seed=5, eps=1e-3, n_freq=9):
    atom = synth.TwoLevelAtom(gamma_prd=gamma, n_freq=n_freq)
    return synth.stratified_two_level(nx, ny, nz, eps=eps, sigma=0.3, seed=seed, atom=atom)


@pytest.mark.parametrize("shape,config", [((16, 16, 33), None), ((12, 8, 17), (4, 3, 128, 0)),
                                          ((16, 16, 17), (2, 6, 64, 2)),
                                          ((8, 31, 9), (9, 16, 32, 1)), ((2, 2, 9), None)])
def test_prd_sweeps_and_formal_solution_fp64(shape, config):
    """Three MALI sweeps (the lagged field enters from the second), then a
    formal solution; odd and even frequency groups map table positions to
    natural frequencies both ways."""
    atm, atom = prd_box(*shape)
    p = O.TwoLevelProblem(atm, atom)
    n = p.zero_radiation(1)
    h = m.mg3d_create(atm, atom, n_grids=1, **PARAMS)
    try:
        if config is not None:
            m.mg3d_set_fs_config(h, 1, *config, 0)
        for _ in range(3):
            c_gpu = m.mg3d_mali_sweep(h, 1, 1)
            n, c_orc = p.mali_sweep(1, n)
            assert abs(c_gpu - c_orc) <= 1e-8 * c_orc
        assert rel(m.mg3d_get_populations(h, 1), n) < TOL_POP64
        jeff, u = m.mg3d_formal_solve(h, 1)
    finally:
        m.mg3d_destroy(h)
    _, jo, uo = p.formal_solution(1, n)
    assert rel(jeff, jo) < 1e-11 and rel(u, uo) < 1e-11


@pytest.mark.parametrize("n_grids", [2, 3])
def test_prd_fas_vcycles_and_fmg_fp64(n_grids):
    atm, atom = prd_box()
    h = m.mg3d_create(atm, atom, n_grids=n_grids, **PARAMS)
    p = O.TwoLevelProblem(atm, atom, n_grids=n_grids)
    n = p.zero_radiation(n_grids)
    try:
        for cyc in range(2):
            c_gpu = m.mg3d_fas_vcycle(h, cyc == 0)
            n, c_orc = p.fas_cycle(n, cyc == 0, PARAMS)
            assert abs(c_gpu - c_orc) <= 1e-8 * c_orc
            assert rel(m.mg3d_get_populations(h, n_grids), n) < TOL_POP64
        st = m.mg3d_fmg_solve(h, 1e-3, n_grids=n_grids)
        n_fmg = m.mg3d_get_populations(h, n_grids)
    finally:
        m.mg3d_destroy(h)
    p2 = O.TwoLevelProblem(atm, atom, n_grids=n_grids)
    n_f, cyc = O.fmg_solve(p2, 1e-3, PARAMS)
    assert st["iterations"] == cyc
    assert rel(n_fmg, n_f) < TOL_POP64


def test_prd_fp32_autotuned_and_differs_from_crd():
    atm, atom = prd_box(gamma=1.0, n_freq=17)
    p = O.TwoLevelProblem(atm, atom)
    n = p.zero_radiation(1)
    for _ in range(6):
        n, _ = p.mali_sweep(1, n)
    h = m.mg3d_create(atm, atom, n_grids=1, fs_prec=m.MG3D_PREC_F32, **PARAMS)
    try:
        m.mg3d_autotune(h)
        assert m.mg3d_get_fs_config(h, 1)[4] == 0
        m.mg3d_mali_sweep(h, 1, 6)
        n_gpu = m.mg3d_get_populations(h, 1)
    finally:
        m.mg3d_destroy(h)
    assert rel(n_gpu, n) < 1e-4
    atom.gamma_prd = 0.0
    q = O.TwoLevelProblem(atm, atom)
    nc = q.zero_radiation(1)
    for _ in range(6):
        nc, _ = q.mali_sweep(1, nc)
    assert rel(nc, n) > 1e-3


def test_prd_refusals():
    atm, atom = prd_box(8, 8, 17)
    with pytest.raises(m.MG3DError, match="static atmosphere"):
        m.mg3d_create(atm, atom, n_grids=1, sc_interp=m.MG3D_INTERP_HERMITE, **PARAMS)
    atom.gamma_prd = 1.5
    with pytest.raises(m.MG3DError, match="gamma_prd"):
        m.mg3d_create(atm, atom, n_grids=1, **PARAMS)
    atom.gamma_prd = 0.5
    h = m.mg3d_create(atm, atom, n_grids=2, **PARAMS)
    try:
        with pytest.raises(m.MG3DError, match="unstaged"):
            m.mg3d_set_fs_config(h, 2, 3, 2, 128, 0, 1)
        with pytest.raises(m.MG3DError, match="partial redistribution"):
            m.mg3d_batch_create([h])
    finally:
        m.mg3d_destroy(h)
    vatm, _ = synth.stratified_two_level(8, 8, 17, eps=1e-3, atom=atom, velocity=1.0)
    with pytest.raises(m.MG3DError, match="static atmosphere"):
        m.mg3d_create(vatm, atom, n_grids=1, **PARAMS)


# ------------------------------------------------------------ damping (Voigt)

def test_damped_crd_formal_solution_and_prd_sweeps_fp64():
    """Voigt profiles (a = 0.05) and, with full coherence, R_II-A: the formal
    solution after the zero-radiation start (CRD) and three MALI sweeps with
    partial redistribution against the oracle."""
    atom = synth.TwoLevelAtom(n_freq=13, x_max=5.0, a_damp=0.05)
    atm, atom = synth.stratified_two_level(16, 16, 33, eps=1e-3, sigma=0.3, seed=5, atom=atom)
    h = m.mg3d_create(atm, atom, n_grids=1, **PARAMS)
    try:
        jeff, u = m.mg3d_formal_solve(h, 1)
    finally:
        m.mg3d_destroy(h)
    p = O.TwoLevelProblem(atm, atom)
    _, jo, uo = p.formal_solution(1, p.zero_radiation(1))
    assert rel(jeff, jo) < 1e-12 and rel(u, uo) < 1e-12

    atom.gamma_prd = 1.0
    p = O.TwoLevelProblem(atm, atom, n_grids=2)
    n = p.zero_radiation(2)
    h = m.mg3d_create(atm, atom, n_grids=2, **PARAMS)
    try:
        for _ in range(3):
            m.mg3d_mali_sweep(h, 2, 1)
            n, _ = p.mali_sweep(2, n)
        assert rel(m.mg3d_get_populations(h, 2), n) < TOL_POP64
        c_gpu = m.mg3d_fas_vcycle(h, False)
        n, c_orc = p.fas_cycle(n, False, PARAMS)
        assert abs(c_gpu - c_orc) <= 1e-8 * c_orc
        assert rel(m.mg3d_get_populations(h, 2), n) < TOL_POP64
    finally:
        m.mg3d_destroy(h)


def test_prd_is_bit_reproducible():
    """The new mean intensity is stored per ray and summed in ray order, so
    two runs of the same problem agree bit for bit."""
    atm, atom = prd_box(gamma=1.0)
    out = []
    for _ in range(2):
        h = m.mg3d_create(atm, atom, n_grids=2, **PARAMS)
        try:
            m.mg3d_mali_sweep(h, 2, 3)
            m.mg3d_fas_vcycle(h, False)
            out.append(m.mg3d_get_populations(h, 2))
        finally:
            m.mg3d_destroy(h)
    assert np.array_equal(out[0], out[1])
