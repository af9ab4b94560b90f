"""Partial redistribution of multi-level lines on the GPU against the oracle.

The next step Sec. 6 names, in the oracle's reading: each PRD line (the
resonance lines of the seeded hydrogen-like atom, coherence fraction gamma)
emits with the profile rho_f phi_f, rho_f = 1 + gamma f_rad (sum_f' wq_f'
R(f', f) J_f' / (phi_f Jbar) - 1), with R the angle-averaged Doppler
redistribution at each node's Doppler width scaled symmetrically to the
node's profile, J the lagged mean intensity of the previous formal solution
on the grid and f_rad the radiative share of the inflow into the upper
level.  The GPU computes the scaling once per grid and rho before each
formal solution; the opacity step applies it to the source function and to
the transition's shares.  Bars: populations to 1e-10 after a fixed number of
FP64 sweeps, V-cycles or an FMG solve; 1e-5 with the FP32 formal solution
(after sweeps, and converged against the converged oracle).
"""

import numpy as np
import pytest

from oracle import mg3d_oracle as O
from paper_1701_01607_gb300 import mg3d as m
from paper_1701_01607_gb300 import synth

pytestmark = pytest.mark.gpu

PARAMS = dict(nu_fmg=8, nu0=10, nu1=2, nu2=4, nu3=16)


def rel(a, b):
    return float(np.max(np.abs(a - b) / np.abs(b)))


@pytest.fixture(scope="module", autouse=True)
def lib():
    m.load(build_if_missing=True)


def prd_box(gamma=1.0, nx=8, nz=17, line_freq=7, scattering=0.0):
    atom = synth.hydrogen_like_atom(line_freq=line_freq, cont_freq=4, seed=2, gamma_prd=gamma)
    atm = synth.chromosphere(nx, nx, nz, atom, seed=2, ground_collisions=1e-3,
                             scattering=scattering)
    return atm, atom


@pytest.mark.parametrize("gamma", [0.5, 1.0])
def test_ml_prd_mali_sweeps_fp64(gamma):
    atm, atom = prd_box(gamma)
    p = O.MultiLevelProblem(atm, atom)
    n = p.zero_radiation(1)
    h = m.mg3d_create_ml(atm, atom, n_grids=1)
    try:
        assert rel(m.mg3d_get_populations(h, 1), n) < 1e-11
        for sweep in range(4):
            c_gpu = m.mg3d_mali_sweep(h, 1, 1)
            n, c_o = p.mali_sweep(1, n)
            assert rel(m.mg3d_get_populations(h, 1), n) < 1e-10, sweep
            assert abs(c_gpu - c_o) <= 1e-8 * c_o
    finally:
        m.mg3d_destroy(h)
    # the redistribution did something: the populations differ from CRD's
    atm_c, atom_c = prd_box(0.0)
    pc = O.MultiLevelProblem(atm_c, atom_c)
    nc = pc.zero_radiation(1)
    for _ in range(4):
        nc, _ = pc.mali_sweep(1, nc)
    assert rel(n, nc) > 1e-6


def test_ml_prd_vcycles_and_fmg_fp64():
    atm, atom = prd_box(1.0, nx=8, nz=17)
    p = O.MultiLevelProblem(atm, atom, n_grids=2)
    n = p.zero_radiation(2)
    h = m.mg3d_create_ml(atm, atom, n_grids=2, **PARAMS)
    try:
        for cyc in range(2):
            m.mg3d_fas_vcycle(h, cyc == 0)
            n, _ = p.fas_cycle(n, cyc == 0, PARAMS)
            assert rel(m.mg3d_get_populations(h, 2), n) < 1e-10, cyc
    finally:
        m.mg3d_destroy(h)
    p2 = O.MultiLevelProblem(atm, atom, n_grids=2)
    n_f, cycles = O.fmg_solve(p2, 1e-3, PARAMS)
    h = m.mg3d_create_ml(atm, atom, n_grids=2, **PARAMS)
    try:
        st = m.mg3d_fmg_solve(h, 1e-3, 40, n_grids=2)
        assert st["iterations"] == cycles
        assert rel(m.mg3d_get_populations(h, 2), n_f) < 1e-10
    finally:
        m.mg3d_destroy(h)


def test_ml_prd_with_background_scattering_fp64():
    """PRD lines and background scattering read the same lagged field (the
    zero-radiation start Lambda-iterates it for the scattering): MALI sweeps
    and a 2-grid V-cycle against the oracle."""
    atm, atom = prd_box(1.0, nx=8, nz=17, scattering=1.0)
    p = O.MultiLevelProblem(atm, atom, n_grids=2)
    n = p.zero_radiation(2)
    h = m.mg3d_create_ml(atm, atom, n_grids=2, **PARAMS)
    try:
        assert rel(m.mg3d_get_populations(h, 2), n) < 1e-10
        for _ in range(2):
            m.mg3d_mali_sweep(h, 2, 1)
            n, _ = p.mali_sweep(2, n)
        assert rel(m.mg3d_get_populations(h, 2), n) < 1e-10
        m.mg3d_fas_vcycle(h, False)
        n, _ = p.fas_cycle(n, False, PARAMS)
        assert rel(m.mg3d_get_populations(h, 2), n) < 1e-10
    finally:
        m.mg3d_destroy(h)


def test_ml_prd_chunks_and_ray_groups():
    """The ratios are formed once per formal solution for all frequencies:
    frequency chunks that split a PRD line and blocks of 3 rays give the
    oracle's populations."""
    atm, atom = prd_box(0.7, nx=8, nz=17)
    p = O.MultiLevelProblem(atm, atom)
    n = p.zero_radiation(1)
    for _ in range(3):
        n, _ = p.mali_sweep(1, n)
    h = m.mg3d_create_ml(atm, atom, n_grids=1, ml_chunk=5)
    try:
        m.mg3d_set_ml_shape(h, 1, 2, 3, 64)
        m.mg3d_mali_sweep(h, 1, 3)
        assert rel(m.mg3d_get_populations(h, 1), n) < 1e-10
    finally:
        m.mg3d_destroy(h)


def test_ml_prd_fp32_formal_solution():
    """FP32 formal solution, FP64 rates.  The line's local operator U sums
    1 - w0 rho chi_t/chi over frequencies whose terms take both signs (rho
    above and below 1) and nearly cancel in a thick line, while the MALI
    populations of a scattering-dominated line follow the small difference
    between U and the Lambda* implicit in Jx: that term stays in FP64
    (1 - rho chi_t/chi from the ratios kernel, U = oc + (1 - oc) sum w u).
    Formed in FP32 it put the populations 1e-4 off after a few sweeps; they
    now stay within a few FP32 ulps, after sweeps and converged."""
    atm, atom = prd_box(1.0)
    p = O.MultiLevelProblem(atm, atom)
    n = p.zero_radiation(1)
    for _ in range(4):
        n, _ = p.mali_sweep(1, n)
    h = m.mg3d_create_ml(atm, atom, n_grids=1, fs_prec=m.MG3D_PREC_F32)
    try:
        m.mg3d_mali_sweep(h, 1, 4)
        assert rel(m.mg3d_get_populations(h, 1), n) < 1e-5
    finally:
        m.mg3d_destroy(h)
    n_c, _ = O.mali_solve(O.MultiLevelProblem(atm, atom), 1e-8)
    h = m.mg3d_create_ml(atm, atom, n_grids=1, fs_prec=m.MG3D_PREC_F32)
    try:
        m.mg3d_mali_solve(h, 1e-6, 500)
        assert rel(m.mg3d_get_populations(h, 1), n_c) < 1e-5
    finally:
        m.mg3d_destroy(h)


def test_ml_prd_batches_refused():
    atm, atom = prd_box(1.0, nx=8, nz=17)
    h = m.mg3d_create_ml(atm, atom, n_grids=1)
    try:
        with pytest.raises(m.MG3DError) as ei:
            m.mg3d_batch_create([h])
        assert ei.value.code == m.MG3D_E_ARG and "partial redistribution" in m.mg3d_last_error()
    finally:
        m.mg3d_destroy(h)


def test_ml_prd_formal_solution_angle_sums():
    """mg3d_formal_solve_ml returns the angle sums the rates use: for a PRD
    frequency Ux = sum_r w (1 - w0 rho chi_t/chi), whose local term the
    library adds in FP64 to the sweep's sum of u.  After two MALI sweeps on
    both sides (the same lagged field), every frequency's Jx and Ux against
    the oracle on its own scale."""
    atm, atom = prd_box(1.0)
    p = O.MultiLevelProblem(atm, atom)
    n = p.zero_radiation(1)
    h = m.mg3d_create_ml(atm, atom, n_grids=1)
    try:
        for _ in range(2):
            m.mg3d_mali_sweep(h, 1, 1)
            n, _ = p.mali_sweep(1, n)
        jx, ux = m.mg3d_formal_solve_ml(h, 1)
    finally:
        m.mg3d_destroy(h)
    Jo, Uo, _ = p.formal_solution(1, n)
    nf = Jo.shape[0]
    for got, ref in ((jx, Jo), (ux, Uo)):
        g2, r2 = got.reshape(nf, -1), ref.reshape(nf, -1)
        err = np.max(np.abs(g2 - r2), axis=1) / np.max(np.abs(r2), axis=1)
        assert float(np.max(err)) < 1e-10
