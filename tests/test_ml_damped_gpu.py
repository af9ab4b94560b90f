"""Damped (Voigt) lines of the multi-level atom on the GPU against the oracle.

A line carries a damping parameter a at t_ref; the damping width does not
scale with temperature while the Doppler width d = sqrt(T/t_ref) does, so a
node's profile is H(a/d, x/d)/(sqrt(pi) d) (the oracle takes H from scipy's
Faddeeva function, the library from its rational Voigt function, whose
relative error is below 5e-14 + 2e-14/(a/d)).  Bars: per-frequency angle sums
to 1e-11 on each frequency's scale, populations to 1e-10 after FP64 sweeps or
cycles, 1e-5 with the FP32 formal solution; refused in a flow, with partial
redistribution in the atom, and in batches.
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


def per_frequency_error(got, ref):
    nf = ref.shape[0]
    g2, r2 = got.reshape(nf, -1), ref.reshape(nf, -1)
    return float(np.max(np.max(np.abs(g2 - r2), axis=1) / np.max(np.abs(r2), axis=1)))


@pytest.fixture(scope="module", autouse=True)
def lib():
    m.load(build_if_missing=True)


def damped_box(a=0.03, nx=8, nz=17, line_freq=9, **kw):
    atom = synth.hydrogen_like_atom(line_freq=line_freq, cont_freq=4, seed=2, a_damp=a)
    atm = synth.chromosphere(nx, nx, nz, atom, seed=2, **kw)
    return atm, atom


@pytest.mark.parametrize("a", [0.01, 0.3])
def test_damped_formal_solution_and_sweeps_fp64(a):
    atm, atom = damped_box(a, ground_collisions=1e-3)
    p = O.MultiLevelProblem(atm, atom)
    n = p.zero_radiation(1)
    Jo, Uo, _ = p.formal_solution(1, n)
    h = m.mg3d_create_ml(atm, atom, n_grids=1)
    try:
        assert rel(m.mg3d_get_populations(h, 1), n) < 1e-11
        jx, ux = m.mg3d_formal_solve_ml(h, 1)
        assert per_frequency_error(jx, Jo) < 1e-11
        assert per_frequency_error(ux, Uo) < 1e-11
        for _ in range(4):
            m.mg3d_mali_sweep(h, 1, 1)
            n, _ = p.mali_sweep(1, n)
        assert rel(m.mg3d_get_populations(h, 1), n) < 1e-10
    finally:
        m.mg3d_destroy(h)
    # the damping changed the solution: the Doppler atom's populations differ
    atm_d, atom_d = damped_box(0.0, ground_collisions=1e-3)
    pd = O.MultiLevelProblem(atm_d, atom_d)
    nd = pd.zero_radiation(1)
    for _ in range(4):
        nd, _ = pd.mali_sweep(1, nd)
    assert rel(n, nd) > 1e-6


def test_damped_vcycles_fmg_and_hermite_upwind():
    """2-grid V-cycles and FMG in FP64 against the oracle (the coarse grids'
    profiles at their own temperatures), and MALI sweeps with the Hermite
    upwind interpolation, which reads the same opacity."""
    atm, atom = damped_box(0.05)
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
    n_f, cycles = O.fmg_solve(O.MultiLevelProblem(atm, atom, n_grids=2), 1e-3, PARAMS)
    h = m.mg3d_create_ml(atm, atom, n_grids=2, **PARAMS)
    try:
        st = m.mg3d_fmg_solve(h, 1e-3, 40, n_grids=2)
        assert st["iterations"] == cycles
        assert rel(m.mg3d_get_populations(h, 2), n_f) < 1e-10
    finally:
        m.mg3d_destroy(h)
    q = O.MultiLevelProblem(atm, atom, sc_interp=1)
    nq = q.zero_radiation(1)
    h = m.mg3d_create_ml(atm, atom, n_grids=1, sc_interp=m.MG3D_INTERP_HERMITE)
    try:
        for _ in range(3):
            m.mg3d_mali_sweep(h, 1, 1)
            nq, _ = q.mali_sweep(1, nq)
        assert rel(m.mg3d_get_populations(h, 1), nq) < 1e-10
    finally:
        m.mg3d_destroy(h)


def test_damped_fp32_autotuned_and_chunked():
    """FP32 formal solution (the Voigt profile evaluated in FP64 and rounded
    once) after autotuning, with chunks that split the damped lines: four
    sweeps within 1e-5 of the oracle."""
    atm, atom = damped_box(0.03, nx=16, ground_collisions=1e-3)
    p = O.MultiLevelProblem(atm, atom)
    n = p.zero_radiation(1)
    for _ in range(4):
        n, _ = p.mali_sweep(1, n)
    h = m.mg3d_create_ml(atm, atom, n_grids=1, fs_prec=m.MG3D_PREC_F32, ml_chunk=7)
    try:
        m.mg3d_autotune(h)
        m.mg3d_mali_sweep(h, 1, 4)
        assert rel(m.mg3d_get_populations(h, 1), n) < 1e-5
    finally:
        m.mg3d_destroy(h)


def test_damped_batches_refused():
    atm, atom = damped_box(0.03)
    h = m.mg3d_create_ml(atm, atom, n_grids=1)
    try:
        with pytest.raises(m.MG3DError) as ei:
            m.mg3d_batch_create([h])
        assert ei.value.code == m.MG3D_E_ARG and "damped" in m.mg3d_last_error()
    finally:
        m.mg3d_destroy(h)
