"""GPU parity of the cubic Hermite operators (Sec. 3 and Sec. 4.5) through the
C ABI against the oracle."""

import numpy as np
import pytest

from oracle import mg3d_oracle as O
from paper_1701_01607_gb300 import mg3d as m
from paper_1701_01607_gb300 import synth

pytestmark = pytest.mark.gpu

PARAMS = dict(nu_fmg=16, nu0=0, nu1=2, nu2=2, nu3=32)
HERM = m.MG3D_INTERP_HERMITE
TOL_POP64 = 1e-10


def rel(a, b):
    return float(np.max(np.abs(a - b) / np.abs(b)))


@pytest.fixture(scope="module", autouse=True)
def lib():
    m.load(build_if_missing=True)


# ---------------------------------------------------- prolongation (Sec. 4.5)

def test_hermite_prolongation_matches_oracle():
    """Non-uniform heights, odd and even nodes on every axis, 2- and 3-grid
    transfers, several components; data with large contrasts."""
    atm, atom = synth.stratified_two_level(16, 8, 17, eps=1e-3)
    atm.z = np.cumsum(np.r_[0.0, np.random.default_rng(3).uniform(0.5, 1.5, 16)])
    h = m.mg3d_create(atm, atom, n_grids=3, interpolation=HERM, **PARAMS)
    rng = np.random.default_rng(19)
    try:
        c2 = np.exp(2.0 * rng.normal(size=(3, 9, 4, 8)))
        up = m.mg3d_prolong(h, 3, c2)
        assert rel(up, O.prolong_hermite(c2, atm.z)) < 1e-13
        c1 = rng.normal(size=(2, 5, 2, 4))          # signed data: slopes switch off
        up1 = m.mg3d_prolong(h, 2, c1)
        ref1 = O.prolong_hermite(c1, atm.z[::2])
        assert np.max(np.abs(up1 - ref1)) < 1e-13 * np.max(np.abs(ref1))
    finally:
        m.mg3d_destroy(h)


@pytest.mark.parametrize("n_grids", [2, 3])
def test_hermite_fas_vcycles_fp64(n_grids):
    atm, atom = synth.stratified_two_level(16, 16, 33, eps=1e-3, sigma=0.3, seed=5)
    h = m.mg3d_create(atm, atom, n_grids=n_grids, interpolation=HERM, **PARAMS)
    prob = O.TwoLevelProblem(atm, atom, n_grids=n_grids, interpolation=1)
    n = prob.zero_radiation(n_grids)
    try:
        for cyc in range(3):
            c_gpu = m.mg3d_fas_vcycle(h, cyc == 0)
            n, c_orc = prob.fas_cycle(n, cyc == 0, PARAMS)
            assert abs(c_gpu - c_orc) <= 1e-8 * c_orc
            assert rel(m.mg3d_get_populations(h, n_grids), n) < TOL_POP64
    finally:
        m.mg3d_destroy(h)


def test_hermite_fmg_and_negative_rule_fp64():
    """FMG transfers the full approximation with the Hermite operator; an
    under-smoothed case exercises the 10 % rule on the Hermite correction."""
    atm, atom = synth.stratified_two_level(16, 16, 33, eps=1e-3, sigma=0.3, seed=6)
    h = m.mg3d_create(atm, atom, n_grids=3, interpolation=HERM, **PARAMS)
    try:
        st = m.mg3d_fmg_solve(h, 1e-3, n_grids=3)
        n_fmg = m.mg3d_get_populations(h, 3)
    finally:
        m.mg3d_destroy(h)
    prob = O.TwoLevelProblem(atm, atom, n_grids=3, interpolation=1)
    n_f, cyc = O.fmg_solve(prob, 1e-3, PARAMS)
    assert st["iterations"] == cyc
    assert rel(n_fmg, n_f) < TOL_POP64

    # far from equilibrium (upper level scaled by exp(3 G) node by node), no
    # smoothing: the coarse grid returns negative populations at some nodes
    atm, atom = synth.stratified_two_level(16, 16, 33, eps=1e-3, sigma=0.3, seed=5)
    kw = dict(PARAMS, nu0=0, nu1=0, nu2=0, nu3=8)
    prob = O.TwoLevelProblem(atm, atom, n_grids=2, interpolation=1)
    n0 = prob.zero_radiation(2)
    n0[1] *= np.exp(3.0 * np.random.default_rng(1).normal(size=n0[1].shape))
    n, _ = prob.fas_cycle(n0, False, kw)
    assert prob.negatives > 0
    h = m.mg3d_create(atm, atom, n_grids=2, interpolation=HERM, **kw)
    try:
        m.mg3d_set_populations(h, 2, n0)
        m.mg3d_fas_vcycle(h, False)
        assert rel(m.mg3d_get_populations(h, 2), n) < TOL_POP64
    finally:
        m.mg3d_destroy(h)


def test_hermite_prolongation_multilevel_with_scattering():
    """The 6-level atom with background scattering: FMG prolongs populations
    and the background field with the Hermite operator."""
    atom = synth.hydrogen_like_atom(line_freq=7, cont_freq=4, seed=2)
    atm = synth.chromosphere(16, 16, 33, atom, seed=2, scattering=2.0)
    ml = dict(nu_fmg=8, nu0=4, nu1=2, nu2=2, nu3=16)
    h = m.mg3d_create_ml(atm, atom, n_grids=2, interpolation=HERM, **ml)
    try:
        st = m.mg3d_fmg_solve(h, 1e-6, n_grids=2)
        n_gpu = m.mg3d_get_populations(h, 2)
    finally:
        m.mg3d_destroy(h)
    p = O.MultiLevelProblem(atm, atom, n_grids=2, interpolation=1)
    n_o, cyc = O.fmg_solve(p, 1e-6, ml)
    assert st["iterations"] == cyc
    assert rel(n_gpu, n_o) < TOL_POP64


def test_batch_members_must_agree_on_interpolation():
    atm, atom = synth.stratified_two_level(8, 8, 17, eps=1e-2)
    h1 = m.mg3d_create(atm, atom, n_grids=2, **PARAMS)
    h2 = m.mg3d_create(atm, atom, n_grids=2, interpolation=HERM, **PARAMS)
    try:
        with pytest.raises(m.MG3DError, match="equal"):
            m.mg3d_batch_create([h1, h2])
    finally:
        m.mg3d_destroy(h1)
        m.mg3d_destroy(h2)


# ------------------------------------- Hermite-spline upwind interpolation (Sec. 3)

def _fs_parity(atm, atom, tol, prec=m.MG3D_PREC_F64, config=None, **kw):
    h = m.mg3d_create(atm, atom, n_grids=1, fs_prec=prec, sc_interp=HERM, **PARAMS, **kw)
    try:
        if config is not None:
            m.mg3d_set_fs_config(h, 1, *config, 0)
            assert m.mg3d_get_fs_config(h, 1) == tuple(config) + (0,)
        jeff, u = m.mg3d_formal_solve(h, 1)
    finally:
        m.mg3d_destroy(h)
    prob = O.TwoLevelProblem(atm, atom, sc_interp=1, **kw)
    _, jo, uo = prob.formal_solution(1, prob.zero_radiation(1))
    assert rel(jeff, jo) < tol
    assert rel(u, uo) < tol
    return jeff


@pytest.mark.parametrize("shape", [(16, 16, 33), (12, 8, 17), (2, 2, 9), (1, 1, 3)])
def test_hermite_formal_solution_fp64(shape):
    nx, ny, nz = shape
    atm, atom = synth.stratified_two_level(nx, ny, nz, eps=1e-3, sigma=0.3, seed=11)
    _fs_parity(atm, atom, 1e-12)


@pytest.mark.parametrize("ng,bands,th,lean", [(1, 1, 128, 0), (9, 1, 128, 1), (4, 3, 128, 0),
                                              (2, 6, 64, 2), (3, 8, 128, 0), (5, 6, 32, 1)])
def test_hermite_formal_solution_every_launch_shape(ng, bands, th, lean):
    """Ragged frequency groups and bands; with one or two rows per band the
    four upwind rows span up to three peer blocks."""
    atm, atom = synth.stratified_two_level(16, 16, 17, eps=1e-3, sigma=0.3, seed=2)
    _fs_parity(atm, atom, 1e-12, config=(ng, bands, th, lean))


@pytest.mark.parametrize("ng,lean", [(3, 0), (9, 1)])
def test_hermite_formal_solution_sixteen_block_cluster(ng, lean):
    atm, atom = synth.stratified_two_level(8, 31, 9, eps=1e-3, sigma=0.3, seed=5)
    _fs_parity(atm, atom, 1e-12, config=(ng, 16, 32, lean))


def test_hermite_formal_solution_differs_from_linear_and_fp32():
    """The Hermite result is a different discretisation (not the linear one
    by accident), and the FP32 sweep follows the FP64 oracle."""
    atm, atom = synth.stratified_two_level(16, 16, 33, eps=1e-3, sigma=0.3, seed=11)
    jh = _fs_parity(atm, atom, 1e-12)
    h = m.mg3d_create(atm, atom, n_grids=1, **PARAMS)
    try:
        jl, _ = m.mg3d_formal_solve(h, 1)
    finally:
        m.mg3d_destroy(h)
    assert rel(jh, jl) > 1e-6
    _fs_parity(atm, atom, 1e-5, prec=m.MG3D_PREC_F32)


def test_hermite_mali_fas_and_fmg_fp64():
    """Both Hermite operators together: MALI sweeps, V-cycles and an FMG
    solve follow the oracle iteration by iteration."""
    atm, atom = synth.stratified_two_level(16, 16, 33, eps=1e-3, sigma=0.3, seed=5)
    kw = dict(sc_interp=HERM, interpolation=HERM)
    h = m.mg3d_create(atm, atom, n_grids=3, **kw, **PARAMS)
    prob = O.TwoLevelProblem(atm, atom, n_grids=3, sc_interp=1, interpolation=1)
    try:
        n = prob.zero_radiation(3)
        for _ in range(2):
            c_gpu = m.mg3d_mali_sweep(h, 3, 1)
            n, c_orc = prob.mali_sweep(3, n)
            assert abs(c_gpu - c_orc) <= 1e-8 * c_orc
        assert rel(m.mg3d_get_populations(h, 3), n) < TOL_POP64
        for cyc in range(2):
            c_gpu = m.mg3d_fas_vcycle(h, False)
            n, c_orc = prob.fas_cycle(n, False, PARAMS)
            assert abs(c_gpu - c_orc) <= 1e-8 * c_orc
            assert rel(m.mg3d_get_populations(h, 3), n) < TOL_POP64
        st = m.mg3d_fmg_solve(h, 1e-3, n_grids=3)
        n_fmg = m.mg3d_get_populations(h, 3)
    finally:
        m.mg3d_destroy(h)
    p2 = O.TwoLevelProblem(atm, atom, n_grids=3, sc_interp=1, interpolation=1)
    n_f, cyc = O.fmg_solve(p2, 1e-3, PARAMS)
    assert st["iterations"] == cyc
    assert rel(n_fmg, n_f) < TOL_POP64


def test_hermite_autotune_keeps_parity_and_refuses_staging():
    atm, atom = synth.stratified_two_level(16, 16, 33, eps=1e-3, sigma=0.3, seed=11)
    h = m.mg3d_create(atm, atom, n_grids=1, sc_interp=HERM, **PARAMS)
    try:
        with pytest.raises(m.MG3DError, match="unstaged"):
            m.mg3d_set_fs_config(h, 1, 3, 2, 128, 0, 1)
        m.mg3d_autotune(h)
        assert m.mg3d_get_fs_config(h, 1)[4] == 0
        jeff, u = m.mg3d_formal_solve(h, 1)
    finally:
        m.mg3d_destroy(h)
    prob = O.TwoLevelProblem(atm, atom, sc_interp=1)
    _, jo, uo = prob.formal_solution(1, prob.zero_radiation(1))
    assert rel(jeff, jo) < 1e-12 and rel(u, uo) < 1e-12


# ------------------------------------------------- multi-level atom, Hermite sweep

def _ml_box(nx=8, ny=8, nz=17, seed=2, scattering=0.0):
    atom = synth.hydrogen_like_atom(line_freq=7, cont_freq=4, seed=seed)
    atm = synth.chromosphere(nx, ny, nz, atom, seed=seed, scattering=scattering)
    return atm, atom


def _per_freq_err(got, ref):
    nf = ref.shape[0]
    err = np.max(np.abs(got.reshape(nf, -1) - ref), axis=1) / np.max(np.abs(ref), axis=1)
    return float(np.max(err))


@pytest.mark.parametrize("shape,rpb,bands", [((8, 8, 17), 12, 1), ((8, 8, 17), 3, 4),
                                             ((12, 8, 9), 6, 8), ((2, 2, 5), 12, 2)])
def test_hermite_ml_formal_solution_and_sweeps_fp64(shape, rpb, bands):
    """Per-frequency angle sums, then two MALI sweeps in chunks that split
    transitions, with ray groups and bands of one or two rows."""
    atm, atom = _ml_box(*shape)
    p = O.MultiLevelProblem(atm, atom, sc_interp=1)
    n0 = p.zero_radiation(1)
    Jo, Uo, _ = p.formal_solution(1, n0)
    n1, _ = p.mali_sweep(1, n0)
    n2, _ = p.mali_sweep(1, n1)
    h = m.mg3d_create_ml(atm, atom, n_grids=1, sc_interp=HERM)
    try:
        m.mg3d_set_ml_shape(h, 1, bands, rpb, 64)
        jx, ux = m.mg3d_formal_solve_ml(h, 1)
        assert _per_freq_err(jx, Jo) < 1e-11 and _per_freq_err(ux, Uo) < 1e-11
        m.mg3d_set_ml_chunk(h, 11)
        m.mg3d_mali_sweep(h, 1, 2)
        assert rel(m.mg3d_get_populations(h, 1), n2) < TOL_POP64
    finally:
        m.mg3d_destroy(h)


def test_hermite_ml_fas_with_scattering_and_fp32():
    """Both Hermite operators with background scattering through 2-grid
    V-cycles (FP64); the FP32 sweep's angle sums follow the oracle."""
    atm, atom = _ml_box(16, 16, 33, scattering=2.0)
    kw = dict(sc_interp=HERM, interpolation=HERM)
    ml = dict(nu_fmg=8, nu0=4, nu1=2, nu2=2, nu3=16)
    h = m.mg3d_create_ml(atm, atom, n_grids=2, **kw, **ml)
    p = O.MultiLevelProblem(atm, atom, n_grids=2, sc_interp=1, interpolation=1)
    n = p.zero_radiation(2)
    try:
        for cyc in range(2):
            c_gpu = m.mg3d_fas_vcycle(h, cyc == 0)
            n, c_orc = p.fas_cycle(n, cyc == 0, ml)
            assert abs(c_gpu - c_orc) <= 1e-6 * c_orc
            assert rel(m.mg3d_get_populations(h, 2), n) < TOL_POP64
    finally:
        m.mg3d_destroy(h)
    atm, atom = _ml_box()
    h = m.mg3d_create_ml(atm, atom, n_grids=1, fs_prec=m.MG3D_PREC_F32, sc_interp=HERM)
    try:
        jx, ux = m.mg3d_formal_solve_ml(h, 1)
        m.mg3d_autotune(h)
        jx2, _ = m.mg3d_formal_solve_ml(h, 1)
    finally:
        m.mg3d_destroy(h)
    p = O.MultiLevelProblem(atm, atom, sc_interp=1)
    Jo, Uo, _ = p.formal_solution(1, p.zero_radiation(1))
    assert _per_freq_err(jx, Jo) < 1e-5 and _per_freq_err(ux, Uo) < 1e-5
    assert _per_freq_err(jx2, Jo) < 1e-5
