"""Multi-level chromospheres at their full sizes, against the oracle.

The oracle cannot run a 128x128x257 or 256x256x385 formal solution with 600
frequencies in seconds.  Two kinds of case pin the full-size GPU path:

* a horizontally homogeneous atmosphere at the full size: with every plane
  uniform the bilinear upwind interpolation is exact, so the 3D solution is
  the same in every column and equals the solution on a 2x2 column with the
  same stratification, which the oracle computes in seconds.  This runs the
  full size's planes, frequency chunks and launch configuration, but cannot
  see a wrong upwind row, ray-group slot or wrap;
* the full width with horizontal structure: 3D-perturbed chromospheres with
  128- and 256-wide planes, few planes and few frequencies, swept in the
  launch shapes the full sizes take (their row bands, rays per block and
  block sizes), compared with the oracle element by element.  A wrong peer
  band, slot or wrap changes these results.

Bars: per-frequency angle sums 1e-11 (FP64) and 2e-4 (FP32), populations
1e-10 (FP64) and 1e-4 (FP32 formal solution).
"""

import numpy as np
import pytest

from oracle import mg3d_oracle as O
from paper_1701_01607_gb300 import mg3d as m
from paper_1701_01607_gb300 import synth

pytestmark = [pytest.mark.gpu, pytest.mark.slow]

SWEEPS = 2


@pytest.fixture(scope="module", autouse=True)
def lib():
    m.load(build_if_missing=True)


@pytest.fixture(scope="module")
def atom():
    return synth.hydrogen_like_atom(line_freq=100, cont_freq=20, seed=2)


def oracle_column(atom, nz):
    col = synth.chromosphere(2, 2, nz, atom, seed=2, sigma_t=0.0)
    p = O.MultiLevelProblem(col, atom)
    n = p.zero_radiation(1)
    for _ in range(SWEEPS):
        n, _ = p.mali_sweep(1, n)
    return n[:, :, :1, :1]          # every column is the same


def run_full(atom, nx, nz, n_grids, prec):
    atm = synth.chromosphere(nx, nx, nz, atom, seed=2, sigma_t=0.0)
    h = m.mg3d_create_ml(atm, atom, n_grids=n_grids, fs_prec=prec)
    try:
        shape = m.mg3d_get_ml_shape(h, n_grids)
        chunk = m.mg3d_get_ml_chunk(h)
        m.mg3d_mali_sweep(h, n_grids, SWEEPS)
        n = m.mg3d_get_populations(h, n_grids)
    finally:
        m.mg3d_destroy(h)
    return atm, n, shape, chunk


def check(atm, n, ref, tol):
    assert np.all(np.isfinite(n)) and n.min() > 0
    # particle conservation holds in the FP64 rate solve whatever the
    # formal-solution precision
    assert np.max(np.abs(n.sum(axis=0) / atm.n_tot - 1.0)) < 1e-13
    err = float(np.max(np.abs(n - ref) / np.abs(ref)))
    assert err < tol, err


def test_chromosphere_128x128x257_fp64(atom):
    ref = oracle_column(atom, 257)
    atm, n, shape, chunk = run_full(atom, 128, 257, 3, m.MG3D_PREC_F64)
    # the full size needs its own launch configuration: fewer than 12 rays
    # per block (a 128-wide plane of 12 FP64 intensity planes does not fit)
    assert shape[1] < 12
    check(atm, n, ref, 1e-10)


def test_chromosphere_128x128x257_fp32(atom):
    ref = oracle_column(atom, 257)
    atm, n, _, _ = run_full(atom, 128, 257, 3, m.MG3D_PREC_F32)
    check(atm, n, ref, 1e-4)


def test_chromosphere_256x256x385_fp32_four_grids(atom):
    ref = oracle_column(atom, 385)
    atm, n, shape, chunk = run_full(atom, 256, 385, 4, m.MG3D_PREC_F32)
    assert shape[1] < 12
    check(atm, n, ref, 1e-4)


def test_chromosphere_64x64x129_mixed_precision_converged(atom):
    """The mixed-precision bar on the 6-level atom at 600 frequencies: FAS
    solves to C < 1e-3 with the FP32 formal solution (FP64 rates) and with
    FP64 throughout take the same number of V-cycles and give populations
    within 1e-4 of each other; the FP64 path itself follows the oracle to
    1e-10 in the parity tests."""
    atm = synth.chromosphere(64, 64, 129, atom, seed=7)
    params = dict(n_grids=3, nu_fmg=16, nu0=20, nu1=4, nu2=8, nu3=32)
    res = {}
    for prec in (m.MG3D_PREC_F64, m.MG3D_PREC_F32):
        h = m.mg3d_create_ml(atm, atom, fs_prec=prec, **params)
        try:
            st = m.mg3d_fas_solve(h, 1e-3, 40, n_grids=3)
            res[prec] = (st["iterations"], m.mg3d_get_populations(h, 3))
        finally:
            m.mg3d_destroy(h)
    (c64, n64), (c32, n32) = res[m.MG3D_PREC_F64], res[m.MG3D_PREC_F32]
    assert c32 == c64
    assert np.all(n32 > 0)
    assert float(np.max(np.abs(n32 - n64) / n64)) < 1e-4


# ------------------------ the 64x64x129 bench box with a flow and with PRD

def _two_level_sweeps(atm, atom, sweeps=2):
    h = m.mg3d_create(atm, atom, n_grids=1, nu_fmg=16, nu0=0, nu1=2, nu2=2, nu3=32)
    try:
        m.mg3d_autotune(h)
        m.mg3d_mali_sweep(h, 1, sweeps)
        n_gpu = m.mg3d_get_populations(h, 1)
    finally:
        m.mg3d_destroy(h)
    p = O.TwoLevelProblem(atm, atom)
    n = p.zero_radiation(1)
    for _ in range(sweeps):
        n, _ = p.mali_sweep(1, n)
    return float(np.max(np.abs(n_gpu - n) / np.abs(n)))


def test_bench_box_moving_fp64():
    """The 64x64x129 workload (eps = 1e-4, sigma = 0.3) with a flow of rms 1
    Doppler width and autotuned shapes: two MALI sweeps against the oracle."""
    atom = synth.TwoLevelAtom(n_freq=9)
    atm, atom = synth.stratified_two_level(64, 64, 129, eps=1e-4, sigma=0.3, seed=1, atom=atom,
                                           velocity=1.0)
    assert _two_level_sweeps(atm, atom) < 1e-10


def test_bench_box_prd_fp64():
    """The same box with full coherence (gamma = 1): the second sweep uses the
    mean intensity of the first."""
    atom = synth.TwoLevelAtom(n_freq=9, gamma_prd=1.0)
    atm, atom = synth.stratified_two_level(64, 64, 129, eps=1e-4, sigma=0.3, seed=1, atom=atom)
    assert _two_level_sweeps(atm, atom) < 1e-10


# ------------------- full width with horizontal structure, full-size shapes

# Launch shapes (bands, rays per block, threads) of the full sizes: the
# library's defaults at 128x128x257 and 256x256x385 (600 frequencies), and the
# FP32 shape the autotuner takes at 128x128x257.
FULL_WIDTH_SHAPES = [
    (128, m.MG3D_PREC_F64, (8, 6, 256)),
    (128, m.MG3D_PREC_F32, (8, 12, 256)),
    (128, m.MG3D_PREC_F32, (8, 3, 512)),
    (256, m.MG3D_PREC_F64, (6, 1, 256)),
    (256, m.MG3D_PREC_F32, (8, 3, 256)),
]

_FS = {}


def structured(nx, nz):
    """A 3D-perturbed chromosphere (temperature perturbations 10 %) with 15
    frequencies (5 lines x 2, 5 continua x 1)."""
    atom = synth.hydrogen_like_atom(line_freq=2, cont_freq=1, seed=2)
    return synth.chromosphere(nx, nx, nz, atom, seed=5), atom


def per_frequency_error(got, ref):
    nf = ref.shape[0]
    err = np.max(np.abs(got.reshape(nf, -1) - ref), axis=1) / np.max(np.abs(ref), axis=1)
    return float(err.max())


@pytest.mark.parametrize("nx,prec,shape", FULL_WIDTH_SHAPES)
def test_full_width_structured_formal_solution(nx, prec, shape):
    nz = 9 if nx == 128 else 5
    atm, atom = structured(nx, nz)
    if nx not in _FS:
        p = O.MultiLevelProblem(atm, atom)
        Jo, Uo, _ = p.formal_solution(1, p.zero_radiation(1))
        _FS[nx] = (Jo, Uo)
    Jo, Uo = _FS[nx]
    h = m.mg3d_create_ml(atm, atom, n_grids=1, fs_prec=prec)
    try:
        m.mg3d_set_ml_shape(h, 1, *shape)
        assert m.mg3d_get_ml_shape(h, 1) == shape
        jx, ux = m.mg3d_formal_solve_ml(h, 1)
    finally:
        m.mg3d_destroy(h)
    tol = 1e-11 if prec == m.MG3D_PREC_F64 else 2e-4
    assert per_frequency_error(jx, Jo) < tol
    assert per_frequency_error(ux, Uo) < tol


def test_full_width_structured_fas_vcycle_fp64():
    """A 3-grid FAS V-cycle on 128x128x9 with the finest grid in the
    128x128x257 FP64 launch shape, and the two coarser grids in theirs:
    populations after the cycle against the oracle's cycle to 1e-10."""
    atm, atom = structured(128, 9)
    params = dict(nu_fmg=4, nu0=1, nu1=1, nu2=1, nu3=4)
    p = O.MultiLevelProblem(atm, atom, n_grids=3)
    n_o, _ = p.fas_cycle(p.zero_radiation(3), True, params)
    h = m.mg3d_create_ml(atm, atom, n_grids=3, fs_prec=m.MG3D_PREC_F64, **params)
    try:
        for level, shape in ((3, (8, 6, 256)), (2, (4, 12, 256)), (1, (2, 12, 256))):
            m.mg3d_set_ml_shape(h, level, *shape)
        m.mg3d_fas_vcycle(h, True)
        n = m.mg3d_get_populations(h, 3)
    finally:
        m.mg3d_destroy(h)
    assert float(np.max(np.abs(n - n_o) / np.abs(n_o))) < 1e-10


# ---------------- mixed precision against the FP64 oracle: FAS and FMG solves

TWO_LEVEL_PARAMS = dict(nu_fmg=16, nu0=0, nu1=2, nu2=2, nu3=32)


@pytest.mark.parametrize("method", ["fas", "fmg"])
def test_two_level_fp32_solve_against_fp64_oracle(method):
    """The mixed-precision bar on converged populations: a two-grid FAS (or FMG) solve to
    C < 1e-3 with the FP32 formal solution and FP64 rates matches the FP64
    oracle's solve of the same schedule to 1e-4 relative on the populations,
    with the same number of V-cycles (16x16x33 box, eps = 1e-4, log-normal
    sigma = 0.3; the oracle's solves take seconds at this size)."""
    atm, atom = synth.stratified_two_level(16, 16, 33, eps=1e-4, sigma=0.3, seed=3)
    prob = O.TwoLevelProblem(atm, atom, n_grids=2)
    solve_o = O.fas_solve if method == "fas" else O.fmg_solve
    n_o, cycles_o = solve_o(prob, 1e-3, TWO_LEVEL_PARAMS)
    h = m.mg3d_create(atm, atom, n_grids=2, fs_prec=m.MG3D_PREC_F32, **TWO_LEVEL_PARAMS)
    try:
        solve = m.mg3d_fas_solve if method == "fas" else m.mg3d_fmg_solve
        st = solve(h, 1e-3, 100, n_grids=2)
        n = m.mg3d_get_populations(h, 2)
    finally:
        m.mg3d_destroy(h)
    assert st["iterations"] == cycles_o
    assert float(np.max(np.abs(n - n_o) / np.abs(n_o))) < 1e-4


def test_config4_fmg_stages_fp32_against_fp64():
    """Config 4 in small: full multigrid with 4 grids and (16, 20, 4, 8, 32) on
    a stretched-height chromosphere (spacing 13/24 to 60/24 of dx, seed 3) with
    30 frequencies.  After every FMG stage the FP32 formal solution's
    approximation on that grid stays within 1e-4 of FP64's, and so do the
    populations after the V-cycles to C < 1e-3, with the same cycle count."""
    atom = synth.hydrogen_like_atom(line_freq=4, cont_freq=2, seed=2)
    z = synth.stretched_heights(49, 13.0 / 24.0, 60.0 / 24.0)
    atm = synth.chromosphere(32, 32, 49, atom, seed=3, z=z, dx=1.0)
    params = dict(nu_fmg=16, nu0=20, nu1=4, nu2=8, nu3=32)
    res = {}
    for prec in (m.MG3D_PREC_F64, m.MG3D_PREC_F32):
        h = m.mg3d_create_ml(atm, atom, n_grids=4, fs_prec=prec, **params)
        try:
            pops = []
            for k in range(1, 5):
                m.mg3d_fmg_stage(h, k)
                pops.append(m.mg3d_get_populations(h, k))
            cycles = 0
            while cycles < 20:
                c = m.mg3d_fas_vcycle(h, cycles == 0)
                cycles += 1
                if c < 1e-3:
                    break
            res[prec] = (pops, cycles, m.mg3d_get_populations(h, 4))
        finally:
            m.mg3d_destroy(h)
    (p64, c64, n64), (p32, c32, n32) = res[m.MG3D_PREC_F64], res[m.MG3D_PREC_F32]
    for k in range(4):
        assert float(np.max(np.abs(p32[k] - p64[k]) / p64[k])) < 1e-4, k + 1
    assert c32 == c64
    assert float(np.max(np.abs(n32 - n64) / n64)) < 1e-4
