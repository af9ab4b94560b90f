"""Multi-level chromospheres at their full sizes, against the oracle.

The oracle cannot run a 128x128x257 or 256x256x385 formal solution with 600
frequencies in seconds, but a horizontally homogeneous atmosphere pins the
full-size GPU path all the same: with every plane uniform, the bilinear
upwind interpolation is exact, so the 3D solution is the same in every column
and equals the solution on a 2x2 column with the same stratification, which
the oracle computes in seconds.  The GPU runs in the launch configuration of
the full size (its row bands, rays per block and frequency chunks).
Bars: 1e-10 on FP64 populations, 1e-4 with the FP32 formal solution.
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
