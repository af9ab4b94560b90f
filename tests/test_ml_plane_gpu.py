"""Parity of the multi-level shifted-plane sweep (kind 1 of
mg3d_set_ml_shape_ex) with the multi-level FP64 oracle, through the C ABI.

Each ray's finished plane is stored shifted by the offset of the step that
reads it, with the opacity and source function of the block's frequencies as
channels beside the intensity (Sec. 3, periodic boundaries of Sec. 4.2).  The
cases cover what the layout can get wrong: ragged bands and clusters of up to
16 blocks, one-band planes (the halo is the block's own first row), groups of
1, 2 and 4 frequencies with a partial last group (chunks that split them),
every rays-per-block count, several passes of a block over its band, the
lagged mean intensity of background scattering and partial redistribution,
and both precisions.  Bars: per-frequency angle sums to 1e-11 (FP64) and
2e-4 (FP32) on each frequency's scale, populations to 1e-10 after FP64
sweeps or cycles and 1e-5 with the FP32 formal solution.
"""

import numpy as np
import pytest

from oracle import mg3d_oracle as O
from paper_1701_01607_gb300 import mg3d as m
from paper_1701_01607_gb300 import synth

pytestmark = pytest.mark.gpu

TOL_FS_ML = 1e-11
PARAMS = dict(nu_fmg=8, nu0=10, nu1=2, nu2=4, nu3=16)


def rel(a, b):
    return float(np.max(np.abs(a - b) / np.abs(b)))


def per_frequency_error(got, ref):
    nf = ref.shape[0]
    err = np.max(np.abs(got.reshape(nf, -1) - ref.reshape(nf, -1)), axis=1) / \
        np.max(np.abs(ref.reshape(nf, -1)), axis=1)
    return float(np.max(err))


@pytest.fixture(scope="module", autouse=True)
def lib():
    m.load(build_if_missing=True)


def small(nx=8, ny=8, nz=17, seed=2, line_freq=7, cont_freq=4, **kw):
    atom = synth.hydrogen_like_atom(line_freq=line_freq, cont_freq=cont_freq, seed=seed,
                                    gamma_prd=kw.pop("gamma_prd", 0.0))
    atm = synth.chromosphere(nx, ny, nz, atom, seed=seed, **kw)
    return atm, atom


_ORACLE = {}


def oracle_fs(key, atm, atom):
    if key not in _ORACLE:
        p = O.MultiLevelProblem(atm, atom)
        Jo, Uo, _ = p.formal_solution(1, p.zero_radiation(1))
        _ORACLE[key] = (Jo, Uo)
    return _ORACLE[key]


# (bands, rays per block, threads, frequencies per block) on a 12 x 16 plane:
# 16 rows as 16, 8+8, 6+6+4, 3x5+1, 2x8, 1x16
SHAPES = [(1, 6, 256, 1), (2, 6, 128, 2), (3, 4, 64, 4), (6, 3, 32, 1), (8, 2, 64, 2),
          (16, 1, 32, 4), (3, 12, 128, 2), (1, 1, 512, 4), (6, 6, 32, 2)]


@pytest.mark.parametrize("bands,rpb,threads,nf", SHAPES)
def test_plane_shapes_fp64_and_fp32(bands, rpb, threads, nf):
    atm, atom = small(12, 16, 17)
    Jo, Uo = oracle_fs("12x16x17", atm, atom)
    for prec, tol in ((m.MG3D_PREC_F64, TOL_FS_ML), (m.MG3D_PREC_F32, 2e-4)):
        if prec == m.MG3D_PREC_F64 and nf > 1:
            continue   # one frequency per block in FP64
        h = m.mg3d_create_ml(atm, atom, n_grids=1, fs_prec=prec)
        try:
            m.mg3d_set_ml_shape_ex(h, 1, bands, rpb, threads, 1, nf)
            assert m.mg3d_get_ml_shape_ex(h, 1) == (bands, rpb, threads, 1, nf)
            jx, ux = m.mg3d_formal_solve_ml(h, 1)
        finally:
            m.mg3d_destroy(h)
        assert per_frequency_error(jx, Jo) < tol, prec
        assert per_frequency_error(ux, Uo) < tol, prec


def test_plane_mali_sweeps_and_chunks():
    """Five FP64 MALI sweeps with chunks of 5 frequencies (groups of 1 split
    nothing; of 2 and 4 the last group of a chunk is partial) against the
    oracle, and the FP32 sweeps with 4 frequencies per block."""
    atm, atom = small()
    p = O.MultiLevelProblem(atm, atom)
    n = p.zero_radiation(1)
    for _ in range(5):
        n, _ = p.mali_sweep(1, n)
    for prec, nf, tol in ((m.MG3D_PREC_F64, 1, 1e-10), (m.MG3D_PREC_F32, 4, 1e-5),
                          (m.MG3D_PREC_F32, 2, 1e-5)):
        h = m.mg3d_create_ml(atm, atom, n_grids=1, fs_prec=prec, ml_chunk=5)
        try:
            m.mg3d_set_ml_shape_ex(h, 1, 2, 3, 128, 1, nf)
            m.mg3d_mali_sweep(h, 1, 5)
            assert rel(m.mg3d_get_populations(h, 1), n) < tol, (prec, nf)
        finally:
            m.mg3d_destroy(h)


def test_plane_vcycles_with_scattering_and_prd():
    """The lagged mean intensity (background scattering and partial
    redistribution read it) comes from the plane sweep's per-ray-group sums:
    2-grid V-cycles on both grids with kind 1 against the oracle."""
    for kw in (dict(scattering=2.0), dict(gamma_prd=1.0, ground_collisions=1e-3)):
        atm, atom = small(8, 8, 17, **kw)
        p = O.MultiLevelProblem(atm, atom, n_grids=2)
        n = p.zero_radiation(2)
        h = m.mg3d_create_ml(atm, atom, n_grids=2, **PARAMS)
        try:
            m.mg3d_set_ml_shape_ex(h, 1, 1, 3, 64, 1, 1)
            m.mg3d_set_ml_shape_ex(h, 2, 2, 6, 64, 1, 1)
            for cyc in range(2):
                m.mg3d_fas_vcycle(h, cyc == 0)
                n, _ = p.fas_cycle(n, cyc == 0, PARAMS)
                assert rel(m.mg3d_get_populations(h, 2), n) < 1e-10, (kw, cyc)
        finally:
            m.mg3d_destroy(h)


def test_plane_autotuned_fp32_converges_with_oracle():
    """The autotuner times both kinds; whatever it keeps, FP32 MALI to
    C < 1e-6 on a scattering-dominated chromosphere stays within 1e-5 of the
    converged oracle."""
    atm, atom = small(16, 16, 17, ground_collisions=1e-3)
    n_c, _ = O.mali_solve(O.MultiLevelProblem(atm, atom), 1e-8)
    h = m.mg3d_create_ml(atm, atom, n_grids=1, fs_prec=m.MG3D_PREC_F32)
    try:
        info = m.mg3d_autotune(h)
        assert info["evaluated"] > 20
        bands, rpb, threads, kind, nf = m.mg3d_get_ml_shape_ex(h, 1)
        assert kind in (0, 1) and 12 % rpb == 0 and 1 <= bands <= 16
        m.mg3d_mali_solve(h, 1e-6, 500)
        assert rel(m.mg3d_get_populations(h, 1), n_c) < 1e-5
    finally:
        m.mg3d_destroy(h)


def test_plane_kind_refused_where_it_does_not_apply():
    atm, atom = small()
    h = m.mg3d_create_ml(atm, atom, n_grids=1, fs_prec=m.MG3D_PREC_F64)
    try:
        for bad in [(2, 3, 64, 1, 2),      # FP64: one frequency per block
                    (2, 3, 64, 1, 3),      # 3 frequencies per block: not built
                    (2, 5, 64, 1, 1),      # 5 does not divide 12
                    (2, 3, 64, 2, 1)]:     # no kind 2
            with pytest.raises(m.MG3DError):
                m.mg3d_set_ml_shape_ex(h, 1, *bad)
    finally:
        m.mg3d_destroy(h)
    atm, atom = small(16, 16, 17)
    h = m.mg3d_create_ml(atm, atom, n_grids=1, fs_prec=m.MG3D_PREC_F32)
    try:
        with pytest.raises(m.MG3DError) as ei:
            m.mg3d_set_ml_shape_ex(h, 1, 1, 3, 32, 1, 4)   # 256 nodes, 32 threads x 2 passes
        assert "too few threads" in m.mg3d_last_error()
    finally:
        m.mg3d_destroy(h)
    atm, atom = small(velocity=0.5)
    h = m.mg3d_create_ml(atm, atom, n_grids=1)
    try:
        with pytest.raises(m.MG3DError):
            m.mg3d_set_ml_shape_ex(h, 1, 2, 3, 64, 1, 1)
        assert "static" in m.mg3d_last_error()
    finally:
        m.mg3d_destroy(h)
