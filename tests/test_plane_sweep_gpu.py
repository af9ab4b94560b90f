"""Parity of the shifted-plane sweep (stage 2 of mg3d_set_fs_config) with the
FP64 CPU oracle, through the C ABI.

The kernel stores each finished plane shifted by the next step's upwind
offset, so that every node reads its four corners at fixed offsets; writes
go to the block owning the shifted row (distributed shared memory), with
copies into a halo row and a pad column.  The cases below exercise that
layout where it can go wrong: ragged bands (the last band shorter), clusters
of up to 16 blocks, a single band (the halo is the block's own first row),
planes one node wide or one row high, frequency groups (several clusters per
ray, the last group with a single-frequency slot), several passes of a block
over its band, and both register budgets of the FP32 kernel.

FP64 formal solutions agree with the oracle to 1e-12 relative (rounding
order, fused multiply-adds and the last bits of exp and 1/x differ); FP32 to
2e-5 relative on Jeff and U (its exp and 1/x are the hardware approximations,
within a few ulp, compounded over the planes of a sweep).
"""

import numpy as np
import pytest

from oracle import mg3d_oracle as O
from paper_1701_01607_gb300 import mg3d as m
from paper_1701_01607_gb300 import synth

pytestmark = pytest.mark.gpu

TOL_FS64 = 1e-12
TOL_FS32 = 2e-5
PLANE = 2   # stage value that selects the shifted-plane sweep


def rel(a, b):
    return float(np.max(np.abs(a - b) / np.abs(b)))


@pytest.fixture(scope="module", autouse=True)
def lib():
    m.load(build_if_missing=True)


_ORACLE = {}


def oracle_fs(atm, atom, key, quad_a=None):
    """Jeff and U of the oracle's formal solution from the zero-radiation
    populations (cached per case); quad_a None is the oracle's default A4 set."""
    if key not in _ORACLE:
        prob = O.TwoLevelProblem(atm, atom, quad_a=quad_a)
        _, jo, uo = prob.formal_solution(1, prob.zero_radiation(1))
        _ORACLE[key] = (jo, uo)
    return _ORACLE[key]


def gpu_fs(atm, atom, prec=m.MG3D_PREC_F64, shape=None, quad_a=0.0):
    h = m.mg3d_create(atm, atom, quad_a=quad_a, n_grids=1, fs_prec=prec)
    try:
        if shape is not None:
            m.mg3d_set_fs_config(h, 1, *shape)
        cfg = m.mg3d_get_fs_config(h, 1)
        jeff, u = m.mg3d_formal_solve(h, 1)
    finally:
        m.mg3d_destroy(h)
    return jeff, u, cfg


@pytest.mark.parametrize("shape", [(16, 16, 33), (12, 8, 17), (2, 2, 9), (1, 1, 3), (64, 64, 17)])
def test_default_shape_is_the_plane_sweep(shape):
    nx, ny, nz = shape
    atm, atom = synth.stratified_two_level(nx, ny, nz, eps=1e-3, sigma=0.3, seed=11)
    jeff, u, cfg = gpu_fs(atm, atom)
    assert cfg[4] == PLANE, cfg
    jo, uo = oracle_fs(atm, atom, ("default",) + shape)
    assert rel(jeff, jo) < TOL_FS64
    assert rel(u, uo) < TOL_FS64


# 16 rows as 1, 2, 3 (6+6+4), 4, 6 (3x5+1), 8 and 16 bands
SHAPES64 = [
    (9, 1, 128, 0), (9, 3, 64, 0), (9, 6, 32, 0), (9, 8, 96, 0), (9, 16, 32, 0),
    (2, 3, 128, 0), (4, 6, 64, 0), (6, 2, 256, 0), (9, 2, 512, 0), (9, 4, 32, 0),
]


@pytest.mark.parametrize("fpb,bands,threads,lean", SHAPES64)
def test_every_plane_shape_fp64(fpb, bands, threads, lean):
    atm, atom = synth.stratified_two_level(16, 16, 17, eps=1e-3, sigma=0.3, seed=2)
    jeff, u, cfg = gpu_fs(atm, atom, shape=(fpb, bands, threads, lean, PLANE))
    assert cfg == (fpb, bands, threads, lean, PLANE)
    jo, uo = oracle_fs(atm, atom, "16x16x17")
    assert rel(jeff, jo) < TOL_FS64
    assert rel(u, uo) < TOL_FS64


SHAPES32 = [
    (9, 1, 256, 0), (9, 3, 64, 1), (9, 6, 32, 1), (9, 8, 64, 0), (9, 16, 32, 1),
    (2, 4, 128, 1), (4, 6, 64, 0), (6, 2, 512, 1), (9, 2, 160, 1),
]


@pytest.mark.parametrize("fpb,bands,threads,lean", SHAPES32)
def test_every_plane_shape_fp32(fpb, bands, threads, lean):
    atm, atom = synth.stratified_two_level(16, 16, 17, eps=1e-3, sigma=0.3, seed=2)
    jeff, u, cfg = gpu_fs(atm, atom, prec=m.MG3D_PREC_F32, shape=(fpb, bands, threads, lean, PLANE))
    assert cfg == (fpb, bands, threads, lean, PLANE)
    jo, uo = oracle_fs(atm, atom, "16x16x17")
    assert rel(jeff, jo) < TOL_FS32
    assert rel(u, uo) < TOL_FS32


@pytest.mark.parametrize("n_freq", [1, 2, 3, 4, 5, 7, 11, 17, 33])
def test_frequency_counts_and_groups(n_freq):
    """One group up to 16 frequencies (single-frequency slot when n_freq is
    odd); beyond 16 the default takes groups of 16, the last one partial."""
    atom = synth.TwoLevelAtom(n_freq=n_freq)
    atm, _ = synth.stratified_two_level(8, 12, 17, eps=1e-2, atom=atom, sigma=0.2, seed=4)
    jeff, u, cfg = gpu_fs(atm, atom)
    assert cfg[4] == PLANE
    jo, uo = oracle_fs(atm, atom, ("nf", n_freq))
    assert rel(jeff, jo) < TOL_FS64
    assert rel(u, uo) < TOL_FS64


def test_groups_of_two_frequencies_with_custom_quadrature():
    """Five clusters per ray (pairs, then the line centre alone) with the
    a = 1/3 quadrature, whose steps cross at other horizontal offsets."""
    atm, atom = synth.stratified_two_level(12, 8, 17, eps=1e-2, sigma=0.3, seed=6)
    jeff, u, cfg = gpu_fs(atm, atom, shape=(2, 4, 64, 0, PLANE), quad_a=1.0 / 3.0)
    assert cfg == (2, 4, 64, 0, PLANE)
    jo, uo = oracle_fs(atm, atom, "quad13", quad_a=1.0 / 3.0)
    assert rel(jeff, jo) < TOL_FS64
    assert rel(u, uo) < TOL_FS64


def test_sixteen_block_cluster_with_ragged_last_band():
    """31 rows as 15 bands of 2 and a last band of 1: most stored rows are
    written by other blocks, and the last band's halo is row 0."""
    atm, atom = synth.stratified_two_level(8, 31, 9, eps=1e-3, sigma=0.3, seed=5)
    for prec, tol in ((m.MG3D_PREC_F64, TOL_FS64), (m.MG3D_PREC_F32, TOL_FS32)):
        jeff, u, cfg = gpu_fs(atm, atom, prec=prec, shape=(9, 16, 32, 0, PLANE))
        assert cfg == (9, 16, 32, 0, PLANE)
        jo, uo = oracle_fs(atm, atom, "8x31x9")
        assert rel(jeff, jo) < tol
        assert rel(u, uo) < tol


def test_full_bench_box_fp64_and_fp32():
    """The 64x64x129 bench atmosphere (log-normal sigma 0.3) at the default
    shape, every node against the oracle."""
    atm, atom = synth.box_64x64x129_lognormal(seed=1)
    jo, uo = oracle_fs(atm, atom, "bench")
    jeff, u, cfg = gpu_fs(atm, atom)
    assert cfg[4] == PLANE
    assert rel(jeff, jo) < TOL_FS64
    assert rel(u, uo) < TOL_FS64
    jeff, u, cfg = gpu_fs(atm, atom, prec=m.MG3D_PREC_F32)
    assert cfg[4] == PLANE
    assert rel(jeff, jo) < TOL_FS32
    assert rel(u, uo) < TOL_FS32


def test_plane_sweep_matches_band_sweep_and_is_reproducible():
    """The shifted-plane sweep and the band sweep (stage 0) are two kernels of
    the same arithmetic: equal to rounding; repeated launches are bitwise
    equal (fixed summation order)."""
    atm, atom = synth.stratified_two_level(16, 16, 33, eps=1e-3, sigma=0.3, seed=9)
    h = m.mg3d_create(atm, atom, n_grids=1)
    try:
        m.mg3d_mali_sweep(h, 1, 3)
        m.mg3d_set_fs_config(h, 1, 9, 4, 64, 0, PLANE)
        j1, u1 = m.mg3d_formal_solve(h, 1)
        j2, u2 = m.mg3d_formal_solve(h, 1)
        m.mg3d_set_fs_config(h, 1, 9, 4, 64, 0, 0)
        jb, ub = m.mg3d_formal_solve(h, 1)
    finally:
        m.mg3d_destroy(h)
    assert np.array_equal(j1, j2) and np.array_equal(u1, u2)
    assert rel(j1, jb) < 1e-13
    assert rel(u1, ub) < 1e-13


ASYNC = 3   # stage value of the shifted-plane sweep with transaction-counted stores

ASYNC_SHAPES = [
    # (precision, freq_per_block, bands, threads, lean)
    (m.MG3D_PREC_F64, 9, 2, 512, 0), (m.MG3D_PREC_F64, 9, 3, 64, 0),
    (m.MG3D_PREC_F64, 4, 6, 64, 0), (m.MG3D_PREC_F64, 9, 16, 32, 0),
    (m.MG3D_PREC_F32, 9, 6, 64, 0), (m.MG3D_PREC_F32, 9, 8, 64, 1),
    (m.MG3D_PREC_F32, 2, 4, 128, 1), (m.MG3D_PREC_F32, 4, 2, 1024, 0),
    (m.MG3D_PREC_F32, 6, 3, 64, 0),
]


@pytest.mark.parametrize("prec,fpb,bands,threads,lean", ASYNC_SHAPES)
def test_async_completion_equals_cluster_barriers(prec, fpb, bands, threads, lean):
    """Stores into other blocks counted on the receiving block's mbarrier
    (stage 3) order the same data as the per-plane cluster barrier (stage 2):
    the same arithmetic in the same order, so bitwise equal results, and the
    oracle's to the precision's bar.  Covers ragged bands (16 rows as 6+6+4,
    3x5+1, ...), a 16-block cluster, frequency groups with a one-frequency
    slot, both FP32 register budgets and 1024-thread blocks."""
    atm, atom = synth.stratified_two_level(16, 16, 17, eps=1e-3, sigma=0.3, seed=2)
    out = {}
    for stage in (PLANE, ASYNC):
        jeff, u, cfg = gpu_fs(atm, atom, prec=prec, shape=(fpb, bands, threads, lean, stage))
        assert cfg == (fpb, bands, threads, lean, stage)
        out[stage] = (jeff, u)
    assert np.array_equal(out[PLANE][0], out[ASYNC][0])
    assert np.array_equal(out[PLANE][1], out[ASYNC][1])
    tol = TOL_FS64 if prec == m.MG3D_PREC_F64 else TOL_FS32
    jo, uo = oracle_fs(atm, atom, "16x16x17")
    assert rel(out[ASYNC][0], jo) < tol
    assert rel(out[ASYNC][1], uo) < tol


def test_async_completion_on_the_bench_box_and_in_cycles():
    """The 64x64x129 bench box at 5 bands in both precisions against the
    oracle, then MALI sweeps and a V-cycle with stage 3 on every level equal
    bitwise to the same with stage 2 (and a graph replay of the cycle)."""
    atm, atom = synth.box_64x64x129_lognormal(seed=1)
    jo, uo = oracle_fs(atm, atom, "bench")
    for prec, tol in ((m.MG3D_PREC_F64, TOL_FS64), (m.MG3D_PREC_F32, TOL_FS32)):
        jeff, u, cfg = gpu_fs(atm, atom, prec=prec, shape=(9, 5, 512, 0, ASYNC))
        assert cfg[4] == ASYNC
        assert rel(jeff, jo) < tol and rel(u, uo) < tol
    atm, atom = synth.stratified_two_level(32, 32, 33, eps=1e-3, sigma=0.3, seed=3)
    res = {}
    for stage in (PLANE, ASYNC):
        h = m.mg3d_create(atm, atom, n_grids=2, fs_prec=m.MG3D_PREC_F64, nu0=2, nu1=2,
                          nu2=2, nu3=8)
        try:
            for level, bands in ((1, 2), (2, 4)):
                m.mg3d_set_fs_config(h, level, 9, bands, 128, 0, stage)
            m.mg3d_mali_sweep(h, 2, 2)
            m.mg3d_fas_vcycle(h, True)
            m.mg3d_fas_vcycle(h, False)
            res[stage] = m.mg3d_get_populations(h, 2)
        finally:
            m.mg3d_destroy(h)
    assert np.array_equal(res[PLANE], res[ASYNC])


def test_plane_shapes_refused_where_they_do_not_apply():
    atm, atom = synth.stratified_two_level(16, 16, 17, eps=1e-3, sigma=0.3, seed=2)
    h = m.mg3d_create(atm, atom, n_grids=1)
    try:
        for bad in [(3, 2, 64, 0, PLANE),     # odd group below n_freq
                    (8, 2, 64, 0, PLANE),     # 4 slots: not built
                    (9, 2, 64, 1, PLANE),     # FP64 has no 64-register variant
                    (9, 2, 48, 0, PLANE),     # not a multiple of 32 threads
                    (9, 2, 64, 0, 4)]:        # no sweep kind 4
            with pytest.raises(m.MG3DError):
                m.mg3d_set_fs_config(h, 1, *bad)
    finally:
        m.mg3d_destroy(h)
    atm, atom = synth.stratified_two_level(8, 8, 9, eps=1e-3, sigma=0.3, seed=2)
    h = m.mg3d_create(atm, atom, n_grids=1, sc_interp=1)
    try:
        assert m.mg3d_get_fs_config(h, 1)[4] != PLANE
        with pytest.raises(m.MG3DError):
            m.mg3d_set_fs_config(h, 1, 9, 2, 64, 0, PLANE)
    finally:
        m.mg3d_destroy(h)
