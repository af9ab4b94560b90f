"""Parity of the CUDA path (through the C ABI) with the FP64 CPU oracle.

FP64 formal solutions must agree with the oracle to 1e-12 relative on Jeff and
U, and populations to 1e-10 relative after a fixed number of sweeps or cycles
(the only differences are rounding order, fused multiply-adds and the
last-bit differences of exp between CUDA and the C library).  The FP32 formal
solution is held to 1e-4 relative on populations.
"""

import numpy as np
import pytest

from oracle import mg3d_oracle as O
from paper_1701_01607_gb300 import mg3d as m
from paper_1701_01607_gb300 import synth

pytestmark = pytest.mark.gpu

PARAMS = dict(nu_fmg=16, nu0=0, nu1=2, nu2=2, nu3=32)
TOL_FS64 = 1e-12
TOL_POP64 = 1e-10
TOL_POP32 = 1e-4


def rel(a, b):
    return float(np.max(np.abs(a - b) / np.abs(b)))


@pytest.fixture(scope="module", autouse=True)
def lib():
    m.load(build_if_missing=True)


def make(atm, atom, n_grids=1, prec=m.MG3D_PREC_F64, **kw):
    p = dict(PARAMS)
    p.update(kw)
    return m.mg3d_create(atm, atom, n_grids=n_grids, fs_prec=prec, **p)


# ------------------------------------------------------------ formal solution

@pytest.mark.parametrize("shape", [(16, 16, 33), (12, 8, 17), (2, 2, 9), (1, 1, 3)])
def test_formal_solution_fp64(shape):
    nx, ny, nz = shape
    atm, atom = synth.stratified_two_level(nx, ny, nz, eps=1e-3, sigma=0.3, seed=11)
    h = make(atm, atom)
    try:
        jeff, u = m.mg3d_formal_solve(h, 1)
    finally:
        m.mg3d_destroy(h)
    prob = O.TwoLevelProblem(atm, atom)
    _, jo, uo = prob.formal_solution(1, prob.zero_radiation(1))
    assert rel(jeff, jo) < TOL_FS64
    assert rel(u, uo) < TOL_FS64


@pytest.mark.parametrize("ng,bands,lean", [(1, 1, 0), (9, 1, 1), (4, 3, 0), (2, 6, 1), (3, 8, 0),
                                           (9, 2, 1), (5, 6, 0)])
def test_formal_solution_every_launch_shape(ng, bands, lean):
    """Ragged frequency groups (9 = 4+4+1) and ragged bands (16 rows as 6+6+4
    or 3x5+1) exercise the distributed-shared-memory reads across blocks."""
    atm, atom = synth.stratified_two_level(16, 16, 17, eps=1e-3, sigma=0.3, seed=2)
    h = make(atm, atom)
    try:
        m.mg3d_set_fs_config(h, 1, ng, bands, 128, lean)
        assert m.mg3d_get_fs_config(h, 1) == (ng, bands, 128, lean, 1)
        jeff, u = m.mg3d_formal_solve(h, 1)
    finally:
        m.mg3d_destroy(h)
    prob = O.TwoLevelProblem(atm, atom)
    _, jo, uo = prob.formal_solution(1, prob.zero_radiation(1))
    assert rel(jeff, jo) < TOL_FS64
    assert rel(u, uo) < TOL_FS64


@pytest.mark.parametrize("ng,lean", [(3, 0), (9, 1), (2, 2)])
def test_formal_solution_sixteen_block_cluster(ng, lean):
    """Clusters of 16 blocks (a non-portable size): 31 rows as 15 bands of 2
    and a last band of 1, so most upwind rows come from peer blocks."""
    atm, atom = synth.stratified_two_level(8, 31, 9, eps=1e-3, sigma=0.3, seed=5)
    h = make(atm, atom)
    try:
        m.mg3d_set_fs_config(h, 1, ng, 16, 32, lean)
        assert m.mg3d_get_fs_config(h, 1) == (ng, 16, 32, lean, 1)
        jeff, u = m.mg3d_formal_solve(h, 1)
    finally:
        m.mg3d_destroy(h)
    prob = O.TwoLevelProblem(atm, atom)
    _, jo, uo = prob.formal_solution(1, prob.zero_radiation(1))
    assert rel(jeff, jo) < TOL_FS64
    assert rel(u, uo) < TOL_FS64


def test_formal_solution_single_frequency_and_custom_quadrature():
    atom = synth.TwoLevelAtom(n_freq=1)
    atm, _ = synth.stratified_two_level(8, 8, 17, eps=1e-2, atom=atom, sigma=0.2, seed=4)
    h = m.mg3d_create(atm, atom, quad_a=1.0 / 3.0, n_grids=1)
    try:
        jeff, u = m.mg3d_formal_solve(h, 1)
    finally:
        m.mg3d_destroy(h)
    prob = O.TwoLevelProblem(atm, atom, quad_a=1.0 / 3.0)
    _, jo, uo = prob.formal_solution(1, prob.zero_radiation(1))
    assert rel(jeff, jo) < TOL_FS64 and rel(u, uo) < TOL_FS64


# ------------------------------------------------------------------ MALI

def test_mali_sweeps_fp64():
    atm, atom = synth.box_16x16x33()
    h = make(atm, atom)
    prob = O.TwoLevelProblem(atm, atom)
    n = prob.zero_radiation(1)
    try:
        assert rel(m.mg3d_get_populations(h, 1), n) < 1e-14
        for _ in range(5):
            c_gpu = m.mg3d_mali_sweep(h, 1, 1)
            n, c_orc = prob.mali_sweep(1, n)
            assert abs(c_gpu - c_orc) <= 1e-9 * c_orc
        assert rel(m.mg3d_get_populations(h, 1), n) < TOL_POP64
        r_gpu = m.mg3d_residual(h, 1)
    finally:
        m.mg3d_destroy(h)
    _, je, uu = prob.formal_solution(1, n)
    M = prob.rate_matrix(1, je, uu)
    r_orc = prob.default_rhs(1) - prob.apply(M, n)
    # the residual is a difference of nearly equal rates: compare it on the
    # scale of the individual terms n_u P_ul and n_l P_lu
    scale = (np.abs(M[:, 1, 0] * n[0].reshape(-1)) +
             np.abs(M[:, 1, 1] * n[1].reshape(-1))).reshape(n[0].shape)
    assert np.max(np.abs(r_gpu[1] - r_orc[1]) / scale) < 1e-12


def test_mali_solve_matches_oracle_iteration_by_iteration():
    atm, atom = synth.box_16x16x33()
    h = make(atm, atom)
    try:
        st = m.mg3d_mali_solve(h, 1e-3)
        n_gpu = m.mg3d_get_populations(h, 1)
    finally:
        m.mg3d_destroy(h)
    prob = O.TwoLevelProblem(atm, atom)
    n_orc, it = O.mali_solve(prob, 1e-3)
    assert st["iterations"] == it
    assert rel(n_gpu, n_orc) < TOL_POP64
    np.testing.assert_allclose(n_gpu.sum(axis=0), atm.n_tot, rtol=1e-13)


def test_lte_limit_on_gpu():
    atm, atom = synth.stratified_two_level(8, 8, 17, eps=1e-3)
    atm.c_ul[:] = 1e12 * atom.a_ul
    h = make(atm, atom)
    try:
        m.mg3d_mali_sweep(h, 1, 1)
        n = m.mg3d_get_populations(h, 1)
    finally:
        m.mg3d_destroy(h)
    boltz = atom.g_ratio * np.exp(-atom.theta / atm.T)
    assert rel(n[1] / n[0], boltz) < 1e-11


# ------------------------------------------------------------ grid transfer

def test_restriction_and_prolongation_match_oracle():
    atm, atom = synth.stratified_two_level(16, 8, 17, eps=1e-3)
    atm.z = np.cumsum(np.r_[0.0, np.random.default_rng(3).uniform(0.5, 1.5, 16)])
    h = make(atm, atom, n_grids=3)
    rng = np.random.default_rng(9)
    try:
        fine = rng.uniform(0.1, 2.0, size=(3, 17, 8, 16))
        coarse = m.mg3d_restrict(h, 3, fine)
        assert rel(coarse, O.restrict_fw(fine)) < 1e-14
        c2 = rng.uniform(0.1, 2.0, size=(2, 9, 4, 8))
        up = m.mg3d_prolong(h, 3, c2)
        assert rel(up, O.prolong_trilinear(c2, atm.z)) < 1e-14
        c1 = rng.uniform(0.1, 2.0, size=(5, 2, 4))
        up1 = m.mg3d_prolong(h, 2, c1)
        assert rel(up1, O.prolong_trilinear(c1, atm.z[::2])) < 1e-14
        # coarse grids carry the full-weighted atmosphere
        shapes = [m.mg3d_level_shape(h, k) for k in (1, 2, 3)]
        assert shapes == [(4, 2, 5), (8, 4, 9), (16, 8, 17)]
    finally:
        m.mg3d_destroy(h)


# --------------------------------------------------------------- multigrid

@pytest.mark.parametrize("n_grids", [2, 3])
def test_fas_vcycles_fp64(n_grids):
    atm, atom = synth.stratified_two_level(16, 16, 33, eps=1e-3, sigma=0.3, seed=5)
    h = make(atm, atom, n_grids=n_grids)
    prob = O.TwoLevelProblem(atm, atom, n_grids=n_grids)
    n = prob.zero_radiation(n_grids)
    try:
        for cyc in range(3):
            c_gpu = m.mg3d_fas_vcycle(h, cyc == 0)
            n, c_orc = prob.fas_cycle(n, cyc == 0, PARAMS)
            assert abs(c_gpu - c_orc) <= 1e-8 * c_orc
            assert rel(m.mg3d_get_populations(h, n_grids), n) < TOL_POP64
    finally:
        m.mg3d_destroy(h)


def test_fas_and_fmg_solves_fp64():
    atm, atom = synth.stratified_two_level(16, 16, 33, eps=1e-3, sigma=0.3, seed=6)
    h = make(atm, atom, n_grids=3)
    try:
        st = m.mg3d_fas_solve(h, 1e-3, n_grids=3)
        n_fas = m.mg3d_get_populations(h, 3)
        st2 = m.mg3d_fmg_solve(h, 1e-3, n_grids=3)
        n_fmg = m.mg3d_get_populations(h, 3)
    finally:
        m.mg3d_destroy(h)
    prob = O.TwoLevelProblem(atm, atom, n_grids=3)
    n_o, cyc = O.fas_solve(prob, 1e-3, PARAMS)
    assert st["iterations"] == cyc
    assert st["formal_solutions"] == prob.fs_count
    assert rel(n_fas, n_o) < TOL_POP64
    prob2 = O.TwoLevelProblem(atm, atom, n_grids=3)
    n_f, cyc2 = O.fmg_solve(prob2, 1e-3, PARAMS)
    assert st2["iterations"] == cyc2
    assert rel(n_fmg, n_f) < TOL_POP64


def test_negative_population_rule_on_gpu():
    """The 10 % rule must act at the same nodes.  From the zero-radiation
    start the relative correction keeps populations positive (Sec. 4.6), so
    the case starts far from equilibrium instead (upper level scaled by
    exp(3 G) node by node) and runs one V-cycle without smoothing, after
    which the coarse grid returns negative populations at some nodes."""
    atm, atom = synth.stratified_two_level(16, 16, 33, eps=1e-3, sigma=0.3, seed=5)
    kw = dict(nu0=0, nu1=0, nu2=0, nu3=8)
    p = dict(PARAMS)
    p.update(kw)
    prob = O.TwoLevelProblem(atm, atom, n_grids=2)
    n0 = prob.zero_radiation(2)
    n0[1] *= np.exp(3.0 * np.random.default_rng(1).normal(size=n0[1].shape))
    n, _ = prob.fas_cycle(n0, False, p)
    assert prob.negatives > 0
    h = make(atm, atom, n_grids=2, **kw)
    try:
        m.mg3d_set_populations(h, 2, n0)
        m.mg3d_fas_vcycle(h, False)
        r = rel(m.mg3d_get_populations(h, 2), n)
        assert r < 1e-10, r
    finally:
        m.mg3d_destroy(h)


# ------------------------------------------------------------ mixed precision

def test_fp32_formal_solution_and_converged_populations():
    atm, atom = synth.box_16x16x33()
    h = make(atm, atom, prec=m.MG3D_PREC_F32)
    try:
        jeff, u = m.mg3d_formal_solve(h, 1)
        st = m.mg3d_mali_solve(h, 1e-3)
        n32 = m.mg3d_get_populations(h, 1)
    finally:
        m.mg3d_destroy(h)
    prob = O.TwoLevelProblem(atm, atom)
    _, jo, uo = prob.formal_solution(1, prob.zero_radiation(1))
    assert rel(jeff, jo) < 1e-5 and rel(u, uo) < 1e-5
    n_o = prob.zero_radiation(1)
    for _ in range(st["iterations"]):
        n_o, _ = prob.mali_sweep(1, n_o)
    assert rel(n32, n_o) < TOL_POP32


# --------------------------------------- full size, bench launch configuration

def test_full_size_formal_solution_fp64_and_fp32():
    """64x64x129, perturbed, 9 frequencies: the sweep shapes the bench uses."""
    atm, atom = synth.box_64x64x129_lognormal()
    prob = O.TwoLevelProblem(atm, atom, n_grids=3)
    n0 = prob.zero_radiation(3)
    _, jo, uo = prob.formal_solution(3, n0)
    for prec, tol in ((m.MG3D_PREC_F64, TOL_FS64), (m.MG3D_PREC_F32, 2e-5)):
        h = make(atm, atom, n_grids=3, prec=prec)
        try:
            jeff, u = m.mg3d_formal_solve(h, 3)
            m.mg3d_mali_sweep(h, 3, 1)
            n1 = m.mg3d_get_populations(h, 3)
        finally:
            m.mg3d_destroy(h)
        assert rel(jeff, jo) < tol, prec
        assert rel(u, uo) < tol, prec
        if prec == m.MG3D_PREC_F64:
            n1o, _ = prob.mali_sweep(3, n0)
            assert rel(n1, n1o) < TOL_POP64


# ------------------------------------------------------- sweep internals

def test_sweep_exp_matches_cuda_exp():
    """The sweep's table-driven FP64 e^{-x} against CUDA's exp (within 2 ulp)."""
    x = np.concatenate([np.linspace(0.0, 707.9, 200001),
                        np.logspace(-14, np.log10(707.9), 50001), [0.0, 5e-324, 1e-300]])
    ours, ref = m.mg3d_check_exp(x)
    assert np.all(np.isfinite(ours))
    assert np.max(np.abs(ours - ref) / ref) < 4.5e-16
    big, _ = m.mg3d_check_exp(np.array([708.5, 745.2, 1000.0, 1e300]))
    assert np.all(big == 0.0)


def test_autotuned_shapes_keep_parity():
    atm, atom = synth.stratified_two_level(16, 16, 33, eps=1e-3, sigma=0.3, seed=12)
    h = make(atm, atom, n_grids=2)
    prob = O.TwoLevelProblem(atm, atom, n_grids=2)
    try:
        info = m.mg3d_autotune(h)
        assert info["evaluated"] > 10
        for k in (1, 2):
            jeff, u = m.mg3d_formal_solve(h, k)
            _, jo, uo = prob.formal_solution(k, prob.zero_radiation(k))
            assert rel(jeff, jo) < TOL_FS64 and rel(u, uo) < TOL_FS64, k
        c = m.mg3d_fas_vcycle(h, True)
        n, co = prob.fas_cycle(prob.zero_radiation(2), True, PARAMS)
        assert rel(m.mg3d_get_populations(h, 2), n) < TOL_POP64
    finally:
        m.mg3d_destroy(h)


def test_graph_replayed_vcycles_equal_direct_launches():
    """V-cycles replayed from CUDA graphs give bit-identical populations and
    the same counters as the same cycles launched one kernel at a time."""
    atm, atom = synth.stratified_two_level(16, 16, 33, eps=1e-3, sigma=0.3, seed=13)
    hg = make(atm, atom, n_grids=3)
    hd = make(atm, atom, n_grids=3)
    try:
        m.mg3d_set_graphs(hd, False)
        m.mg3d_set_timing(hg, True)
        for cyc in range(4):
            cg = m.mg3d_fas_vcycle(hg, cyc == 0)
            cd = m.mg3d_fas_vcycle(hd, cyc == 0)
            assert cg == cd
        assert np.array_equal(m.mg3d_get_populations(hg, 3), m.mg3d_get_populations(hd, 3))
        ctg, ctd = m.mg3d_get_counters(hg), m.mg3d_get_counters(hd)
        assert ctg["fs_launches"] == ctd["fs_launches"]
        assert ctg["fs_units"] == ctd["fs_units"]
        assert ctg["kernel_launches"] == ctd["kernel_launches"]
        assert ctg["level_fs_timed_launches"][3] == ctg["level_fs_launches"][3]
        assert ctg["level_fs_kernel_ms"][3] > 0
    finally:
        m.mg3d_destroy(hg)
        m.mg3d_destroy(hd)


# ------------------------------------------------ checkpoint and failures

def test_resume_from_checkpoint_is_bitwise_identical():
    """MALI for 6 sweeps equals 3 sweeps, a host checkpoint of the
    populations, a fresh handle and 3 more sweeps, bit for bit; the same for
    FAS V-cycles."""
    atm, atom = synth.stratified_two_level(16, 16, 33, eps=1e-3, sigma=0.3, seed=14)
    for n_grids, step in ((1, lambda h: m.mg3d_mali_sweep(h, 1, 1)),
                          (3, lambda h: m.mg3d_fas_vcycle(h, False))):
        full = make(atm, atom, n_grids=n_grids)
        a = make(atm, atom, n_grids=n_grids)
        try:
            for _ in range(6):
                step(full)
            for _ in range(3):
                step(a)
            ckpt = m.mg3d_get_populations(a, n_grids)
        finally:
            m.mg3d_destroy(a)
        b = make(atm, atom, n_grids=n_grids)
        try:
            m.mg3d_set_populations(b, n_grids, ckpt)
            for _ in range(3):
                step(b)
            assert np.array_equal(m.mg3d_get_populations(b, n_grids),
                                  m.mg3d_get_populations(full, n_grids))
        finally:
            m.mg3d_destroy(b)
            m.mg3d_destroy(full)


def test_non_finite_populations_are_reported_not_faulted():
    """A NaN planted in the populations makes the next sweep and V-cycle
    return MG3D_E_DIVERGED; the GPU context stays usable afterwards."""
    atm, atom = synth.stratified_two_level(8, 8, 17, eps=1e-3, seed=15)
    h = make(atm, atom, n_grids=2)
    try:
        n = m.mg3d_get_populations(h, 2)
        n[1, 5, 3, 4] = np.nan
        m.mg3d_set_populations(h, 2, n)
        with pytest.raises(m.MG3DError) as ei:
            m.mg3d_mali_sweep(h, 2, 1)
        assert ei.value.code == m.MG3D_E_DIVERGED
        m.mg3d_set_populations(h, 2, n)
        with pytest.raises(m.MG3DError) as ei:
            m.mg3d_fas_vcycle(h, False)
        assert ei.value.code == m.MG3D_E_DIVERGED
        m.mg3d_init_zero_radiation(h, 2)
        assert np.isfinite(m.mg3d_mali_sweep(h, 2, 1))
    finally:
        m.mg3d_destroy(h)
    h2 = make(atm, atom)
    try:
        m.mg3d_mali_sweep(h2, 1, 1)
    finally:
        m.mg3d_destroy(h2)


def test_iteration_cap_returns_maxiter():
    atm, atom = synth.stratified_two_level(8, 8, 17, eps=1e-3, seed=16)
    h = make(atm, atom, n_grids=2)
    try:
        with pytest.raises(m.MG3DError) as ei:
            m.mg3d_mali_solve(h, 1e-12, 3)
        assert ei.value.code == m.MG3D_E_MAXITER
        with pytest.raises(m.MG3DError) as ei:
            m.mg3d_fas_solve(h, 1e-14, 2, n_grids=2)
        assert ei.value.code == m.MG3D_E_MAXITER
    finally:
        m.mg3d_destroy(h)


@pytest.mark.parametrize("mode", [m.MG3D_RESTRICT_HALF, m.MG3D_RESTRICT_INJECT])
def test_restriction_variants_match_oracle(mode):
    atm, atom = synth.stratified_two_level(16, 16, 33, eps=1e-3, sigma=0.3, seed=17)
    h = m.mg3d_create(atm, atom, n_grids=3, restriction=mode, **PARAMS)
    prob = O.TwoLevelProblem(atm, atom, n_grids=3, restriction=mode)
    n = prob.zero_radiation(3)
    try:
        f = np.random.default_rng(3).uniform(0.5, 1.5, size=(2, 33, 16, 16))
        ref = O.restrict_hw(f) if mode == m.MG3D_RESTRICT_HALF else O.restrict_inj(f)
        assert rel(m.mg3d_restrict(h, 3, f), ref) < 1e-14
        for cyc in range(2):
            m.mg3d_fas_vcycle(h, cyc == 0)
            n, _ = prob.fas_cycle(n, cyc == 0, PARAMS)
        assert rel(m.mg3d_get_populations(h, 3), n) < TOL_POP64
    finally:
        m.mg3d_destroy(h)
