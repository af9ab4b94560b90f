"""The boundary's device-pointer calls and the per-call precision, through the
C ABI with PyTorch device buffers and a PyTorch stream.

mg3d_formal_solve_dev writes Jeff and U (the formal solution's outputs the
MALI update of Sec. 2.1 takes) into caller-owned device buffers, ordered on
the caller's stream; mg3d_get/set_populations_dev move the populations (n of
Eq. 4) between the handle and device buffers the same way;
mg3d_formal_solve_ex runs the formal solution in a precision other than the
handle's.  Each must give what the host-buffer path gives, and the oracle's
values to the bars of the parity tests (1e-12 FP64, 2e-5 FP32 on Jeff, U).
"""

import numpy as np
import pytest

from oracle import mg3d_oracle as O
from paper_1701_01607_gb300 import mg3d as m
from paper_1701_01607_gb300 import synth

pytestmark = pytest.mark.gpu

TOL_FS64 = 1e-12
TOL_FS32 = 2e-5


def rel(a, b):
    return float(np.max(np.abs(a - b) / np.abs(b)))


@pytest.fixture(scope="module", autouse=True)
def lib():
    m.load(build_if_missing=True)


@pytest.fixture(scope="module")
def case():
    atm, atom = synth.stratified_two_level(16, 16, 33, eps=1e-3, sigma=0.3, seed=8)
    prob = O.TwoLevelProblem(atm, atom)
    n0 = prob.zero_radiation(1)
    _, jo, uo = prob.formal_solution(1, n0)
    n1, _ = prob.mali_sweep(1, n0)
    return atm, atom, jo, uo, n1


def test_formal_solve_dev_on_a_torch_stream(case):
    torch = pytest.importorskip("torch")
    atm, atom, jo, uo, _ = case
    h = m.mg3d_create(atm, atom, n_grids=1, fs_prec=m.MG3D_PREC_F64)
    try:
        j_host, u_host = m.mg3d_formal_solve(h, 1)
        stream = torch.cuda.Stream()
        with torch.cuda.stream(stream):
            j = torch.full(atm.shape, float("nan"), dtype=torch.float64, device="cuda")
            u = torch.full(atm.shape, float("nan"), dtype=torch.float64, device="cuda")
            m.mg3d_formal_solve_dev(h, 1, m.MG3D_PREC_F64, j.data_ptr(), u.data_ptr(),
                                    stream.cuda_stream)
            # work queued on the stream after the call sees the results
            total = (j * 2.0 + u).sum()
        stream.synchronize()
        j_dev, u_dev = j.cpu().numpy(), u.cpu().numpy()
    finally:
        m.mg3d_destroy(h)
    assert np.array_equal(j_dev, j_host) and np.array_equal(u_dev, u_host)
    assert abs(float(total) - float((2.0 * j_host + u_host).sum())) < 1e-9 * abs(float(total))
    assert rel(j_dev, jo) < TOL_FS64 and rel(u_dev, uo) < TOL_FS64


def test_populations_dev_round_trip_and_ordering(case):
    torch = pytest.importorskip("torch")
    atm, atom, _, _, n1 = case
    h = m.mg3d_create(atm, atom, n_grids=1, fs_prec=m.MG3D_PREC_F64)
    try:
        n0_host = m.mg3d_get_populations(h, 1)
        stream = torch.cuda.Stream()
        with torch.cuda.stream(stream):
            buf = torch.zeros((2,) + atm.shape, dtype=torch.float64, device="cuda")
            m.mg3d_get_populations_dev(h, 1, buf.data_ptr(), stream.cuda_stream)
            got = buf.clone()
            # produced by a torch kernel on the same stream just before the call
            scaled = buf * 3.0
            m.mg3d_set_populations_dev(h, 1, scaled.data_ptr(), stream.cuda_stream)
        stream.synchronize()
        assert np.array_equal(got.cpu().numpy(), n0_host)
        assert np.array_equal(m.mg3d_get_populations(h, 1), 3.0 * n0_host)
        # back to the zero-radiation start through device memory, then one
        # MALI sweep: the oracle's first sweep
        with torch.cuda.stream(stream):
            m.mg3d_set_populations_dev(h, 1, buf.data_ptr(), stream.cuda_stream)
        stream.synchronize()
        m.mg3d_mali_sweep(h, 1, 1)
        assert rel(m.mg3d_get_populations(h, 1), n1) < 1e-10
    finally:
        m.mg3d_destroy(h)


@pytest.mark.parametrize("handle_prec", [m.MG3D_PREC_F64, m.MG3D_PREC_F32])
def test_formal_solve_in_the_other_precision(case, handle_prec):
    """An FP64 handle asked for an FP32 formal solution gives what an FP32
    handle gives (same kernel and launch shape, so the same bits), and an
    FP32 handle asked for FP64 gives the FP64 oracle's values; the handle's
    own precision is untouched."""
    torch = pytest.importorskip("torch")
    atm, atom, jo, uo, _ = case
    other = m.MG3D_PREC_F32 if handle_prec == m.MG3D_PREC_F64 else m.MG3D_PREC_F64
    h = m.mg3d_create(atm, atom, n_grids=1, fs_prec=handle_prec)
    ref = m.mg3d_create(atm, atom, n_grids=1, fs_prec=other)
    try:
        j_own, u_own = m.mg3d_formal_solve(h, 1)
        j_o, u_o = m.mg3d_formal_solve_ex(h, 1, other)
        j_ref, u_ref = m.mg3d_formal_solve(ref, 1)
        j2, u2 = m.mg3d_formal_solve_ex(h, 1, other)          # buffers reused
        j_same, _ = m.mg3d_formal_solve_ex(h, 1, handle_prec)
        jd = torch.empty(atm.shape, dtype=torch.float64, device="cuda")
        m.mg3d_formal_solve_dev(h, 1, other, jd.data_ptr(), None, None)
        torch.cuda.synchronize()
    finally:
        m.mg3d_destroy(h)
        m.mg3d_destroy(ref)
    assert np.array_equal(j_o, j_ref) and np.array_equal(u_o, u_ref)
    assert np.array_equal(j2, j_o) and np.array_equal(u2, u_o)
    assert np.array_equal(jd.cpu().numpy(), j_o)
    assert np.array_equal(j_same, j_own)
    tol_other = TOL_FS64 if other == m.MG3D_PREC_F64 else TOL_FS32
    tol_own = TOL_FS64 if handle_prec == m.MG3D_PREC_F64 else TOL_FS32
    assert rel(j_o, jo) < tol_other and rel(u_o, uo) < tol_other
    assert rel(j_own, jo) < tol_own and rel(u_own, uo) < tol_own


def test_device_calls_refused_where_they_do_not_apply():
    torch = pytest.importorskip("torch")
    atom = synth.hydrogen_like_atom(line_freq=3, cont_freq=2, seed=2)
    atm = synth.chromosphere(8, 8, 9, atom, seed=2)
    h = m.mg3d_create_ml(atm, atom, n_grids=1)
    buf = torch.zeros(8 * 8 * 9 * 6, dtype=torch.float64, device="cuda")
    try:
        with pytest.raises(m.MG3DError) as ei:
            m.mg3d_formal_solve_dev(h, 1, m.MG3D_PREC_F64, buf.data_ptr(), None, None)
        assert ei.value.code == m.MG3D_E_STATE
        # populations move for either kind of atom
        m.mg3d_get_populations_dev(h, 1, buf.data_ptr(), None)
        torch.cuda.synchronize()
        assert np.array_equal(buf.cpu().numpy().reshape(6, 9, 8, 8),
                              m.mg3d_get_populations(h, 1))
    finally:
        m.mg3d_destroy(h)
    atm2, atom2 = synth.stratified_two_level(8, 8, 9, eps=1e-3, sigma=0.3, seed=2)
    h = m.mg3d_create(atm2, atom2, n_grids=1, sc_interp=1)
    try:
        with pytest.raises(m.MG3DError) as ei:
            m.mg3d_formal_solve_ex(h, 1, m.MG3D_PREC_F32)
        assert ei.value.code == m.MG3D_E_ARG
        with pytest.raises(m.MG3DError):
            m.mg3d_formal_solve_ex(h, 1, 7)
    finally:
        m.mg3d_destroy(h)
