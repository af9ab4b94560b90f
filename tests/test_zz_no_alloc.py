"""Allocation-free formal solution against the handle-based one.

mg3d_formal_solve_noalloc is for callers that cannot allocate device memory
when they need a formal solution (code under another framework's memory pool,
allocation-free sections of a pipeline, a process whose device memory is all
held by a caching allocator).  Here the caller's buffers come from torch; the
entry point itself must allocate nothing.  Two calls in a row must both give
the Jeff and U of mg3d_formal_solve to the FP64 formal-solution tolerance of
the parity tests (1e-12 relative), so nothing left in the shared scratch by
one call may leak into the next.

This file is named to be collected last.
"""

import numpy as np
import pytest

from paper_1701_01607_gb300 import mg3d as m
from paper_1701_01607_gb300 import synth

pytestmark = pytest.mark.gpu

TOL_FS64 = 1e-12


def rel(a, b):
    return float(np.max(np.abs(a - b) / np.abs(b)))


def test_noalloc_formal_solution_matches_handle_path_twice():
    torch = pytest.importorskip("torch")
    m.load(build_if_missing=True)
    atm, atom = synth.stratified_two_level(16, 16, 33, eps=1e-3, sigma=0.3, seed=21)
    h = m.mg3d_create(atm, atom, n_grids=1, fs_prec=m.MG3D_PREC_F64)
    try:
        m.mg3d_mali_sweep(h, 1, 2)
        n = m.mg3d_get_populations(h, 1)
        j_ref, u_ref = m.mg3d_formal_solve(h, 1)
    finally:
        m.mg3d_destroy(h)

    # the caller's inputs, from the same populations
    diff = n[0] * atom.g_ratio - n[1]
    chi0 = atom.kappa * diff
    S = n[1] / diff
    bbot = 1.0 / np.expm1(atom.theta / atm.T[0])
    dev = torch.device("cuda")

    def d(a):
        return torch.tensor(np.ascontiguousarray(a), dtype=torch.float64, device=dev)

    z_d, chi_d, S_d, b_d = d(atm.z), d(chi0), d(S), d(bbot)
    j_d = torch.empty(atm.shape, dtype=torch.float64, device=dev)
    u_d = torch.empty(atm.shape, dtype=torch.float64, device=dev)
    stream = torch.cuda.current_stream().cuda_stream
    for call in range(2):
        j_d.fill_(float("nan"))
        u_d.fill_(-1.0)
        torch.cuda.synchronize()
        rc = m.mg3d_formal_solve_noalloc(atm.nx, atm.ny, atm.nz, atm.dx, atm.dy,
                                         z_d.data_ptr(), atom, 0.0, chi_d.data_ptr(),
                                         S_d.data_ptr(), b_d.data_ptr(), j_d.data_ptr(),
                                         u_d.data_ptr(), stream)
        torch.cuda.synchronize()
        assert rc == m.MG3D_OK, m.mg3d_last_error()
        j = j_d.cpu().numpy()
        u = u_d.cpu().numpy()
        assert rel(j, j_ref) < TOL_FS64, call
        assert rel(u, u_ref) < TOL_FS64, call


def test_noalloc_rejects_grids_beyond_its_limit():
    torch = pytest.importorskip("torch")
    m.load(build_if_missing=True)
    atom = synth.TwoLevelAtom()
    buf = torch.zeros(16, dtype=torch.float64, device="cuda")
    p = buf.data_ptr()
    rc = m.mg3d_formal_solve_noalloc(256, 256, 33, 1.0, 1.0, p, atom, 0.0, p, p, p, p, p, None)
    assert rc == m.MG3D_E_ARG
    assert "exceeds the allocation-free limit" in m.mg3d_last_error()
    many = synth.TwoLevelAtom(n_freq=m.MG3D_NOALLOC_MAX_FREQ + 1)
    rc = m.mg3d_formal_solve_noalloc(8, 8, 9, 1.0, 1.0, p, many, 0.0, p, p, p, p, p, None)
    assert rc == m.MG3D_E_ARG
