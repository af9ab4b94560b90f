"""Allocation-free formal solution against the handle-based one.

mg3d_formal_solve_noalloc is for callers that cannot allocate device memory
when they need a formal solution (code under another framework's memory pool,
allocation-free sections of a pipeline, a process whose device memory is all
held by a caching allocator).  Here the caller's buffers come from torch; the
entry point itself must allocate nothing.  Calls in a row on different
problems must each give the Jeff and U of mg3d_formal_solve on that problem to
the FP64 formal-solution tolerance of the parity tests (1e-12 relative), so
nothing left in the shared scratch by one call may leak into the next.

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


def _case(nx, ny, nz, seed, sweeps):
    """A box, its handle-path Jeff and U after `sweeps` MALI sweeps, and the
    caller's inputs (chi0, S, bottom intensity) from the same populations."""
    atm, atom = synth.stratified_two_level(nx, ny, nz, eps=1e-3, sigma=0.3, seed=seed)
    h = m.mg3d_create(atm, atom, n_grids=1, fs_prec=m.MG3D_PREC_F64)
    try:
        m.mg3d_mali_sweep(h, 1, sweeps)
        n = m.mg3d_get_populations(h, 1)
        j_ref, u_ref = m.mg3d_formal_solve(h, 1)
    finally:
        m.mg3d_destroy(h)
    diff = n[0] * atom.g_ratio - n[1]
    return atm, atom, atom.kappa * diff, n[1] / diff, 1.0 / np.expm1(atom.theta / atm.T[0]), \
        j_ref, u_ref


def test_noalloc_formal_solution_matches_handle_path_twice():
    """Two calls in a row on different problems (the second on a smaller grid
    with other opacities and source functions), each against its own
    handle-path result; outputs start as NaN, and after the first call (which
    reserves the scratch on this device) the calls change the device's free
    memory by nothing."""
    torch = pytest.importorskip("torch")
    m.load(build_if_missing=True)
    dev = torch.device("cuda")

    def d(a):
        return torch.tensor(np.ascontiguousarray(a), dtype=torch.float64, device=dev)

    cases = [_case(16, 16, 33, 21, 2), _case(8, 12, 17, 22, 5), _case(16, 16, 33, 21, 2)]
    bufs = []
    for atm, atom, chi0, S, bbot, _, _ in cases:
        bufs.append((d(atm.z), d(chi0), d(S), d(bbot),
                     torch.empty(atm.shape, dtype=torch.float64, device=dev),
                     torch.empty(atm.shape, dtype=torch.float64, device=dev)))
    torch.cuda.synchronize()
    stream = torch.cuda.current_stream().cuda_stream
    free_after_first = None
    for call, ((atm, atom, _, _, _, j_ref, u_ref), (z_d, chi_d, S_d, b_d, j_d, u_d)) in \
            enumerate(zip(cases, bufs)):
        j_d.fill_(float("nan"))
        u_d.fill_(float("nan"))
        torch.cuda.synchronize()
        rc = m.mg3d_formal_solve_noalloc(atm.nx, atm.ny, atm.nz, atm.dx, atm.dy,
                                         z_d.data_ptr(), atom, 0.0, chi_d.data_ptr(),
                                         S_d.data_ptr(), b_d.data_ptr(), j_d.data_ptr(),
                                         u_d.data_ptr(), stream)
        torch.cuda.synchronize()
        assert rc == m.MG3D_OK, m.mg3d_last_error()
        free = torch.cuda.mem_get_info()[0]
        if call == 0:
            free_after_first = free
        else:
            assert free == free_after_first, call
        assert rel(j_d.cpu().numpy(), j_ref) < TOL_FS64, call
        assert rel(u_d.cpu().numpy(), u_ref) < TOL_FS64, call


def test_noalloc_refuses_planes_beyond_shared_memory():
    """Within the node, plane and frequency limits a plane can still be too
    large for one band's intensities of every frequency: 64 x 64 with 32
    frequencies is refused with a message, before any work is enqueued."""
    torch = pytest.importorskip("torch")
    m.load(build_if_missing=True)
    atom = synth.TwoLevelAtom(n_freq=32)
    buf = torch.zeros(16, dtype=torch.float64, device="cuda")
    p = buf.data_ptr()
    rc = m.mg3d_formal_solve_noalloc(64, 64, 9, 1.0, 1.0, p, atom, 0.0, p, p, p, p, p, None)
    assert rc == m.MG3D_E_ARG
    assert "shared memory" in m.mg3d_last_error()


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
