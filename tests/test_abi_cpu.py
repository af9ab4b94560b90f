"""CPU-side checks of the C ABI: the library builds, loads without a GPU and
exports every function include/mg3d.h declares; argument validation that
happens before any CUDA call returns the documented error codes."""

import os
import re

import numpy as np
import pytest

from paper_1701_01607_gb300 import build as B
from paper_1701_01607_gb300 import mg3d as m
from paper_1701_01607_gb300 import synth

HEADER = os.path.join(B.ROOT, "include", "mg3d.h")


def declared_functions():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(mg3d_[a-z_0-9]+)\s*\(", text)))


@pytest.fixture(scope="module")
def lib():
    B.build()
    return m.load()


def test_header_declares_the_boundary():
    names = declared_functions()
    for required in ("mg3d_create", "mg3d_formal_solve", "mg3d_mali_sweep",
                     "mg3d_fas_vcycle", "mg3d_fmg_solve", "mg3d_destroy"):
        assert required in names


def test_library_exports_every_declared_symbol(lib):
    for name in declared_functions():
        assert hasattr(lib, name), name
        assert name in m._SIGNATURES, name


def test_create_rejects_bad_grids_before_touching_the_gpu(lib):
    atm, atom = synth.stratified_two_level(16, 16, 33, eps=1e-3)
    # 33 nodes coarsen 5 times at most (32 = 2^5): 7 grids are impossible
    with pytest.raises(m.MG3DError) as ei:
        m.mg3d_create(atm, atom, n_grids=7)
    assert ei.value.code == m.MG3D_E_GRID
    atm2, _ = synth.stratified_two_level(12, 12, 33, eps=1e-3)
    with pytest.raises(m.MG3DError) as ei:
        m.mg3d_create(atm2, atom, n_grids=4)   # 12 is not a multiple of 8
    assert ei.value.code == m.MG3D_E_GRID
    with pytest.raises(m.MG3DError) as ei:
        m.mg3d_create(atm, atom, n_grids=1, fs_prec=5)
    assert ei.value.code == m.MG3D_E_ARG
    bad = synth.Atmosphere(atm.nx, atm.ny, atm.nz, atm.dx, atm.dy, atm.z[::-1].copy(),
                           atm.T, atm.n_tot, atm.c_ul)
    with pytest.raises(m.MG3DError) as ei:
        m.mg3d_create(bad, atom, n_grids=1)
    assert ei.value.code == m.MG3D_E_ARG
    assert "z must increase" in m.mg3d_last_error()


def test_null_handle_is_an_argument_error(lib):
    assert lib.mg3d_destroy(None) == m.MG3D_OK
    assert lib.mg3d_fas_vcycle(None, 0, None) == m.MG3D_E_ARG
    assert lib.mg3d_set_timing(None, 1) == m.MG3D_E_ARG
