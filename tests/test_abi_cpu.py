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
    with open(HEADER) as fh:
        text = fh.read()
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


def test_every_declaration_is_documented_with_its_passage():
    """Each function of the header sits under a comment that cites the
    passage of the paper it follows (Sec., Eq., Table or Fig.) or says that
    it has no counterpart in the paper; grouped declarations share their
    group's comment."""
    with open(HEADER) as fh:
        text = fh.read()
    decls = list(re.finditer(r"^(?:int|const char|void)\s*\**\s*(mg3d_[a-z_0-9]+)\s*\(",
                             text, flags=re.M))
    assert {d.group(1) for d in decls} == set(declared_functions())
    for d in decls:
        before = text[:d.start()]
        end = before.rfind("*/")
        comment = before[before.rfind("/*", 0, end):end]
        assert re.search(r"Sec\.|Eqs?\.|Table|Fig\.|no counterpart in the paper", comment,
                         flags=re.I), d.group(1)


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
    # damping: non-negative, and not with a velocity field
    with pytest.raises(m.MG3DError) as ei:
        m.mg3d_create(atm, synth.TwoLevelAtom(a_damp=-0.1), n_grids=1)
    assert ei.value.code == m.MG3D_E_ARG and "a_damp" in m.mg3d_last_error()
    vatm, _ = synth.stratified_two_level(16, 16, 33, eps=1e-3, velocity=1.0)
    with pytest.raises(m.MG3DError) as ei:
        m.mg3d_create(vatm, synth.TwoLevelAtom(a_damp=0.05), n_grids=1)
    assert ei.value.code == m.MG3D_E_ARG and "Doppler" in m.mg3d_last_error()
    # damped lines of a multi-level atom: non-negative, static, not with PRD
    ml_atom = synth.hydrogen_like_atom(line_freq=5, cont_freq=3, a_damp=-0.01)
    ml_atm = synth.chromosphere(8, 8, 17, ml_atom)
    with pytest.raises(m.MG3DError) as ei:
        m.mg3d_create_ml(ml_atm, ml_atom, n_grids=1)
    assert ei.value.code == m.MG3D_E_ARG and "a_damp" in m.mg3d_last_error()
    ml_atom = synth.hydrogen_like_atom(line_freq=5, cont_freq=3, a_damp=0.01)
    vml = synth.chromosphere(8, 8, 17, ml_atom, velocity=0.5)
    with pytest.raises(m.MG3DError) as ei:
        m.mg3d_create_ml(vml, ml_atom, n_grids=1)
    assert ei.value.code == m.MG3D_E_ARG and "static" in m.mg3d_last_error()
    ml_atom = synth.hydrogen_like_atom(line_freq=5, cont_freq=3, a_damp=0.01, gamma_prd=0.5)
    with pytest.raises(m.MG3DError) as ei:
        m.mg3d_create_ml(ml_atm, ml_atom, n_grids=1)
    assert ei.value.code == m.MG3D_E_ARG and "damped" in m.mg3d_last_error()


def test_allocation_free_call_refuses_prd_and_damping(lib):
    """Checked before any CUDA call: the dummy addresses are never touched."""
    for atom in (synth.TwoLevelAtom(gamma_prd=0.5), synth.TwoLevelAtom(a_damp=0.1)):
        rc = m.mg3d_formal_solve_noalloc(4, 4, 5, 1.0, 1.0, 256, atom, 0.0, 256, 256, 256,
                                         256, 256)
        assert rc == m.MG3D_E_ARG
        assert "Doppler" in m.mg3d_last_error()


def test_quadrature_parameter_is_checked_before_the_gpu(lib):
    """a >= 1/sqrt(2) leaves b = sqrt(1 - 2a^2) without a real positive value,
    and a non-finite a is no quadrature: both entry points refuse them before
    any CUDA call (the dummy addresses are never touched)."""
    atm, atom = synth.stratified_two_level(8, 8, 9, eps=1e-3)
    for a in (0.75, 2.0 ** -0.5, float("nan"), float("inf")):
        with pytest.raises(m.MG3DError) as ei:
            m.mg3d_create(atm, atom, quad_a=a, n_grids=1)
        assert ei.value.code == m.MG3D_E_ARG and "quadrature" in m.mg3d_last_error()
        rc = m.mg3d_formal_solve_noalloc(4, 4, 5, 1.0, 1.0, 256, synth.TwoLevelAtom(), a, 256,
                                         256, 256, 256, 256)
        assert rc == m.MG3D_E_ARG and "quadrature" in m.mg3d_last_error()


def test_host_line_tables_match_scipy_and_the_oracle(lib):
    """The Voigt function and R_II-A the library tabulates for damped atoms
    (host code, no GPU) against scipy's Faddeeva function and the oracle's
    angle-averaged redistribution."""
    special = pytest.importorskip("scipy.special")
    from oracle import mg3d_oracle as O
    x = np.array([0.0, 0.3, 1.0, 2.5, 5.0, 8.0, -1.7])
    xp = np.array([0.0, 1.3, -0.7, 4.0, -5.0, 2.0, 1.1])
    for a in (0.01, 0.05, 0.5):
        H, R = m.mg3d_check_profiles(a, x, xp)
        assert np.allclose(H, special.wofz(x + 1j * a).real, rtol=1e-12, atol=0)
        ref = np.array([O.redistribution_r2a(u, v, a) for u, v in zip(x, xp)])
        assert np.allclose(R, ref, rtol=1e-8, atol=1e-15)
    H0, R0 = m.mg3d_check_profiles(0.0, x, xp)
    assert np.allclose(H0, np.exp(-x * x), rtol=1e-15)
    assert np.allclose(R0, 0.5 * special.erfc(np.maximum(np.abs(x), np.abs(xp))), rtol=1e-15)


def test_rational_voigt_function_within_its_error_bound(lib):
    """The 40-term rational Voigt function against scipy's Faddeeva function
    over damping 1e-4 .. 1e4 and offsets to 1e5: relative error below
    5e-14 + 2e-14/a (its rounding bound); invalid damping is refused."""
    special = pytest.importorskip("scipy.special")
    x = np.r_[np.linspace(0.0, 10.0, 401), np.linspace(10.0, 100.0, 91),
              np.geomspace(100.0, 1e5, 16)]
    x = np.r_[-x[::-1], x]
    for a in (1e-4, 1e-3, 0.01, 0.05, 0.5, 1.0, 3.0, 30.0, 1e4):
        H = m.mg3d_check_voigt(a, x)
        ref = special.wofz(x + 1j * a).real
        assert np.all(np.abs(H / ref - 1.0) <= 5e-14 + 2e-14 / a), a
    for bad in (0.0, -1.0, np.inf, np.nan):
        with pytest.raises(m.MG3DError):
            m.mg3d_check_voigt(bad, x[:3])


def test_null_handle_is_an_argument_error(lib):
    assert lib.mg3d_destroy(None) == m.MG3D_OK
    assert lib.mg3d_fas_vcycle(None, 0, None) == m.MG3D_E_ARG
    assert lib.mg3d_set_timing(None, 1) == m.MG3D_E_ARG


STRUCTS = ("mg3d_atmosphere", "mg3d_atom", "mg3d_quadrature", "mg3d_params", "mg3d_stats",
           "mg3d_counters", "mg3d_line", "mg3d_continuum", "mg3d_ml_atom", "mg3d_ml_atmosphere")


def test_binding_structs_match_the_header_layout(tmp_path):
    """Every struct of the header has the binding's size and field offsets
    (gcc compiles the header and prints them), so a field added on one side
    only fails here."""
    import ctypes
    import subprocess
    lines = ['#include <stddef.h>', '#include <stdio.h>', '#include "mg3d.h"', 'int main(void) {']
    for name in STRUCTS:
        lines.append(f'printf("{name} size %zu\\n", sizeof({name}));')
        for field, _ in getattr(m, name)._fields_:
            lines.append(f'printf("{name} {field} %zu\\n", offsetof({name}, {field}));')
    lines.append("return 0; }")
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines))
    exe = tmp_path / "layout"
    subprocess.check_call(["gcc", "-std=c99", "-I", os.path.dirname(HEADER), "-o", str(exe),
                           str(src)])
    out = subprocess.check_output([str(exe)], text=True).split("\n")
    got = {tuple(l.split()[:2]): int(l.split()[2]) for l in out if l.strip()}
    for name in STRUCTS:
        cls = getattr(m, name)
        assert got[(name, "size")] == ctypes.sizeof(cls), name
        for field, _ in cls._fields_:
            assert got[(name, field)] == getattr(cls, field).offset, (name, field)


# Every argument check of the two create calls runs before any CUDA call, so
# each refusal is exercised here without a GPU: (mutation, words of the
# message).  Each mutation turns one valid input into an invalid one.
def _grid(nx, ny, nz):
    atm, _ = synth.stratified_two_level(nx, ny, nz, eps=1e-3)
    return atm


TWO_LEVEL_REFUSALS = [
    (dict(params=dict(n_grids=0)), "n_grids"),
    (dict(params=dict(n_grids=99)), "n_grids"),
    (dict(params=dict(nu1=-1)), "negative iteration"),
    (dict(params=dict(nu_fmg=-2)), "negative iteration"),
    (dict(params=dict(restriction=3)), "restriction"),
    (dict(params=dict(interpolation=2)), "interpolation"),
    (dict(params=dict(sc_interp=-1)), "sc_interp"),
    (dict(atom=dict(gamma_prd=1.5)), "gamma_prd"),
    (dict(atom=dict(gamma_prd=float("nan"))), "gamma_prd"),
    (dict(atom=dict(a_damp=1e3)), "a_damp"),
    (dict(atom=dict(gamma_prd=0.5), params=dict(sc_interp=1)), "partial redistribution"),
    (dict(atom=dict(n_freq=0)), "bad atom"),
    (dict(atom=dict(n_freq=4097)), "bad atom"),
    (dict(atom=dict(x_max=-1.0)), "bad atom"),
    (dict(atom=dict(a_ul=0.0)), "bad atom"),
    (dict(atom=dict(g_ratio=-1.0)), "bad atom"),
    (dict(atom=dict(theta=0.0)), "bad atom"),
    (dict(atom=dict(kappa=float("nan"))), "bad atom"),
    (dict(atm=dict(nz=1, z=np.zeros(1))), "grid too small"),
    (dict(atm=dict(dx=0.0)), "dx, dy"),
    (dict(atm=dict(dy=-1.0)), "dx, dy"),
    (dict(atm="wide"), "below 65536"),
    (dict(atm="moving", params=dict(sc_interp=1)), "linear upwind"),
]


@pytest.mark.parametrize("mut,words", TWO_LEVEL_REFUSALS)
def test_create_refuses_each_bad_argument(lib, mut, words):
    import dataclasses
    atm, atom = synth.stratified_two_level(8, 8, 17, eps=1e-3)
    if mut.get("atm") == "wide":
        atm = _grid(65536, 1, 3)
    elif mut.get("atm") == "moving":
        atm, _ = synth.stratified_two_level(8, 8, 17, eps=1e-3, velocity=1.0)
    elif "atm" in mut:
        atm = dataclasses.replace(atm, **mut["atm"])
    atom = dataclasses.replace(atom, **mut.get("atom", {}))
    with pytest.raises(m.MG3DError) as ei:
        m.mg3d_create(atm, atom, **mut.get("params", {}))
    assert ei.value.code == m.MG3D_E_ARG
    assert words in m.mg3d_last_error()


def _ml_inputs():
    atom = synth.hydrogen_like_atom(line_freq=5, cont_freq=3)
    return synth.chromosphere(8, 8, 17, atom), atom


def _bad_line(i, **kw):
    def mutate(atom):
        import dataclasses
        atom.lines[i] = dataclasses.replace(atom.lines[i], **kw)
    return mutate


def _bad_cont(i, **kw):
    def mutate(atom):
        import dataclasses
        atom.continua[i] = dataclasses.replace(atom.continua[i], **kw)
    return mutate


def _set(**kw):
    def mutate(atom):
        for k, v in kw.items():
            setattr(atom, k, v)
    return mutate


ML_REFUSALS = [
    (_bad_line(0, lower=1, upper=1), "bad line 0"),
    (_bad_line(1, upper=9), "bad line 1"),
    (_bad_line(2, n_freq=0), "bad line 2"),
    (_bad_line(0, rho=0.0), "bad line 0"),
    (_bad_line(0, a_ul=-1.0), "bad line 0"),
    (_bad_line(0, kappa=-1.0), "bad line 0"),
    (_bad_line(0, x_max=float("nan")), "bad line 0"),
    (_bad_cont(0, lower=5), "bad continuum 0"),
    (_bad_cont(1, y_max=0.5), "bad continuum 1"),
    (_bad_cont(0, n_freq=0), "bad continuum 0"),
    (_bad_cont(0, beta=-1.0), "bad continuum 0"),
    (_bad_line(0, n_freq=70000), "too many frequencies"),
    (_set(theta_ref=0.0), "theta_ref"),
    (_set(t_ref=-1.0), "t_ref"),
    (_set(lines=[], continua=[]), "no transitions"),
    (_bad_line(0, gamma_prd=1.5), "gamma_prd must lie in [0, 1]"),
    (_bad_line(0, gamma_prd=float("nan")), "gamma_prd must lie in [0, 1]"),
    (_bad_line(0, gamma_prd=0.5, n_freq=200), "partial redistribution takes at most"),
]


def test_create_ml_refuses_prd_with_hermite_or_a_flow(lib):
    """Partial redistribution of multi-level lines is built for static
    atmospheres with the linear upwind interpolation; the other combinations
    are refused before any CUDA call."""
    atm, atom = _ml_inputs()
    atom.lines[0].gamma_prd = 0.5
    with pytest.raises(m.MG3DError) as ei:
        m.mg3d_create_ml(atm, atom, n_grids=1, sc_interp=1)
    assert ei.value.code == m.MG3D_E_ARG and "static atmosphere" in m.mg3d_last_error()
    atm.vel = np.zeros((3,) + atm.shape)
    with pytest.raises(m.MG3DError) as ei:
        m.mg3d_create_ml(atm, atom, n_grids=1)
    assert ei.value.code == m.MG3D_E_ARG and "static atmosphere" in m.mg3d_last_error()


@pytest.mark.parametrize("mutate,words", ML_REFUSALS)
def test_create_ml_refuses_each_bad_argument(lib, mutate, words):
    atm, atom = _ml_inputs()
    mutate(atom)
    with pytest.raises(m.MG3DError) as ei:
        m.mg3d_create_ml(atm, atom, n_grids=1)
    assert ei.value.code == m.MG3D_E_ARG
    assert words in m.mg3d_last_error()


def test_create_ml_refuses_bad_levels_grids_and_options(lib):
    import dataclasses
    atm, atom = _ml_inputs()
    for kw, words in ((dict(n_grids=0), "n_grids"), (dict(fs_prec=7), "fs_prec"),
                      (dict(nu3=-1), "negative iteration"), (dict(restriction=5), "restriction"),
                      (dict(interpolation=-1), "interpolation"), (dict(sc_interp=3), "sc_interp")):
        with pytest.raises(m.MG3DError) as ei:
            m.mg3d_create_ml(atm, atom, **kw)
        assert ei.value.code == m.MG3D_E_ARG and words in m.mg3d_last_error(), kw
    vatm = synth.chromosphere(8, 8, 17, atom, velocity=1.0)
    with pytest.raises(m.MG3DError):
        m.mg3d_create_ml(vatm, atom, n_grids=1, sc_interp=1)
    assert "linear upwind" in m.mg3d_last_error()
    for bad_atm, words in ((dataclasses.replace(atm, dx=0.0), "dx, dy"),
                           (dataclasses.replace(atm, nz=1, z=atm.z[:1]), "grid too small"),
                           (dataclasses.replace(atm, z=atm.z[::-1].copy()), "z must increase")):
        with pytest.raises(m.MG3DError) as ei:
            m.mg3d_create_ml(bad_atm, atom, n_grids=1)
        assert ei.value.code == m.MG3D_E_ARG and words in m.mg3d_last_error()
    with pytest.raises(m.MG3DError) as ei:
        m.mg3d_create_ml(atm, atom, n_grids=5)      # 8 nodes coarsen three times at most
    assert ei.value.code == m.MG3D_E_GRID
    # more than eight levels
    big = synth.hydrogen_like_atom(n_bound=8, line_freq=3, cont_freq=2)
    with pytest.raises(m.MG3DError) as ei:
        m.mg3d_create_ml(synth.chromosphere(8, 8, 17, big), big, n_grids=1)
    assert ei.value.code == m.MG3D_E_ARG and "n_levels" in m.mg3d_last_error()


def test_oracle_and_library_share_no_code():
    """The product package never imports, includes or loads the oracle, and
    the oracle never imports the package (inputs reach it as arguments);
    bench.py reaches the oracle only inside its CPU-baseline and reference
    functions."""
    import ast
    pkg = os.path.join(B.ROOT, "paper_1701_01607_gb300")
    for root, _, files in os.walk(pkg):
        if "_build" in root or "__pycache__" in root:
            continue
        for f in files:
            path = os.path.join(root, f)
            with open(path, encoding="utf-8", errors="replace") as fh:
                src = fh.read()
            if f.endswith(".py"):
                for node in ast.walk(ast.parse(src)):
                    if isinstance(node, (ast.Import, ast.ImportFrom)):
                        mods = [a.name for a in node.names] if isinstance(node, ast.Import) \
                            else [node.module or ""]
                        assert not any(mo.split(".")[0] == "oracle" for mo in mods), path
            elif f.endswith((".cu", ".cuh", ".h", ".cpp", ".c")):
                assert not re.search(r'#include\s*[<"][^>"]*oracle', src), path
                assert "liboracle" not in src, path
    for f in os.listdir(os.path.join(B.ROOT, "oracle")):
        if f.endswith((".py", ".c", ".h")):
            with open(os.path.join(B.ROOT, "oracle", f)) as fh:
                src = fh.read()
            assert "paper_1701_01607_gb300" not in src.split('"""', 2)[-1], f
            assert "libmg3d" not in src and "mg3d.h" not in src, f
    with open(os.path.join(B.ROOT, "bench.py")) as fh:
        tree = ast.parse(fh.read())
    users = set()
    for fn in ast.walk(tree):
        if isinstance(fn, ast.FunctionDef):
            for node in ast.walk(fn):
                if isinstance(node, ast.ImportFrom) and (node.module or "").startswith("oracle"):
                    users.add(fn.name)
    top = [n for n in tree.body if isinstance(n, (ast.Import, ast.ImportFrom))]
    assert not any(isinstance(n, ast.ImportFrom) and (n.module or "").startswith("oracle")
                   for n in top)
    assert users and all("cpu" in u or "reference" in u for u in users), users


def test_binding_fails_loudly_without_the_library(monkeypatch, tmp_path):
    """No fallback: with the library absent every entry point raises before
    computing anything."""
    monkeypatch.setattr(m, "_lib", None)
    monkeypatch.setattr(m, "library_path", lambda: str(tmp_path / "libmg3d.so"))
    with pytest.raises(RuntimeError, match="not built"):
        m.load()
    atm, atom = synth.stratified_two_level(8, 8, 17, eps=1e-3)
    with pytest.raises(RuntimeError, match="not built"):
        m.mg3d_create(atm, atom, n_grids=1)
    with pytest.raises(RuntimeError, match="not built"):
        m.mg3d_check_voigt(0.1, np.zeros(3))
