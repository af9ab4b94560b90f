"""Batched lockstep solves against the same problems solved one by one.

A batch mixes two-level atmospheres of different sizes and a multi-level
atmosphere; after batched V-cycles (and in batched FAS and FMG solves) each
member must equal its own solve through the single-problem path, which the
parity tests tie to the oracle.
"""

import numpy as np
import pytest

from paper_1701_01607_gb300 import mg3d as m
from paper_1701_01607_gb300 import synth

pytestmark = pytest.mark.gpu

P2 = dict(nu_fmg=8, nu0=10, nu1=2, nu2=4, nu3=16)


def rel(a, b):
    return float(np.max(np.abs(a - b) / np.abs(b)))


def problems():
    a1 = synth.stratified_two_level(16, 16, 33, eps=1e-3, sigma=0.3, seed=31)
    a2 = synth.stratified_two_level(32, 16, 17, eps=1e-2, sigma=0.2, seed=32)
    atom = synth.hydrogen_like_atom(line_freq=7, cont_freq=4, seed=2)
    a3 = (synth.chromosphere(8, 8, 17, atom, seed=2), atom)
    return [("two", a1), ("two", a2), ("ml", a3)]


def create(kind, pr, prec):
    atm, atom = pr
    if kind == "two":
        return m.mg3d_create(atm, atom, n_grids=3, fs_prec=prec, **P2)
    return m.mg3d_create_ml(atm, atom, n_grids=3, fs_prec=prec, **P2)


@pytest.mark.parametrize("prec", [m.MG3D_PREC_F64, m.MG3D_PREC_F32])
def test_batched_vcycles_equal_single_solves(prec):
    m.load(build_if_missing=True)
    probs = problems()
    members = [create(k, p, prec) for k, p in probs]
    singles = [create(k, p, prec) for k, p in probs]
    b = m.mg3d_batch_create(members)
    try:
        # The batched sweep is a separate kernel: the compiler may fuse its
        # multiply-adds differently, so the two sides agree to rounding, not
        # bitwise.  C is a relative difference of populations, so it carries
        # their rounding in absolute terms: ~1e-15 in FP64, ~1e-7 with the
        # FP32 formal solution.
        c_abs = 0.0 if prec == m.MG3D_PREC_F64 else 1e-7
        for cyc in range(3):
            cb = m.mg3d_batch_fas_vcycle(b, len(members), cyc == 0)
            cs = [m.mg3d_fas_vcycle(h, cyc == 0) for h in singles]
            for i in range(len(members)):
                if cs[i] > 1e-8:
                    assert abs(cb[i] - cs[i]) <= 1e-6 * cs[i] + c_abs, (cyc, i)
        tol = 1e-10 if prec == m.MG3D_PREC_F64 else 1e-5
        for i in range(len(members)):
            assert rel(m.mg3d_get_populations(members[i], 3),
                       m.mg3d_get_populations(singles[i], 3)) < tol, i
        cnt = m.mg3d_batch_counters(b)
        assert cnt["kernel_launches"] > 0 and cnt["fs_units"] > 0
    finally:
        m.mg3d_batch_destroy(b)
        for h in members + singles:
            m.mg3d_destroy(h)


def test_batched_fas_and_fmg_solves():
    m.load(build_if_missing=True)
    probs = problems()
    members = [create(k, p, m.MG3D_PREC_F64) for k, p in probs]
    b = m.mg3d_batch_create(members)
    try:
        st = m.mg3d_batch_fas_solve(b, len(members), 1e-6, n_grids=3)
        n_fas = [m.mg3d_get_populations(h, 3) for h in members]
        st2 = m.mg3d_batch_fmg_solve(b, len(members), 1e-6, n_grids=3)
        n_fmg = [m.mg3d_get_populations(h, 3) for h in members]
    finally:
        m.mg3d_batch_destroy(b)
        for h in members:
            m.mg3d_destroy(h)
    # lockstep: members that met tol early keep cycling until the last one does
    total_fas = max(x["iterations"] for x in st)
    total_fmg = max(x["iterations"] for x in st2)
    for i, (kind, pr) in enumerate(probs):
        h = create(kind, pr, m.MG3D_PREC_F64)
        try:
            s1 = m.mg3d_fas_solve(h, 1e-6, n_grids=3)
            assert s1["iterations"] == st[i]["iterations"], i
            for _ in range(total_fas - s1["iterations"]):
                m.mg3d_fas_vcycle(h, False)
            assert rel(n_fas[i], m.mg3d_get_populations(h, 3)) < 1e-9
            s2 = m.mg3d_fmg_solve(h, 1e-6, n_grids=3)
            assert s2["iterations"] == st2[i]["iterations"], i
            for _ in range(total_fmg - s2["iterations"]):
                m.mg3d_fas_vcycle(h, False)
            assert rel(n_fmg[i], m.mg3d_get_populations(h, 3)) < 1e-9
        finally:
            m.mg3d_destroy(h)


def test_batched_multi_level_members_in_chunks():
    """Multi-level members whose formal solutions run in chunks of different
    sizes (so in different numbers of batched launches) next to a two-level
    member: batched V-cycles equal the members' unchunked single solves."""
    m.load(build_if_missing=True)
    atom = synth.hydrogen_like_atom(line_freq=7, cont_freq=4, seed=2)
    probs = [("ml", (synth.chromosphere(8, 8, 17, atom, seed=2), atom)),
             ("ml", (synth.chromosphere(16, 8, 17, atom, seed=5), atom)),
             ("two", synth.stratified_two_level(16, 16, 33, eps=1e-3, sigma=0.3, seed=31))]
    members = [create(k, p, m.MG3D_PREC_F64) for k, p in probs]
    singles = [create(k, p, m.MG3D_PREC_F64) for k, p in probs]
    m.mg3d_set_ml_chunk(members[0], 9)
    m.mg3d_set_ml_chunk(members[1], 20)
    b = m.mg3d_batch_create(members)
    try:
        for cyc in range(3):
            cb = m.mg3d_batch_fas_vcycle(b, len(members), cyc == 0)
            cs = [m.mg3d_fas_vcycle(h, cyc == 0) for h in singles]
            for i in range(len(members)):
                if cs[i] > 1e-8:
                    assert abs(cb[i] - cs[i]) <= 1e-6 * cs[i], (cyc, i)
        for i in range(len(members)):
            assert rel(m.mg3d_get_populations(members[i], 3),
                       m.mg3d_get_populations(singles[i], 3)) < 1e-10, i
    finally:
        m.mg3d_batch_destroy(b)
        for h in members + singles:
            m.mg3d_destroy(h)
