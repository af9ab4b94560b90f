"""The bench schedule against the schedules the paper prints (Table 1,
stored in tests/golden/table1_schedules.txt with its citation)."""

import os

HERE = os.path.dirname(os.path.abspath(__file__))


def table1():
    rows = []
    with open(os.path.join(HERE, "golden", "table1_schedules.txt")) as fh:
        for line in fh:
            if line.strip() and not line.startswith("#"):
                atm, atom, method, *nus, speed = line.split()
                rows.append(dict(atmosphere=atm, atom=atom, method=method,
                                 nu=[None if v == "-" else int(v) for v in nus],
                                 speedup=None if speed == "-" else float(speed)))
    return rows


def test_fixture_has_the_four_runs():
    rows = table1()
    assert [(r["atmosphere"], r["atom"], r["method"]) for r in rows] == [
        ("model1", "3-level-CaII", "3-grid-MG"), ("model1", "3-level-CaII", "3-grid-FMG"),
        ("model1", "6-level-HI", "3-grid-MG"), ("model2", "6-level-CaII", "3-grid-MG")]
    # nu_3 = 32 coarse-grid iterations in every run
    assert all(r["nu"][4] == 32 for r in rows)


def test_bench_schedule_is_the_three_level_ca_ii_row():
    """The bench's 3-grid FAS step and its FMG leg use Model 1's 3-level Ca II
    schedule, the run whose atom is closest to the two-level bench atom."""
    import bench
    row = next(r for r in table1()
               if r["atom"] == "3-level-CaII" and r["method"] == "3-grid-FMG")
    nu_fmg, nu0, nu1, nu2, nu3 = row["nu"]
    assert bench.NU == dict(nu_fmg=nu_fmg, nu0=nu0, nu1=nu1, nu2=nu2, nu3=nu3)
    mg = next(r for r in table1()
              if r["atom"] == "3-level-CaII" and r["method"] == "3-grid-MG")
    assert mg["nu"][1:] == [nu0, nu1, nu2, nu3]
