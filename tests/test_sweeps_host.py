"""Host logic of the Sec. IV sweep driver (paper_2511_11360_gb300/sweeps.py),
no GPU: the parameter sets are the paper's three sweeps (density ratio at
We = 1.2, xi = 6; Weber number at rho* = 2, xi = 3; interface thickness at
rho* = 2, We = 1.2), their union holds each shared point (rho* 2, We 1.2,
xi 3 or 6) once with both sweeps it belongs to; the six families of the 3D
study are run."""

from paper_2511_11360_gb300 import sweeps as S


def test_sweep_sets_are_the_papers():
    assert [s["rho"] for s in S.DENSITY] == [2.0, 10.0, 50.0, 100.0]
    assert all(s["We"] == 1.2 and s["xi"] == 6.0 for s in S.DENSITY)
    assert [s["We"] for s in S.WEBER] == [1.2, 12.0, 120.0, 600.0]
    assert all(s["rho"] == 2.0 and s["xi"] == 3.0 for s in S.WEBER)
    assert [s["xi"] for s in S.THICKNESS] == [3.0, 6.0, 9.0]
    assert all(s["rho"] == 2.0 and s["We"] == 1.2 for s in S.THICKNESS)
    assert sorted(S.FAMILIES) == sorted([S.C.FAKHARI2017, S.C.LIANG2018, S.C.CHAI2018, S.C.LIU2023,
                                          S.C.LIANG2014, S.C.BAO2024])


def test_union_of_the_sweeps():
    sets = S.sweep_sets()
    assert len(sets) == 4 + 4 + 3 - 2   # (2, 1.2, 3) and (2, 1.2, 6) are shared
    assert sorted(sets[(2.0, 1.2, 3.0)]) == ["thickness", "weber"]
    assert sorted(sets[(2.0, 1.2, 6.0)]) == ["density", "thickness"]
    for key, member in sets.items():
        assert member and len(set(member)) == len(member)

