"""Generator pins for the oracle's diagram enumeration and derived rules:
Table I counts (golden), hole-number distributions, anomalous and mirror
structure, and the third-order prefactors of Eqs. (3)-(5)."""
import collections

import numpy as np
import pytest

import oracle as O
from conftest import golden_rows


@pytest.mark.parametrize("n", [2, 3, 4, 5, 6])
def test_table1_counts(n):
    want = {int(r[0]): int(r[1]) for r in golden_rows("table1_counts.txt")}
    assert len(O.enumerate_diagrams(n)) == want[n]


@pytest.mark.parametrize("n", [2, 3, 4, 5, 6])
def test_table1_group_counts(n):
    """Grouping by the number of hole loop momenta (the particle-hole composition of the integration
    domain) reproduces Table I's N_grp column, anomalous diagrams included or not."""
    want = {int(r[0]): int(r[1]) for r in golden_rows("table1_groups.txt")}
    assert len({O.hole_chords(D) for D in O.enumerate_diagrams(n)}) == want[n]
    assert len(O.groups(n)) == want[n]


def test_hole_distribution_and_ladders():
    h4 = collections.Counter(D.h for D in O.enumerate_diagrams(4))
    assert dict(h4) == {2: 1, 3: 7, 4: 23, 5: 7, 6: 1}
    h5 = collections.Counter(D.h for D in O.enumerate_diagrams(5))
    assert dict(h5) == {2: 1, 3: 21, 4: 207, 5: 382, 6: 207, 7: 21, 8: 1}
    # sixth order: symmetric under h -> 2n + 2 - h (mirror), one all-pp and one all-hh ladder
    h6 = collections.Counter(D.h for D in O.enumerate_diagrams(6))
    assert dict(h6) == {2: 1, 3: 51, 4: 1194, 5: 6554, 6: 11700, 7: 6554, 8: 1194, 9: 51, 10: 1}


def test_anomalous_and_mirror_structure():
    # anomalous: a hole and a particle line forced to equal momentum
    assert sum(O.is_anomalous(D) for D in O.enumerate_diagrams(3)) == 0
    assert sum(O.is_anomalous(D) for D in O.enumerate_diagrams(4)) == 6
    assert sum(O.is_anomalous(D) for D in O.enumerate_diagrams(5)) == 172
    assert sum(O.is_anomalous(D) for D in O.enumerate_diagrams(6)) == 5728
    eff = {int(r[0]): int(r[1]) for r in golden_rows("table1_eff.txt")}
    for n, selfm, orbits in ((4, 23, 27), (5, 84, eff[5]), (6, 1046, eff[6])):
        Ds = O.enumerate_diagrams(n)
        idx = {D.A: k for k, D in enumerate(Ds)}
        assert sum(O.mirror_matrix(D.A) == D.A for D in Ds) == selfm
        # mirror of a diagram is a diagram; mirror is an involution; h is kept
        for D in Ds:
            M = O.mirror_matrix(D.A)
            assert M in idx and O.mirror_matrix(M) == D.A
            assert Ds[idx[M]].h == D.h
            assert O.is_anomalous(Ds[idx[M]]) == O.is_anomalous(D)
        orb = {min(idx[D.A], idx[O.mirror_matrix(D.A)]) for D in Ds if not O.is_anomalous(D)}
        # n = 5, 6: equal to N_diag^(eff) of Table I (375, 11269)
        assert len(orb) == orbits


def test_third_order_matches_eqs_3_to_5():
    rows = {r[0]: (float(r[1]), int(r[2]), int(r[3])) for r in golden_rows("eq3_5_third_order.txt")}
    got = {}
    for D in O.enumerate_diagrams(3):
        pref = (-1) ** (D.h + D.l0) / 2 ** D.n_eq
        nh = D.h
        npart = D.nl - D.h
        name = {4: "hh", 3: "ph", 2: "pp"}[nh]
        got[name] = (pref, nh, npart)
        for m in range(2):
            cut = D.cut_lines(m)
            assert sum(D.hole(l) for l in cut) == 2 and sum(not D.hole(l) for l in cut) == 2
    assert got == rows


def test_second_order_is_eq2():
    (D,) = O.enumerate_diagrams(2)
    assert (-1) ** (D.h + D.l0) / 2 ** D.n_eq == 0.25   # Eq. (2): 1/(4 D_ijab)
    assert D.h == 2 and len(D.cut_lines(0)) == 4


def test_momentum_conservation_rows():
    for n in (2, 3, 4, 5):
        for D in O.enumerate_diagrams(n)[:60]:
            C = D.coef()
            for v in range(n):
                s = np.zeros(n + 1, dtype=int)
                for l, (a, b) in enumerate(D.lines):
                    if b == v:
                        s += C[l]
                    if a == v:
                        s -= C[l]
                assert not s.any()
            for c, l in enumerate(D.chords):
                e = np.zeros(n + 1, dtype=int)
                e[c] = 1
                assert (C[l] == e).all()


@pytest.mark.parametrize("n", [3, 4, 5])
def test_repeated_denominators(n):
    """Diagrams with two cuts carrying the same energy denominator (a 1/D^2 factor): the symbolic
    criterion (equal quadratic forms of the cuts in the loop momenta) agrees with evaluating every
    cut's denominator at random loop momenta; 0, 4 and 124 diagrams at orders 3, 4, 5 (64 of the 124
    at fifth order are not anomalous)."""
    rng = np.random.default_rng(n)
    count = 0
    for D in O.enumerate_diagrams(n):
        C = D.coef()
        k = rng.normal(size=(D.n + 1, 3))
        lines = C @ k
        ksq = np.sum(lines ** 2, axis=1)
        Ds = []
        for m in range(D.n - 1):
            Ds.append(sum((ksq[l] if D.hole(l) else -ksq[l]) for l, (a, b) in enumerate(D.lines)
                          if min(a, b) <= m < max(a, b)))
        numeric = any(abs(Ds[a] - Ds[b]) < 1e-9 * (1 + abs(Ds[a])) for a in range(len(Ds)) for b in range(a))
        assert numeric == O.has_repeated_denominator(D), D.diagram_id
        count += numeric
    assert count == {3: 0, 4: 4, 5: 124}[n]
    if n == 5:
        assert sum(O.has_repeated_denominator(D) and not O.is_anomalous(D) for D in O.enumerate_diagrams(5)) == 64
