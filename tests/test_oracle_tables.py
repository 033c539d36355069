"""Pins of the oracle's velocity sets and force stencils.

The isotropic force stencils are re-derived here from scratch, in exact rational
arithmetic, as the unique solution of the isotropy conditions behind Eq. 2
(sum_a w_a e_ai e_aj ... isotropic up to the stated rank) with sum_a w_a e_ax^2 = 1.
The oracle's tables are then compared with the derived values, and the lattices
with Table 1 of the paper.
"""
import itertools
import json
import os
from fractions import Fraction as Fr

import numpy as np
import pytest

import oracle

GOLD = os.path.join(os.path.dirname(__file__), "golden")


def dfact(n):
    """(n)!! with (-1)!! = 1."""
    r = 1
    while n > 1:
        r *= n
        n -= 2
    return r


def shell_vectors(dim, sq):
    rng = range(-4, 5)
    vs = []
    for v in itertools.product(rng, repeat=dim):
        if sum(x * x for x in v) == sq:
            vs.append(v)
    return vs


def even_multi_indices(dim, n):
    out = []
    for idx in itertools.product(range(0, n + 1, 2), repeat=dim):
        if sum(idx) == n:
            out.append(idx)
    return out


def solve_exact(rows, rhs):
    """Gauss-Jordan over Fractions. Returns the unique solution or raises."""
    m = [list(r) + [b] for r, b in zip(rows, rhs)]
    ncol = len(rows[0])
    piv_row = 0
    pivots = []
    for col in range(ncol):
        p = next((r for r in range(piv_row, len(m)) if m[r][col] != 0), None)
        if p is None:
            raise ValueError("singular: solution not unique")
        m[piv_row], m[p] = m[p], m[piv_row]
        pv = m[piv_row][col]
        m[piv_row] = [x / pv for x in m[piv_row]]
        for r in range(len(m)):
            if r != piv_row and m[r][col] != 0:
                f = m[r][col]
                m[r] = [a - f * b for a, b in zip(m[r], m[piv_row])]
        pivots.append(col)
        piv_row += 1
    for r in range(piv_row, len(m)):
        if m[r][-1] != 0:
            raise ValueError("inconsistent isotropy system")
    return [m[i][-1] for i in range(ncol)]


def derive_stencil(dim, shells, order):
    """Unit-normalised shell weights making sum w e^(n) isotropic for n <= order.

    Unknowns: one weight per shell and the isotropic coefficients e_4..e_order.
    Equations: for every even multi-index (a, b[, c]) of rank n,
    sum_a w e_x^a e_y^b e_z^c = e_n (a-1)!!(b-1)!!(c-1)!!, with e_2 = 1."""
    vecs = {sq: shell_vectors(dim, sq) for sq in shells}
    ranks = list(range(4, order + 1, 2))
    nunk = len(shells) + len(ranks)
    rows, rhs = [], []
    for n in [2] + ranks:
        for idx in even_multi_indices(dim, n):
            row = [Fr(0)] * nunk
            for k, sq in enumerate(shells):
                s = 0
                for v in vecs[sq]:
                    t = 1
                    for comp, p in zip(v, idx):
                        t *= comp ** p
                    s += t
                row[k] = Fr(s)
            coef = 1
            for p in idx:
                coef *= dfact(p - 1)
            if n == 2:
                rows.append(row)
                rhs.append(Fr(coef))
            else:
                row[len(shells) + ranks.index(n)] = Fr(-coef)
                rows.append(row)
                rhs.append(Fr(0))
    sol = solve_exact(rows, rhs)
    w = dict(zip(shells, sol[: len(shells)]))
    e = {2: Fr(1)}
    e.update(dict(zip(ranks, sol[len(shells):])))
    return w, e


STENCILS = [
    (2, 4, [1, 2]),
    (2, 6, [1, 2, 4]),
    (2, 8, [1, 2, 4, 5, 8]),
    (2, 10, [1, 2, 4, 5, 8, 9, 10]),
    (3, 4, [1, 2]),
    (3, 6, [1, 2, 3, 4]),
]


def moment(e, w, idx):
    return sum(wa * np.prod([float(comp) ** p for comp, p in zip(ea, idx)]) for ea, wa in zip(e, w))


@pytest.mark.parametrize("dim,order,shells", STENCILS)
def test_force_stencil_matches_exact_isotropy_solution(dim, order, shells):
    w_exact, _ = derive_stencil(dim, shells, order)
    e, w = oracle.stencil_table(dim, order)
    sq = (e ** 2).sum(axis=1)
    assert sorted(set(sq.tolist())) == shells
    for s in shells:
        n_expected = len(shell_vectors(dim, s))
        assert (sq == s).sum() == n_expected, "every vector of the shell present once"
        np.testing.assert_allclose(w[sq == s], float(w_exact[s]), rtol=2e-16, atol=0)
    # opposite pairs adjacent and no duplicates
    for a in range(0, len(e), 2):
        assert (e[a] == -e[a + 1]).all()
    assert len({tuple(v) for v in e.tolist()}) == len(e)


@pytest.mark.parametrize("dim,order,shells", STENCILS)
def test_force_stencil_isotropic_to_order_and_not_beyond(dim, order, shells):
    w_exact, e_coef = derive_stencil(dim, shells, order)
    e, w = oracle.stencil_table(dim, order)
    ecols = [e[:, i] for i in range(dim)]
    for n in range(2, order + 1, 2):
        for idx in even_multi_indices(dim, n):
            coef = float(e_coef[n]) * np.prod([dfact(p - 1) for p in idx])
            assert moment(e[:, :dim], w, idx) == pytest.approx(coef, rel=1e-14, abs=1e-15)
    # odd moments vanish
    for n in (1, 3, 5):
        for idx in itertools.product(range(n + 1), repeat=dim):
            if sum(idx) == n:
                assert abs(moment(e[:, :dim], w, idx)) < 1e-15
    # the next even rank is NOT isotropic (the stencil is exactly of this order)
    n = order + 2
    vals = []
    for idx in even_multi_indices(dim, n):
        vals.append(moment(e[:, :dim], w, idx) / np.prod([dfact(p - 1) for p in idx]))
    assert max(vals) - min(vals) > 1e-6
    del ecols


def load_table1():
    with open(os.path.join(GOLD, "table1_lattices.json")) as fh:
        return json.load(fh)


LATTICES = {"D2Q9": oracle.D2Q9, "D2Q13": oracle.D2Q13, "D2Q25": oracle.D2Q25}


@pytest.mark.parametrize("name", ["D2Q9", "D2Q13", "D2Q25"])
def test_lattices_match_table1(name):
    t1 = load_table1()[name]
    c, w, cs2 = oracle.lattice_table(LATTICES[name])
    assert cs2 == pytest.approx(float(Fr(t1["cs2"])), rel=1e-16)
    sq = (c ** 2).sum(axis=1)
    assert sorted(set(sq.tolist())) == sorted(int(k) for k in t1["w"])
    for k, v in t1["w"].items():
        assert (sq == int(k)).sum() == len(shell_vectors(2, int(k)))
        np.testing.assert_allclose(w[sq == int(k)], float(Fr(v)), rtol=2e-16)
    assert w.sum() == pytest.approx(1.0, abs=1e-15)
    assert len(c) == {"D2Q9": 9, "D2Q13": 13, "D2Q25": 25}[name]


@pytest.mark.parametrize("name", ["D2Q9", "D2Q13", "D2Q25"])
def test_second_isotropy_order_of_lattice(name):
    """Sec. 3: sum_b w_b c_b...c_b isotropic to 4th/6th/8th order, with e_2 = c_s^2
    (read per component), and not isotropic at the next even rank."""
    t1 = load_table1()
    order = t1["second_isotropy_order"][name]
    c, w, cs2 = oracle.lattice_table(LATTICES[name])
    c = c[:, :2]
    e2 = moment(c, w, (2, 0))
    assert e2 == pytest.approx(cs2, rel=1e-15)
    for n in range(4, order + 1, 2):
        vals = [moment(c, w, idx) / np.prod([dfact(p - 1) for p in idx])
                for idx in even_multi_indices(2, n)]
        assert max(vals) - min(vals) < 1e-15
    vals = [moment(c, w, idx) / np.prod([dfact(p - 1) for p in idx])
            for idx in even_multi_indices(2, order + 2)]
    assert max(vals) - min(vals) > 1e-6


def test_table1_equals_cs2_times_derived_stencils():
    """Table 1 re-derived: D2Q9 = 1/3 E4, D2Q13 = 2/5 E6, D2Q25 = 4/7 E8 on the
    moving shells, the rest weight closing sum w = 1.  This ties the printed
    weights to the exact isotropy solution (and so to the reading that force
    weights scale with the lattice's c_s^2)."""
    t1 = load_table1()
    for name, order, shells in (("D2Q9", 4, [1, 2]), ("D2Q13", 6, [1, 2, 4]),
                                ("D2Q25", 8, [1, 2, 4, 5, 8])):
        w_exact, _ = derive_stencil(2, shells, order)
        cs2 = Fr(t1[name]["cs2"])
        for s in shells:
            assert cs2 * w_exact[s] == Fr(t1[name]["w"][str(s)])
        rest = 1 - sum(cs2 * w_exact[s] * len(shell_vectors(2, s)) for s in shells)
        assert rest == Fr(t1[name]["w"]["0"])


def test_d3q19_table():
    c, w, cs2 = oracle.lattice_table(oracle.D3Q19)
    assert len(c) == 19 and cs2 == pytest.approx(1 / 3)
    w_exact, _ = derive_stencil(3, [1, 2], 4)
    sq = (c ** 2).sum(axis=1)
    for s in (1, 2):
        np.testing.assert_allclose(w[sq == s], float(Fr(1, 3) * w_exact[s]), rtol=2e-16)
    assert w.sum() == pytest.approx(1.0, abs=1e-15)


def test_velocity_order_convention():
    """Rest first, shells by |c|^2, opposite pairs adjacent (shared convention)."""
    for lat in (oracle.D2Q9, oracle.D3Q19, oracle.D2Q13, oracle.D2Q25):
        c, _, _ = oracle.lattice_table(lat)
        assert (c[0] == 0).all()
        sq = (c ** 2).sum(axis=1)
        assert (np.diff(sq) >= 0).all()
        for b in range(1, len(c), 2):
            assert (c[b] == -c[b + 1]).all()
    c, _, _ = oracle.lattice_table(oracle.D2Q9)
    assert c[:, :2].tolist() == [[0, 0], [1, 0], [-1, 0], [0, 1], [0, -1],
                                 [1, 1], [-1, -1], [1, -1], [-1, 1]]


def test_equal_viscosity_relaxation_times():
    """Sec. 3: nu = c_s^2 (tau - 1/2) equal for D2Q9 tau=1, D2Q13 11/12, D2Q25 19/24."""
    with open(os.path.join(GOLD, "paper_claims.json")) as fh:
        claims = json.load(fh)["tau_equal_viscosity"]
    t1 = load_table1()
    nus = {n: Fr(t1[n]["cs2"]) * (Fr(claims[n]) - Fr(1, 2)) for n in ("D2Q9", "D2Q13", "D2Q25")}
    assert len(set(nus.values())) == 1 and nus["D2Q9"] == Fr(1, 6)
