"""Pins for the oracle's tree, balance, Morton order and faces (Sec. 2.1).

Checked against brute force on tiny trees: pairwise box tests for 2:1 balance
across faces, edges and corners, exact tiling, Morton order decoded bit by bit,
minimality of the balanced refinement, and pairwise face enumeration.
"""
import itertools
from fractions import Fraction

import numpy as np
import pytest

import oracle as O
from tests import brute

SMALL_SPECS = [
    # (dim, base, max, pred, c, r, beta, solid, bc)
    (2, 2, 5, O.PRED_BALL, (0.3, 0.6, 0.5), 0.05, 0.0, 0, (0,) * 6),
    (2, 1, 5, O.PRED_SHELL, (0.5, 0.5, 0.5), 0.3, 0.5, 1, (1, 2, 2, 2, 0, 0)),
    (2, 2, 5, O.PRED_BALL, (0.0, 0.0, 0.5), 0.1, 0.0, 0, (0,) * 6),  # refined across the periodic corner
    (3, 1, 4, O.PRED_BALL, (0.3, 0.6, 0.7), 0.05, 0.0, 0, (0,) * 6),
    (3, 2, 4, O.PRED_SHELL, (0.5, 0.5, 0.5), 0.15, 0.3, 1, (1, 2, 2, 2, 2, 2)),
    (3, 1, 4, O.PRED_BALL, (0.97, 0.02, 0.5), 0.05, 0.0, 0, (0, 0, 2, 2, 0, 0)),
]


def spec_of(t):
    return O.make_spec(*t[:4], c=t[4], r=t[5], beta=t[6], solid=t[7], bc=t[8])


@pytest.mark.parametrize("t", SMALL_SPECS)
def test_tiling_morton_and_balance_bruteforce(t):
    dim, L = t[0], t[2]
    keys, lev, sol = O.build_tree(spec_of(t))
    assert 8 < len(keys) <= 1200
    # exact tiling: volumes add to the domain, Morton ranges are contiguous
    tot, dom = brute.volume_sum(lev, dim, L)
    assert tot == dom
    nxt = 0
    for k, l in zip(keys, lev):
        assert int(k) == nxt
        nxt += 1 << (dim * (L - int(l)))
    assert nxt == 1 << (dim * L)
    # anchors decoded bit by bit are aligned to their box size
    for k, l in zip(keys, lev):
        a = brute.decode(k, dim, L)
        for d in range(dim):
            assert a[d] % (1 << (L - int(l))) == 0
    periodic = [t[8][2 * d] == 0 for d in range(dim)]
    assert brute.balance_violations(keys, lev, dim, L, periodic) == []


def _pred(t, lev, a_int, L):
    """Refinement predicate restated with exact rationals (independent of FP)."""
    dim, pred, c, r, beta = t[0], t[3], t[4], t[5], t[6]
    h = Fraction(1, 1 << lev)
    lo = [Fraction(a_int[d], 1 << L) for d in range(dim)]
    cc = [Fraction(c[d]) for d in range(dim)]
    dmin2 = sum(max(lo[d] - cc[d], Fraction(0), cc[d] - lo[d] - h) ** 2 for d in range(dim))
    dmax2 = sum(max(abs(lo[d] - cc[d]), abs(lo[d] + h - cc[d])) ** 2 for d in range(dim))
    R = Fraction(r)
    if pred == O.PRED_BALL:
        return dmin2 <= R * R
    rp, rm = R + Fraction(beta) * h, R - Fraction(beta) * h
    return dmin2 <= rp * rp and (rm <= 0 or dmax2 >= rm * rm)


@pytest.mark.parametrize("t", SMALL_SPECS)
def test_refinement_fixpoint_and_minimality(t):
    """Every leaf below max level fails the predicate; every complete sibling
    group is needed (its parent satisfies the predicate or would break 2:1)."""
    dim, L, top = t[0], t[2], t[2]
    keys, lev, sol = O.build_tree(spec_of(t))
    bx = brute.boxes(keys, lev, dim, L)
    for (a, s), l in zip(bx, lev):
        if int(l) < top:
            assert not _pred(t, int(l), a, L)
    # sibling groups
    groups = {}
    for i, ((a, s), l) in enumerate(zip(bx, lev)):
        ps = s * 2
        pa = tuple(a[d] - a[d] % ps for d in range(dim))
        groups.setdefault((int(l) - 1, pa), []).append(i)
    periodic = [t[8][2 * d] == 0 for d in range(dim)]
    N = 1 << L
    for (pl, pa), members in groups.items():
        if len(members) != 1 << dim or pl < t[1]:
            continue
        if _pred(t, pl, list(pa), L):
            continue
        parent = (list(pa), 1 << (L - pl))
        forced = any(int(lev[j]) > pl + 1 and brute.touching(parent, bx[j], dim, N, periodic)
                     for j in range(len(bx)) if j not in members)
        assert forced, "sibling group at level %d could be merged" % (pl + 1)


@pytest.mark.parametrize("t", SMALL_SPECS)
def test_faces_bruteforce(t):
    dim, L = t[0], t[2]
    p = O.Problem(spec_of(t), (4, 4, 4), (-1, -1, -1), (1, 1, 1))
    keys, lev, sol = p.leaves()
    m, pl, ax, ar = p.faces()
    got = sorted((int(a), int(b), int(c), Fraction(float(d))) for a, b, c, d in zip(m, pl, ax, ar))
    inter, bnd = brute.faces(keys, lev, sol, dim, L, t[8])
    assert got == sorted(inter)
    bl, bax, bside, bkind, bother, bar = p.bfaces()
    gotb = sorted((int(a), int(b), int(c), int(d), int(e), Fraction(float(f)))
                  for a, b, c, d, e, f in zip(bl, bax, bside, bkind, bother, bar))
    assert gotb == sorted(bnd)
    # canonical order: interior by (axis, key(minus), key(plus))
    order = [(int(ax[q]), int(keys[m[q]]), int(keys[pl[q]])) for q in range(len(m))]
    assert order == sorted(order)
    border = [(int(bkind[q]), int(bax[q]), int(bside[q]), int(keys[bl[q]]),
               int(keys[bother[q]]) if bother[q] >= 0 else 0) for q in range(len(bl))]
    assert border == sorted(border)


def test_every_cell_side_is_covered():
    """Each fluid cell side is tiled by its faces: areas add up to h^(dim-1)."""
    t = SMALL_SPECS[4]
    p = O.Problem(spec_of(t), (4, 4, 4), (-1, -1, -1), (1, 1, 1))
    keys, lev, sol = p.leaves()
    dim = t[0]
    cover = {}
    m, pl, ax, ar = p.faces()
    for a, b, d, A in zip(m, pl, ax, ar):
        cover[(int(a), int(d), 1)] = cover.get((int(a), int(d), 1), 0.0) + A
        cover[(int(b), int(d), 0)] = cover.get((int(b), int(d), 0), 0.0) + A
    bl, bax, bside, bkind, bother, bar = p.bfaces()
    for a, d, s, A in zip(bl, bax, bside, bar):
        cover[(int(a), int(d), int(s))] = cover.get((int(a), int(d), int(s)), 0.0) + A
    for i in range(len(keys)):
        if sol[i]:
            continue
        for d, s in itertools.product(range(dim), (0, 1)):
            assert cover[(i, d, s)] == 2.0 ** (-int(lev[i]) * (dim - 1))


def test_config_trees_sizes():
    import workloads as W
    c = W.CONFIGS["c1_2d_bump"]
    s = O.make_spec(c["dim"], c["base_level"], c["max_level"], c["pred"], c["c"], c["r"],
                    c["beta"], c["solid"], c["bc"])
    keys, lev, sol = O.build_tree(s)
    assert len(keys) == 904
    assert np.all(np.diff(keys.astype(np.int64)) > 0)
