"""Pins for the oracle's mesh adaptation with f carried over (Sec. 2.1: the
tree is refined and coarsened as the solution evolves; Sec. 3.1, step 4: the
stencils are rebuilt on every change).

Pinned against: a brute-force statement of the coarsening rule (pairwise box
contacts, one merge undone at a time), pairwise 2:1 balance and exact tiling
of the refined trees, an independent mapping of f from the leaf lists
(injection into the children; the mean over the fluid children), and exact
conservation of the totals sum_j V_j sum_i psi_r f_ij dV on all-fluid trees.
The library's host-side coarsening and refinement give the same leaf lists.
"""
import numpy as np
import pytest

import oracle as O
import paper_1503_00707_gb300 as D
from tests import brute
from tests.test_coarsen_host import CASES, _brute_coarsen


def _problem(case, n=(4, 4, 4)):
    dim, base, L, pred, r, beta, solid, bc, prob, seed = case
    spec = O.make_spec(dim, base, L, pred, (0.5, 0.5, 0.5), r, beta, solid, bc)
    p = O.Problem(spec, n, (-2.0,) * 3, (2.0,) * 3)
    rng = np.random.default_rng(seed + 100)
    p.set_f(rng.uniform(0.1, 1.0, (p.ncells, p.nv)))
    return p


def _cells(keys, lev, sol):
    fl = sol == 0
    return [(int(k), int(l)) for k, l in zip(keys[fl], lev[fl])]


def _volume_totals(p, dim):
    """sum_j V_j sum_i psi_r f_ij dV, from the cell sizes (independent of orc_totals)."""
    _, h = p.centres()
    xi = p.xi.reshape(-1, 3)
    psi = np.stack([np.ones(len(xi)), xi[:, 0], xi[:, 1], xi[:, 2], (xi * xi).sum(1)], 1)
    return ((h ** dim)[:, None] * (p.get_f() @ psi)).sum(0) * p.dV


@pytest.mark.parametrize("case", CASES)
def test_coarsen_leaves_match_brute_force(case):
    dim, base, L, pred, r, beta, solid, bc, prob, seed = case
    p = _problem(case)
    k0, l0, _ = p.leaves()
    flags = (np.random.default_rng(seed).random(len(k0)) < prob).astype(np.uint8)
    periodic = [bc[2 * d] == 0 for d in range(3)]
    want = _brute_coarsen(k0, l0, flags, dim, base, L, periodic)
    p.coarsen_project(flags)
    k1, l1, s1 = p.leaves()
    assert list(zip([int(k) for k in k1], [int(l) for l in l1])) == want
    assert brute.balance_violations(k1, l1, dim, L, periodic) == []


@pytest.mark.parametrize("case", CASES)
def test_coarsen_f_is_the_mean_of_the_fluid_children(case):
    dim, base, L, pred, r, beta, solid, bc, prob, seed = case
    p = _problem(case)
    k0, l0, s0 = p.leaves()
    c0 = _cells(k0, l0, s0)
    f0 = p.get_f()
    flags = (np.random.default_rng(seed).random(len(k0)) < prob).astype(np.uint8)
    p.coarsen_project(flags)
    k1, l1, s1 = p.leaves()
    c1 = _cells(k1, l1, s1)
    f1 = p.get_f()
    old = {kl: i for i, kl in enumerate(c0)}
    fs = np.zeros(p.nv)
    for q, (k, l) in enumerate(c1):
        if (k, l) in old:
            assert np.array_equal(f1[q], f0[old[(k, l)]])
            continue
        sh = dim * (L - l)
        inside = [i for i, (kk, ll) in enumerate(c0) if ll == l + 1 and (kk >> sh) == (k >> sh)]
        want = f0[inside].mean(axis=0) if inside else None
        if want is None:
            # every child was solid: the freestream Maxwellian (rho 1, u 0, T 1)
            xi = p.xi.reshape(-1, 3)
            want = (2 * np.pi) ** -1.5 * np.exp(-0.5 * (xi * xi).sum(1))
        assert np.max(np.abs(f1[q] - want)) <= 4e-16 * np.max(np.abs(want))


@pytest.mark.parametrize("case", [CASES[0], CASES[2]])
def test_coarsen_and_refine_keep_the_totals(case):
    """All-fluid periodic trees: a parent's volume is the sum of its children's,
    so the mean keeps mass, momentum and energy; injection keeps them too."""
    dim = case[0]
    p = _problem(case)
    t0 = _volume_totals(p, dim)
    scale = np.array([t0[0], t0[4], t0[4], t0[4], t0[4]])
    flags = (np.random.default_rng(case[-1]).random(p.nleaves) < case[-2]).astype(np.uint8)
    p.coarsen_project(flags)
    assert np.max(np.abs(_volume_totals(p, dim) - t0) / scale) < 1e-13
    _, lev, _ = p.leaves()
    p.refine_project((lev == case[1] + 1).astype(np.uint8))
    assert np.max(np.abs(_volume_totals(p, dim) - t0) / scale) < 1e-13


@pytest.mark.parametrize("case", CASES)
def test_refine_is_balanced_tiles_and_injects(case):
    dim, base, L, pred, r, beta, solid, bc, prob, seed = case
    p = _problem(case)
    k0, l0, s0 = p.leaves()
    c0 = _cells(k0, l0, s0)
    f0 = p.get_f()
    flags = (np.random.default_rng(seed + 7).random(len(k0)) < 0.2).astype(np.uint8)
    p.refine_project(flags)
    k1, l1, s1 = p.leaves()
    periodic = [bc[2 * d] == 0 for d in range(3)]
    assert brute.balance_violations(k1, l1, dim, L, periodic) == []
    assert sum(2.0 ** (-dim * int(l)) for l in l1) == pytest.approx(1.0, abs=1e-15)
    # every flagged leaf below the deepest level is split
    new = {(int(k), int(l)) for k, l in zip(k1, l1)}
    for a in np.nonzero(flags)[0]:
        if int(l0[a]) < L:
            assert (int(k0[a]), int(l0[a])) not in new
    f1 = p.get_f()
    xi = p.xi.reshape(-1, 3)
    fs = (2 * np.pi) ** -1.5 * np.exp(-0.5 * (xi * xi).sum(1))
    old_leaves = [(int(k), int(l), int(s)) for k, l, s in zip(k0, l0, s0)]
    cell_of = {kl: i for i, kl in enumerate(c0)}
    for q, (k, l) in enumerate(_cells(k1, l1, s1)):
        # the old leaf that contains the new cell
        owner = [(kk, ll, ss) for kk, ll, ss in old_leaves if ll <= l and (k >> (dim * (L - ll))) == (kk >> (dim * (L - ll)))]
        assert len(owner) == 1
        kk, ll, ss = owner[0]
        want = fs if ss else f0[cell_of[(kk, ll)]]
        assert np.array_equal(f1[q], want)


@pytest.mark.parametrize("case", CASES)
def test_library_host_adaptation_matches_oracle(case):
    """The library's coarsening and refinement (host work, no device) give
    the oracle's leaf lists bit for bit."""
    dim, base, L, pred, r, beta, solid, bc, prob, seed = case
    s = D.Solver(D.F32, D.COLL_BGK, 0.1)
    s.build_tree(D.tree_spec(dim, base, L, pred, (0.5, 0.5, 0.5), r, beta, solid, bc))
    p = _problem(case)
    flags = (np.random.default_rng(seed).random(s.nleaves) < prob).astype(np.uint8)
    s.coarsen(flags)
    p.coarsen_project(flags)
    ks, ls, ss = s.leaves()
    ko, lo, so = p.leaves()
    assert np.array_equal(ks, ko) and np.array_equal(ls, lo) and np.array_equal(ss, so)
    rf = (np.random.default_rng(seed + 3).random(s.nleaves) < 0.25).astype(np.uint8)
    s.refine(rf)
    p.refine_project(rf)
    ks, ls, ss = s.leaves()
    ko, lo, so = p.leaves()
    assert np.array_equal(ks, ko) and np.array_equal(ls, lo) and np.array_equal(ss, so)
