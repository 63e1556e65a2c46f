"""Coarsening of the tree (host logic, no GPU): the library's dvm_coarsen
against a brute-force statement of the rule, on refined trees with random
flags.  Rule: 2^dim sibling leaves, all flagged, with the parent at or above
the base level, merge into the parent unless the parent would touch a leaf
two or more levels finer; such merges are undone until none is left."""
import numpy as np
import pytest

import paper_1503_00707_gb300 as D
from tests import brute

CASES = [
    # dim, base, max, predicate, r, beta, solid, bc, flag probability, seed
    (2, 2, 5, D.PRED_BALL if hasattr(D, "PRED_BALL") else 1, 0.2, 0.0, 0, (0,) * 6, 0.8, 1),
    (2, 2, 6, 2, 0.25, 1.5, 1, (1, 2, 0, 0, 0, 0), 0.7, 2),
    (3, 1, 4, 1, 0.3, 0.0, 0, (0,) * 6, 0.9, 3),
    (3, 2, 4, 2, 0.2, 1.0, 1, (1, 2, 3, 3, 3, 3), 0.8, 4),
]


def _brute_coarsen(keys, lev, flags, dim, base, L, periodic):
    keys = [int(k) for k in keys]
    lev = [int(l) for l in lev]
    n, nch = len(keys), 1 << dim
    groups = []
    q = 0
    while q + nch <= n:
        l = lev[q]
        sh = dim * (L - l + 1)
        ok = l > base and all(flags[q + k] and lev[q + k] == l and (keys[q + k] >> sh) == (keys[q] >> sh)
                              for k in range(nch))
        if ok:
            groups.append((q, l - 1, (keys[q] >> sh) << sh))
            q += nch
        else:
            q += 1
    on = [True] * len(groups)

    def leaf_set():
        out = []
        merged = {g[0] for g, o in zip(groups, on) if o}
        q = 0
        while q < n:
            if q in merged:
                g = next(g for g in groups if g[0] == q)
                out.append((g[2], g[1]))
                q += nch
            else:
                out.append((keys[q], lev[q]))
                q += 1
        return out

    N = 1 << L
    changed = True
    while changed:
        changed = False
        cur = leaf_set()
        bx = brute.boxes([k for k, _ in cur], [l for _, l in cur], dim, L)
        for gi, (q, pl, pk) in enumerate(groups):
            if not on[gi]:
                continue
            P = brute.boxes([pk], [pl], dim, L)[0]
            if any(l >= pl + 2 and brute.touching(P, b, dim, N, periodic) for (k, l), b in zip(cur, bx)):
                on[gi] = False
                changed = True
                break
    return leaf_set()


@pytest.mark.parametrize("case", CASES)
def test_coarsen_matches_brute_force(case):
    dim, base, L, pred, r, beta, solid, bc, prob, seed = case
    s = D.Solver(D.F32, D.COLL_BGK, 0.1)
    s.build_tree(D.tree_spec(dim, base, L, pred, (0.5, 0.5, 0.5), r, beta, solid, bc))
    k0, l0, _ = s.leaves()
    rng = np.random.default_rng(seed)
    flags = (rng.random(len(k0)) < prob).astype(np.uint8)
    periodic = [bc[2 * d] == 0 for d in range(3)]
    want = _brute_coarsen(k0, l0, flags, dim, base, L, periodic)
    s.coarsen(flags)
    k1, l1, sol1 = s.leaves()
    got = list(zip([int(k) for k in k1], [int(l) for l in l1]))
    assert got == want
    assert len(got) < len(k0)
    assert brute.balance_violations(k1, l1, dim, L, periodic) == []
    # volumes still tile the domain
    assert sum(2.0 ** (-dim * int(l)) for l in l1) == pytest.approx(1.0, abs=1e-15)


@pytest.mark.parametrize("case", [CASES[1], CASES[3]])
def test_coarsened_mesh_faces_match_brute_force(case):
    """The faces the library builds for a coarsened tree (the input of every
    stencil) equal a pairwise box-contact enumeration, walls against solid
    leaves and domain sides included."""
    from fractions import Fraction
    dim, base, L, pred, r, beta, solid, bc, prob, seed = case
    s = D.Solver(D.F32, D.COLL_BGK, 0.1)
    s.build_tree(D.tree_spec(dim, base, L, pred, (0.5, 0.5, 0.5), r, beta, solid, bc))
    flags = (np.random.default_rng(seed).random(s.nleaves) < prob).astype(np.uint8)
    s.coarsen(flags)
    keys, lev, sol = s.leaves()
    m, pl, ax, ar = s.faces()
    got = sorted((int(a), int(b), int(c), Fraction(float(d))) for a, b, c, d in zip(m, pl, ax, ar))
    inter, bnd = brute.faces(keys, lev, sol, dim, L, bc)
    assert got == sorted(inter)
    bl, bax, bside, bkind, bother, bar = s.bfaces()
    gotb = sorted((int(a), int(b), int(c), int(d), int(e), Fraction(float(f)))
                  for a, b, c, d, e, f in zip(bl, bax, bside, bkind, bother, bar))
    assert gotb == sorted(bnd)


def test_coarsen_rejects_bad_flag_count():
    s = D.Solver(D.F32, D.COLL_BGK, 0.1)
    s.build_tree(D.tree_spec(2, 2, 4, 1, (0.5, 0.5, 0.5), 0.2, 0.0, 0, (0,) * 6))
    with pytest.raises(D.DvmError) as e:
        s.coarsen(np.ones(3, dtype=np.uint8))
    assert e.value.code == -1
