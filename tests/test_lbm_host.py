"""Host logic of the lattice Boltzmann step (no GPU): the library's compact
upwind codes against the oracle's independently built face lists."""
import numpy as np
import pytest

import oracle as O
import paper_1503_00707_gb300 as D
import workloads as W

CELL, WALL, OVF = (1 << 27) - 1, 1 << 27, 1 << 30


def _decode(code, ovf):
    """{(source, wall): m} of one side"""
    out = {}
    ents = [code] if not code & OVF else list(ovf[(code & CELL):(code & CELL) + ((code >> 28) & 3) + 1])
    for e in ents:
        e = int(e)
        k = (e & CELL, bool(e & WALL))
        out[k] = out.get(k, 0) + ((e >> 28) & 3) + 1
    return out


def _expected(o, dim):
    """Per (cell, 2d + s): {(source, wall): m} from the oracle's faces.  Side
    s = 0 of axis d holds the sources a velocity with c_d > 0 comes from."""
    nc = o.ncells
    keys, lev, sol = o.leaves()
    cell_of_leaf = -np.ones(len(keys), dtype=np.int64)
    cell_of_leaf[sol == 0] = np.arange(nc)
    _, h = o.centres()
    exp = [[{} for _ in range(2 * dim)] for _ in range(nc)]
    full = 2 ** (dim - 1)

    def add(c, side, key, area):
        m = area / h[c] ** (dim - 1) * full
        assert abs(m - round(m)) < 1e-9
        d = exp[c][side]
        d[key] = d.get(key, 0) + int(round(m))

    fm, fp, fax, far = o.faces()
    for a, b, ax, ar in zip(fm, fp, fax, far):
        ca, cb = cell_of_leaf[a], cell_of_leaf[b]
        if ca >= 0 and cb >= 0:
            add(cb, 2 * ax, (ca, False), ar)       # b's minus side sees a
            add(ca, 2 * ax + 1, (cb, False), ar)   # a's plus side sees b
    bl, bax, bside, bkind, bother, bar = o.bfaces()
    for leaf, ax, side, kind, other, ar in zip(bl, bax, bside, bkind, bother, bar):
        c = cell_of_leaf[leaf]
        if c < 0:
            continue
        if kind == O.BC_INFLOW:
            key = (nc, False)
        elif kind == O.BC_OUTFLOW:
            key = (c, False)
        else:
            key = (c, True)
        add(c, 2 * ax + side, key, ar)
    return exp


@pytest.mark.parametrize("name", ["l1_2d_disk_d2q9", "l2_sphere_d3q19_small"])
def test_codes_match_oracle_faces(name):
    c = W.CONFIGS[name]
    s = D.Solver(D.F32, D.COLL_NONE, 1.0)
    s.build_tree(D.tree_spec(c["dim"], c["base_level"], c["max_level"], c["pred"], c["c"], c["r"],
                             c["beta"], c["solid"], c["bc"]))
    codes, ovf = s.lbm_codes()
    o = O.Problem(O.make_spec(c["dim"], c["base_level"], c["max_level"], c["pred"], c["c"], c["r"],
                              c["beta"], c["solid"], c["bc"]), lattice=c["lattice"])
    assert o.ncells == s.ncells
    dim = c["dim"]
    exp = _expected(o, dim)
    n_ovf_sides = 0
    for cell in range(o.ncells):
        for side in range(2 * dim):
            code = int(codes[side, cell])
            n_ovf_sides += bool(code & OVF)
            assert _decode(code, ovf) == exp[cell][side], (cell, side)
    # refined trees have coarse cells next to finer ones
    assert n_ovf_sides > 0 and len(ovf) >= 2 * n_ovf_sides


@pytest.mark.parametrize("kind", [D.LBM_D2Q9, D.LBM_D3Q19, D.LBM_D3Q27])
def test_library_velocity_set_equals_oracle(kind):
    """The library's velocity set and weights, written independently of the
    oracle's from the same rule, are the oracle's (which the isotropy pins
    fix) bit for bit."""
    c, w = D.lbm_lattice(kind)
    oc, ow = O.lattice(kind)
    assert np.array_equal(c.astype(np.float64), oc)
    assert np.array_equal(w, ow)


def test_unknown_lattice_is_rejected():
    with pytest.raises(D.DvmError):
        D.lbm_lattice(15)
