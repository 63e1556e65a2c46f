"""The oracle's selected-cell step (for trees whose f it cannot hold) against
its full step, BGK and hard sphere: the same per-cell arithmetic, so the rows
must be identical."""
import numpy as np
import pytest

import oracle as O
import workloads as W
from tests.gpu_util import random_params
from tests.sampling import cell_sample, oracle_rows_after, oracle_sparse_for


def _case():
    # the Mach-3 sphere flow on levels 3-5: walls, inflow, outflow and
    # hanging faces on a tree the dense oracle steps in seconds
    return dict(W.CONFIGS["c2_sphere_m3"], base_level=3, max_level=5, n=(8, 8, 8), lo=(-5.0,) * 3,
                hi=(5.0,) * 3, init="bimodal")


def _dense(c):
    o = O.Problem(O.make_spec(c["dim"], c["base_level"], c["max_level"], c["pred"], c["c"], c["r"],
                              c["beta"], c["solid"], c["bc"]), c["n"], c["lo"], c["hi"])
    o.set_freestream(c["fs_rho"], c["fs_u"], c["fs_T"])
    return o


@pytest.mark.parametrize("coll,nsteps", [(O.COLL_BGK, 1), (O.COLL_BGK, 3), (O.COLL_HS, 2)])
def test_selected_cells_equal_full_step(coll, nsteps):
    c = _case()
    o, sp = _dense(c), oracle_sparse_for(c)
    if coll == O.COLL_HS:
        o.hs_tables(16, W.SEED)
        sp.hs_tables(16, W.SEED)
    xyz, _ = o.centres()
    assert np.array_equal(xyz, sp.centres()[0])
    init = W.initial_state(c, xyz)
    o.init_maxwellian(*init)
    dt = o.dt_cfl(c["cfl"])
    o.step(nsteps, dt, coll, c["kn"])
    cells = cell_sample(sp, 24, 8, seed=5)
    assert cells.size >= 40  # every face kind is present in this tree
    got = oracle_rows_after(sp, cells, init, nsteps, dt, c["kn"], coll)
    assert np.array_equal(got, o.get_f()[cells])


def test_sample_covers_face_kinds():
    c = _case()
    sp = oracle_sparse_for(c)
    cells = cell_sample(sp, 0, 4, seed=1)
    _, lev, sol = sp.leaves()
    cell_of_leaf = np.cumsum(sol == 0) - 1
    leaf, _, _, kind, _, _ = sp.bfaces()
    for k in (O.BC_WALL, O.BC_INFLOW, O.BC_OUTFLOW):
        assert np.intersect1d(cells, cell_of_leaf[leaf[kind == k]]).size > 0, k
    m, p, _, _ = sp.faces()
    hang = lev[m] != lev[p]
    assert np.intersect1d(cells, cell_of_leaf[np.concatenate([m[hang], p[hang]])]).size > 0


def test_inputs_hold_cells_and_neighbours():
    c = _case()
    sp = oracle_sparse_for(c)
    m, p, _, _ = sp.faces()
    _, _, sol = sp.leaves()
    cell_of_leaf = np.cumsum(sol == 0) - 1
    cm, cp = cell_of_leaf[m], cell_of_leaf[p]
    cells = np.array([0, 7, sp.ncells - 1])
    want = set(cells.tolist())
    for x in cells:
        want |= set(cp[cm == x].tolist()) | set(cm[cp == x].tolist())
    assert sp.step_inputs(cells).tolist() == sorted(want)


def test_missing_rows_and_bad_indices_refused():
    c = _case()
    sp = oracle_sparse_for(c)
    xyz, _ = sp.centres()
    init = W.initial_state(c, xyz)
    cells = np.array([3, 40])
    inp = sp.step_inputs(cells)
    w, r, u, T = init
    f = sp.maxwellian_rows(w[inp], r[inp], u[inp], T[inp])
    with pytest.raises(RuntimeError):
        sp.step_cells(cells, inp[1:], f[1:], 1e-4, O.COLL_BGK, c["kn"])
    with pytest.raises(RuntimeError):  # hard sphere without tables
        sp.step_cells(cells, inp, f, 1e-4, O.COLL_HS, c["kn"])
    with pytest.raises(IndexError):
        sp.step_inputs(np.array([sp.ncells]))
    with pytest.raises(RuntimeError):
        sp.get_f()


def test_selected_cells_learned_equal_full_step():
    """Transport, then the learned update with the hard-sphere fallback: the
    sampled rows, local Kn and gate outcomes equal the full step's bit for
    bit, with the threshold splitting the cells."""
    c = dict(_case(), init="bimodal_near")
    o, sp = _dense(c), oracle_sparse_for(c)
    o.hs_tables(16, W.SEED)
    sp.hs_tables(16, W.SEED)
    xyz, _ = o.centres()
    init = W.initial_state(c, xyz)
    o.init_maxwellian(*init)
    params = random_params(3, gain=0.3, bias=0.0).astype(np.float64)
    dt = o.dt_cfl(c["cfl"]) / 4
    o.step(1, dt, O.COLL_NONE, c["kn"])
    knl = o.kn_local(c["kn"])
    ks = np.sort(knl)
    thr = float(0.5 * (ks[len(ks) // 2 - 1] + ks[len(ks) // 2]))
    used, _ = o.learned_collide(dt, c["kn"], params, thr)
    cells = cell_sample(sp, 24, 8, seed=6)
    ring2 = sp.step_inputs(sp.step_inputs(cells))
    w, r, u, T = init
    fin = sp.maxwellian_rows(w[ring2], r[ring2], u[ring2], T[ring2])
    rows, knl_s, used_s = sp.step_cells_learned(cells, ring2, fin, dt, c["kn"], params, thr)
    assert np.array_equal(knl_s, knl[cells])
    assert np.array_equal(used_s, used[cells])
    assert 0 < used_s.sum() < cells.size
    assert np.array_equal(rows, o.get_f()[cells])
    # one ring of rows is not enough: the local Kn reads the neighbours' f*
    ring1 = sp.step_inputs(cells)
    f1 = sp.maxwellian_rows(w[ring1], r[ring1], u[ring1], T[ring1])
    with pytest.raises(RuntimeError):
        sp.step_cells_learned(cells, ring1, f1, dt, c["kn"], params, thr)
