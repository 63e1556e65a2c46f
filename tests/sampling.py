"""Cell samples and sampled oracle steps for parity checks on trees whose f is
too large for the oracle to hold (the full Mach-5 flow: 1.01M cells x 13,824
velocities).

The sample holds seeded random cells plus cells of every face kind the
transport step treats apart: a wall face, an inflow face, an outflow face and
a level change across an interior face.  The oracle steps a sample from the
f rows of the cells it reads (its face neighbours, one ring wider per step),
with the per-cell arithmetic of its full step."""
import numpy as np

import oracle as O


def oracle_sparse_for(c):
    o = O.Problem(O.make_spec(c["dim"], c["base_level"], c["max_level"], c["pred"], c["c"], c["r"],
                              c["beta"], c["solid"], c["bc"]), c["n"], c["lo"], c["hi"], store_f=False)
    o.set_freestream(c["fs_rho"], c["fs_u"], c["fs_T"])
    return o


def cell_sample(o, n_random, n_each, seed):
    """Sorted distinct cell indices: n_random seeded random cells and up to
    n_each cells of each face kind."""
    _, lev, sol = o.leaves()
    cell_of_leaf = np.cumsum(sol == 0) - 1
    g = np.random.default_rng(seed)
    picks = [g.choice(o.ncells, min(n_random, o.ncells), replace=False)]
    leaf, _, _, kind, _, _ = o.bfaces()
    for k in (O.BC_WALL, O.BC_INFLOW, O.BC_OUTFLOW):
        cand = np.unique(cell_of_leaf[leaf[kind == k]])
        if cand.size:
            picks.append(g.choice(cand, min(n_each, cand.size), replace=False))
    m, p, _, _ = o.faces()
    hang = lev[m] != lev[p]
    cand = np.unique(np.concatenate([cell_of_leaf[m[hang]], cell_of_leaf[p[hang]]]))
    if cand.size:
        picks.append(g.choice(cand, min(n_each, cand.size), replace=False))
    return np.unique(np.concatenate(picks)).astype(np.int64)


def oracle_rows_after(o, cells, init, nsteps, dt, kn, coll=O.COLL_BGK):
    """f rows of `cells` after nsteps steps (transport, then the collision
    update coll) from the Maxwellian mixture init = (w, rho, u, T) (per cell
    of the whole tree), in FP64."""
    rings = [np.asarray(cells, dtype=np.int64)]
    for _ in range(nsteps):
        rings.append(o.step_inputs(rings[-1]))
    w, r, u, T = init
    base = rings[-1]
    f = o.maxwellian_rows(w[base], r[base], u[base], T[base])
    for k in range(nsteps, 0, -1):
        f = o.step_cells(rings[k - 1], rings[k], f, dt, coll, kn)
    return f
