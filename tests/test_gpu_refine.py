"""Refinement with the distribution carried over (dvm_refine_project): every
new cell starts with the f of the old cell that contains it.  Checked
against an independent mapping from the leaf lists (Morton keys and levels)
and by exact conservation of mass, momentum and energy, which piecewise-
constant injection keeps because a parent's volume is the sum of its
children's."""
import numpy as np
import pytest

import paper_1503_00707_gb300 as D
import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def gpu():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA GPU")
    from paper_1503_00707_gb300 import _build
    _build.build()


def _cells(s):
    keys, lev, solid = s.leaves()
    fluid = solid == 0
    return keys[fluid].astype(np.uint64), lev[fluid].astype(np.int64)


def _containing(old_keys, old_lev, new_keys, new_lev, dim, L):
    """Old cell index containing each new cell (-1: none), by the Morton
    prefix: a leaf of level l covers the keys that share its top dim*l bits
    below the depth-L anchor."""
    out = np.full(len(new_keys), -1)
    for q, (k, l) in enumerate(zip(new_keys, new_lev)):
        for o in range(len(old_keys)):
            lo_ = int(old_lev[o])
            if lo_ > l:
                continue
            sh = dim * (L - lo_)
            if (int(k) >> sh) == (int(old_keys[o]) >> sh):
                out[q] = o
                break
    return out


def _totals(s, f, dim):
    xyz, h = s.centres()
    xi = s.velocities()
    V = h ** dim
    psi = np.stack([np.ones(len(xi)), xi[:, 0], xi[:, 1], xi[:, 2], (xi ** 2).sum(1)], 1)
    return (V[:, None] * (f @ psi)).sum(0)


@pytest.mark.parametrize("name,precision", [("c1_2d_bump", D.F64), ("c4_hs_bimodal", D.F32)])
def test_refine_project_injects_parent_f(name, precision):
    c = dict(W.CONFIGS[name])
    if name == "c4_hs_bimodal":
        c.update(base_level=2, max_level=4, coll=D.COLL_BGK, r=0.3)
    s = D.solver_from_config(c, precision, D.COLL_BGK)
    xyz, _ = s.centres()
    s.init_maxwellian(*W.initial_state(c, xyz))
    f0 = s.get_f()
    k0, l0 = _cells(s)
    tot0 = _totals(s, f0, c["dim"])
    rng = np.random.default_rng(5)
    flags = (rng.random(s.nleaves) < 0.15).astype(np.uint8)
    s.refine_project(flags)
    f1 = s.get_f()
    k1, l1 = _cells(s)
    assert len(k1) > len(k0)
    src = _containing(k0, l0, k1, l1, c["dim"], c["max_level"])
    assert np.all(src >= 0)
    assert np.array_equal(f1, f0[src])
    tot1 = _totals(s, f1, c["dim"])
    scale = np.array([tot0[0], tot0[4], tot0[4], tot0[4], tot0[4]])
    assert np.max(np.abs(tot1 - tot0) / scale) < 1e-12
    # and the new mesh steps
    dt = s.dt_cfl(c["cfl"])
    s.step(2, dt)
    s.close()


def test_refine_project_needs_f():
    c = W.CONFIGS["c1_2d_bump"]
    s = D.solver_from_config(c, D.F64, D.COLL_BGK)
    with pytest.raises(D.DvmError) as e:
        s.refine_project(np.zeros(s.nleaves, np.uint8))
    assert e.value.code == -4
    s.close()
