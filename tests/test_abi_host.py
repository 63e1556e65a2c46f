"""Host-side checks of libdvm (no GPU): the shared library loads and exports
every entry point declared in include/dvm.h, and its host mesh builder (a
different algorithm: hash-set ripple balance, bit-spread Morton keys) matches
the oracle's tree, Morton order and face lists bit for bit."""
import os
import re

import numpy as np
import pytest

import oracle as O
import paper_1503_00707_gb300 as D
import workloads as W
from paper_1503_00707_gb300 import _build

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module", autouse=True)
def built():
    _build.build()


def _declared():
    txt = open(os.path.join(ROOT, "include", "dvm.h")).read()
    txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
    return sorted(set(re.findall(r"\b(dvm_[a-z0-9_]+)\s*\(", txt)))


def test_exports_every_declared_symbol():
    names = _declared()
    assert len(names) >= 25
    L = D.lib()
    for n in names:
        assert hasattr(L, n), n
    assert sorted(D.EXPORTS) == names


def _both(spec_args, bc):
    dim, base, top, pred, c, r, beta, solid = spec_args
    o = O.Problem(O.make_spec(dim, base, top, pred, c, r, beta, solid, bc), (4, 4, 4), (-1,) * 3, (1,) * 3)
    s = D.Solver(D.F32, D.COLL_BGK, 0.1)
    s.build_tree(D.tree_spec(dim, base, top, pred, c, r, beta, solid, bc))
    return o, s


CASES = [
    ((2, 2, 5, O.PRED_BALL, (0.3, 0.6, 0.5), 0.05, 0.0, 0), (0,) * 6),
    ((2, 1, 5, O.PRED_SHELL, (0.5, 0.5, 0.5), 0.3, 0.5, 1), (1, 2, 2, 2, 0, 0)),
    ((2, 2, 5, O.PRED_BALL, (0.0, 0.0, 0.5), 0.1, 0.0, 0), (0,) * 6),
    ((3, 1, 4, O.PRED_BALL, (0.3, 0.6, 0.7), 0.05, 0.0, 0), (0,) * 6),
    ((3, 2, 4, O.PRED_SHELL, (0.5, 0.5, 0.5), 0.15, 0.3, 1), (1, 2, 2, 2, 2, 2)),
    ((3, 1, 4, O.PRED_BALL, (0.97, 0.02, 0.5), 0.05, 0.0, 0), (0, 0, 2, 2, 0, 0)),
    ((3, 2, 6, O.PRED_SHELL, (0.41, 0.52, 0.47), 0.2, 1.5, 1), (3, 2, 0, 0, 2, 3)),
]


def _compare(o, s):
    ko, lo_, so = o.leaves()
    ks, ls, ss = s.leaves()
    assert np.array_equal(ko, ks) and np.array_equal(lo_, ls) and np.array_equal(so, ss)
    for a, b in zip(o.faces(), s.faces()):
        assert np.array_equal(a, b)
    for a, b in zip(o.bfaces(), s.bfaces()):
        assert np.array_equal(a, b)
    xo, ho = o.centres()
    xs, hs = s.centres()
    assert np.array_equal(xo, xs) and np.array_equal(ho, hs)


@pytest.mark.parametrize("case", CASES)
def test_mesh_bit_exact_small(case):
    o, s = _both(*case)
    _compare(o, s)


@pytest.mark.parametrize("name", ["c1_2d_bump", "c2_sphere_m3", "c4_hs_bimodal", "c3_sphere_m5_reduced"])
def test_mesh_bit_exact_configs(name):
    c = W.CONFIGS[name]
    o, s = _both((c["dim"], c["base_level"], c["max_level"], c["pred"], c["c"], c["r"], c["beta"], c["solid"]), c["bc"])
    _compare(o, s)


@pytest.mark.parametrize("name", ["c3_sphere_m5", "c5_sphere_m3_hs"])
def test_mesh_bit_exact_full_size(name):
    """The full-size trees (1.42M and 388k leaves) match bit for bit."""
    c = W.CONFIGS[name]
    o, s = _both((c["dim"], c["base_level"], c["max_level"], c["pred"], c["c"], c["r"], c["beta"], c["solid"]), c["bc"])
    ko, lo_, so = o.leaves()
    ks, ls, ss = s.leaves()
    assert np.array_equal(ko, ks) and np.array_equal(lo_, ls) and np.array_equal(so, ss)
    for a, b in zip(o.faces(), s.faces()):
        assert np.array_equal(a, b)
    for a, b in zip(o.bfaces(), s.bfaces()):
        assert np.array_equal(a, b)


def test_refine_rebalances():
    s = D.Solver(D.F32, D.COLL_BGK, 0.1)
    s.build_tree(D.tree_spec(2, 3, 6, D.PRED_NONE, bc=(0,) * 6))
    keys, lev, sol = s.leaves()
    flags = np.zeros(len(keys), np.uint8)
    flags[5] = 1
    s.refine(flags)
    flags = np.zeros(s.nleaves, np.uint8)
    keys, lev, sol = s.leaves()
    flags[np.argmax(lev)] = 1  # a level-4 leaf -> level 5 forces its coarse neighbours
    s.refine(flags)
    from tests import brute
    keys, lev, sol = s.leaves()
    assert brute.balance_violations(keys, lev, 2, 6, [True, True]) == []
    assert lev.max() == 5


def test_set_velocity_grid_without_gpu_fails_loudly():
    import torch
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    s = D.Solver(D.F32, D.COLL_BGK, 0.1)
    s.build_tree(D.tree_spec(2, 2, 2))
    with pytest.raises(D.DvmError) as e:
        s.set_velocity_grid((8, 8, 8), (-4,) * 3, (4,) * 3)
    assert e.value.code == -3
