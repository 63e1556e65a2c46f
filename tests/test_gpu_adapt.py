"""Mesh adaptation around the step (GPU): coarsening with f carried over
(dvm_coarsen_project) and the continuum-breakdown sensor (dvm_kn_local,
dvm_flag_kinetic).

Coarsening is checked against an independent mapping from the leaf lists
(Morton keys and levels): a merged parent holds the mean of its children's
f, an unchanged cell its own f.  Mass, momentum and energy are then kept
exactly (a parent's volume is the sum of its children's).  The sensor is
checked against the oracle's local Knudsen number."""
import numpy as np
import pytest

import oracle as O
import paper_1503_00707_gb300 as D
import workloads as W
from tests.gpu_util import oracle_for, pair, rel_linf, same_start

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


def _totals(s, f, dim):
    _, h = s.centres()
    xi = s.velocities()
    V = h ** dim
    psi = np.stack([np.ones(len(xi)), xi[:, 0], xi[:, 1], xi[:, 2], (xi ** 2).sum(1)], 1)
    return (V[:, None] * (f @ psi)).sum(0)


def _expected_after_coarsen(k0, l0, f0, k1, l1, dim, L):
    """f of each new cell: the old cell with the same leaf, else the mean of
    the old cells inside it."""
    out = np.zeros((len(k1), f0.shape[1]))
    old = {(int(k), int(l)): i for i, (k, l) in enumerate(zip(k0, l0))}
    for q, (k, l) in enumerate(zip(k1, l1)):
        k, l = int(k), int(l)
        if (k, l) in old:
            out[q] = f0[old[(k, l)]]
            continue
        sh = dim * (L - l)
        inside = [i for i, (kk, ll) in enumerate(zip(k0, l0)) if int(ll) > l and (int(kk) >> sh) == (k >> sh)]
        assert inside
        out[q] = f0[inside].mean(axis=0)
    return out


@pytest.mark.parametrize("name,precision", [("c1_2d_bump", D.F64), ("c4_hs_bimodal", D.F32)])
def test_coarsen_project_means_children(name, precision):
    """The 3D FP32 case (a 1,464-cell periodic tree coarsened to about 1,150
    cells) runs the 16^3 step kernel at two CTAs per SM: its cells run out
    within the first six of every CTA, where the two solver warps' takes can
    leave an empty slot of one parity before a full slot of the other.  The
    kernel tracks the two parities separately, so that order is harmless."""
    c = dict(W.CONFIGS[name])
    if name == "c4_hs_bimodal":
        c.update(base_level=2, max_level=4, coll=D.COLL_BGK, r=0.3)
    s = D.solver_from_config(c, precision, D.COLL_BGK)
    xyz, _ = s.centres()
    s.init_maxwellian(*W.initial_state(c, xyz))
    s.step(2, s.dt_cfl(c["cfl"]))
    f0 = s.get_f()
    k0, l0 = _cells(s)
    tot0 = _totals(s, f0, c["dim"])
    flags = (np.random.default_rng(8).random(s.nleaves) < 0.85).astype(np.uint8)
    s.coarsen_project(flags)
    f1 = s.get_f()
    k1, l1 = _cells(s)
    assert len(k1) < len(k0)
    want = _expected_after_coarsen(k0, l0, f0, k1, l1, c["dim"], c["max_level"])
    tol = 1e-15 if precision == D.F64 else 1e-6
    assert rel_linf(f1, want) < tol
    tot1 = _totals(s, f1, c["dim"])
    scale = np.array([tot0[0], tot0[4], tot0[4], tot0[4], tot0[4]])
    assert np.max(np.abs(tot1 - tot0) / scale) < (1e-13 if precision == D.F64 else 1e-6)
    s.step(1, s.dt_cfl(c["cfl"]))


def _adapt_cfg(name):
    c = dict(W.CONFIGS[name])
    if name == "c4_hs_bimodal":
        c.update(base_level=2, max_level=4, coll=D.COLL_BGK, r=0.3)
    return c


@pytest.mark.parametrize("name,precision,tol", [("c1_2d_bump", "f64", 1e-12), ("c4_hs_bimodal", "f32", 1e-5)])
@pytest.mark.parametrize("kind", ["coarsen", "refine"])
def test_adapt_project_and_step_match_oracle(name, precision, tol, kind):
    """dvm_coarsen_project / dvm_refine_project against the oracle's
    orc_coarsen_project / orc_refine_project from the same f, then one step on
    the adapted tree (stencils rebuilt) against the oracle's step."""
    c = _adapt_cfg(name)
    s, o = pair(c, precision=precision, collision=D.COLL_BGK)
    dt = o.dt_cfl(c["cfl"])
    o.step(2, dt, O.COLL_BGK, c["kn"])
    same_start(s, o, o.get_f(), precision)  # a developed state, the same values on both sides
    rng = np.random.default_rng(21)
    if kind == "coarsen":
        flags = (rng.random(s.nleaves) < 0.85).astype(np.uint8)
        s.coarsen_project(flags)
        o.coarsen_project(flags)
    else:
        flags = (rng.random(s.nleaves) < 0.15).astype(np.uint8)
        s.refine_project(flags)
        o.refine_project(flags)
    ks, ls, ss = s.leaves()
    ko, lo, so = o.leaves()
    assert np.array_equal(ks, ko) and np.array_equal(ls, lo) and np.array_equal(ss, so)
    # the projection: injection is exact; a mean of 2^dim values rounds once
    # per addition in the storage precision
    ptol = 4e-16 if precision == "f64" else 4e-7
    assert rel_linf(s.get_f(), o.get_f()) <= ptol
    dt1 = o.dt_cfl(c["cfl"])
    assert s.dt_cfl(c["cfl"]) == dt1
    s.step(1, dt1)
    o.step(1, dt1, O.COLL_BGK, c["kn"])
    assert rel_linf(s.get_f(), o.get_f()) < tol
    (r1, u1, T1), (r2, u2, T2) = s.moments(), o.moments()
    assert rel_linf(r1, r2) < tol and rel_linf(T1, T2) < tol and np.max(np.abs(u1 - u2)) < tol


def test_refine_then_coarsen_restores_f():
    """Injection into the children, then their mean: the original f."""
    c = W.CONFIGS["c1_2d_bump"]
    s = D.solver_from_config(c, D.F64, D.COLL_BGK)
    xyz, _ = s.centres()
    s.init_maxwellian(*W.initial_state(c, xyz))
    f0 = s.get_f()
    k0, l0 = _cells(s)
    flags = np.zeros(s.nleaves, dtype=np.uint8)
    keys, lev, _ = s.leaves()
    flags[(lev == c["base_level"])] = 1  # refine the coarse level (the balance adds nothing there)
    s.refine_project(flags)
    k1, l1, _ = s.leaves()
    back = np.zeros(len(k1), dtype=np.uint8)
    new = {(int(k), int(l)) for k, l in zip(k1, l1)} - {(int(k), int(l)) for k, l in zip(k0, l0)}
    for i, (k, l) in enumerate(zip(k1, l1)):
        back[i] = (int(k), int(l)) in new
    s.coarsen_project(back)
    k2, l2 = _cells(s)
    assert np.array_equal(k2, k0) and np.array_equal(l2, l0)
    assert rel_linf(s.get_f(), f0) < 4e-16


@pytest.mark.parametrize("name,precision,tol", [("c1_2d_bump", "f64", 1e-10), ("c2_sphere_m3", "f32", 1e-9)])
def test_kn_local_matches_oracle(name, precision, tol):
    c = W.CONFIGS[name]
    s, o = pair(c, precision=precision)
    dt = o.dt_cfl(c["cfl"])
    o.step(5, dt, O.COLL_BGK, c["kn"])
    same_start(s, o, o.get_f(), precision)
    knl = s.kn_local()
    ko = o.kn_local(c["kn"])
    assert rel_linf(knl, ko) < tol
    thr = float(np.median(ko))
    flags, n = s.flag_kinetic(thr)
    clear = np.abs(ko - thr) > 1e-3 * thr
    assert np.array_equal(flags[clear], (ko[clear] > thr).astype(np.uint8))
    assert n == int(flags.sum())
