"""GPU parity of the fused transport + moments + BGK step against the FP64
oracle, through the C ABI.

Bars: macroscopic fields within relative L-infinity 1e-5 of the oracle after
N steps (FP64 and FP32 storage); f itself within FP64 rounding (1e-12) for
FP64 storage; BF16 storage within its 8-bit mantissa (4e-3 per step).
"""
import math

import numpy as np
import pytest

import oracle as O
import paper_1503_00707_gb300 as D
import workloads as W
from tests.gpu_util import field_errors, oracle_for, pair, rel_linf, same_start, volume_totals

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def gpu():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA GPU")
    from paper_1503_00707_gb300 import _build
    _build.build()


def test_c1_2d_bump_fp64_50_steps():
    c = W.CONFIGS["c1_2d_bump"]
    s, o = pair(c)
    dt = o.dt_cfl(c["cfl"])
    assert s.dt_cfl(c["cfl"]) == dt
    tot0 = volume_totals(s.get_f(), o, c["dim"])
    s.step(c["steps"], dt)
    o.step(c["steps"], dt, O.COLL_BGK, c["kn"])
    fs, fo = s.get_f(), o.get_f()
    assert rel_linf(fs, fo) < 1e-12
    err = field_errors(s.moments(), o.moments())
    assert max(err.values()) < 1e-12, err
    # global conservation over 50 steps on the periodic FP64 mesh
    tot1 = volume_totals(fs, o, c["dim"])
    scale = np.array([tot0[0], tot0[4], tot0[4], tot0[4], tot0[4]])
    assert np.max(np.abs(tot1 - tot0) / scale) < 1e-12


def test_c2_sphere_fp32_200_steps():
    """The Mach-3 sphere flow for its full 200 steps (t = 0.074; the oracle
    takes about four minutes), fields checked every 50 steps.  A compressed
    layer stands ahead of the sphere from the first 50 steps on (peak density
    2.1-2.2 times the freestream's)."""
    c = W.CONFIGS["c2_sphere_m3"]
    assert c["steps"] == 200
    s, o = pair(c)
    dt = o.dt_cfl(c["cfl"])
    for _ in range(4):
        s.step(50, dt)
        o.step(50, dt, O.COLL_BGK, c["kn"])
        err = field_errors(s.moments(), o.moments())
        assert max(err.values()) < 1e-5, err
    rho, _, _ = o.moments()
    assert rho.max() > 1.8
    # the step's own moments of f* agree with the moments of the stored state
    r1, u1, T1 = s.step_moments()
    r2, u2, T2 = s.moments()
    assert rel_linf(r1, r2) < 1e-6 and rel_linf(T1, T2) < 1e-6


def test_c3_flow_small_tree_fp32():
    """The 24^3 Mach-5 sphere flow (the throughput workload's launch shape:
    432 threads per cell, inflow, outflow and wall stencils) on a 17.7k-cell
    tree the oracle finishes in seconds."""
    c = W.CONFIGS["c3_sphere_m5_small"]
    s, o = pair(c)
    # start away from equilibrium so that every term is exercised
    same_start(s, o, o.get_f() * W.random_f_perturbation(o.ncells, o.nv, scale=0.2), "f32")
    dt = o.dt_cfl(c["cfl"])
    s.step(c["steps"], dt)
    o.step(c["steps"], dt, O.COLL_BGK, c["kn"])
    fs, fo = s.get_f(), o.get_f()
    assert rel_linf(fs, fo) < 1e-5
    err = field_errors(s.moments(), o.moments())
    assert max(err.values()) < 1e-5, err


def test_c3_flow_small_tree_bf16():
    c = W.CONFIGS["c3_sphere_m5_small"]
    s, o = pair(c, precision="bf16")
    dt = o.dt_cfl(c["cfl"])
    s.step(2, dt)
    o.step(2, dt, O.COLL_BGK, c["kn"])
    err = field_errors(s.moments(), o.moments())
    assert max(err.values()) < 1e-2, err


@pytest.mark.parametrize("prec", ["f64", "f32"])
def test_transport_only_hanging_faces(prec):
    """Eq. 2 alone on a refined periodic tree with walls and inflow, from a
    random non-equilibrium f: every element against the oracle."""
    c = dict(W.CONFIGS["c2_sphere_m3"])
    c.update(base_level=2, max_level=4, r=0.2, beta=0.5, n=(8, 8, 8), lo=(-3.0,) * 3, hi=(3.0,) * 3,
             bc=(1, 3, 0, 0, 2, 3))
    s, o = pair(c, precision=prec, collision=O.COLL_NONE, init=False)
    rng = np.random.default_rng(11)
    f0 = rng.uniform(0.05, 1.0, (o.ncells, o.nv))
    s.set_f(f0)
    o.set_f(f0)
    dt = o.dt_cfl(0.45)
    s.step(3, dt)
    o.step(3, dt, O.COLL_NONE, 1.0)
    tol = 1e-13 if prec == "f64" else 3e-6
    assert rel_linf(s.get_f(), o.get_f()) < tol


def test_2d_fp32_and_small_velocity_grid():
    """2D quadtree in FP32 with an 8^3 velocity grid (one warp per cell)."""
    c = dict(W.CONFIGS["c1_2d_bump"])
    c["precision"] = "f32"
    s, o = pair(c)
    dt = o.dt_cfl(c["cfl"])
    s.step(10, dt)
    o.step(10, dt, O.COLL_BGK, c["kn"])
    err = field_errors(s.moments(), o.moments())
    assert max(err.values()) < 1e-5, err


def test_bgk_collision_conserves_per_cell_fp64():
    """Homogeneous relaxation in FP64: each cell's moments are unchanged by the
    collision update to 1e-13 (the correction of Eq. 6 at work)."""
    c = dict(W.CONFIGS["c1_2d_bump"])
    c.update(base_level=2, max_level=2, pred=O.PRED_NONE)
    s, o = pair(c, init=False)
    nc = o.ncells
    rng = np.random.default_rng(3)
    u = np.zeros((nc, 2, 3))
    u[:, 0, 0], u[:, 1, 0] = 1.2, -1.2
    w = np.tile([0.4, 0.6], (nc, 1))
    s.init_maxwellian(w, np.ones((nc, 2)), u, np.full((nc, 2), 0.6))
    r0, u0, T0 = s.moments()
    s.step(5, 2e-3)
    r1, u1, T1 = s.moments()
    assert rel_linf(r1, r0) < 1e-13 and np.max(np.abs(u1 - u0)) < 1e-13 and rel_linf(T1, T0) < 1e-13


def test_unstable_dt_is_reported():
    c = W.CONFIGS["c1_2d_bump"]
    s, o = pair(c)
    with pytest.raises(D.DvmError) as e:
        s.step(1, 0.5)  # nu * dt >> 1
    assert e.value.code == -5


def test_negative_density_is_reported():
    c = W.CONFIGS["c1_2d_bump"]
    s, o = pair(c)
    f = s.get_f()
    f[7] = -f[7]
    s.set_f(f)
    with pytest.raises(D.DvmError) as e:
        s.step(1, o.dt_cfl(0.4))
    assert e.value.code == -5
    # the context stays usable after the error
    s.set_f(np.abs(f))
    s.step(1, o.dt_cfl(0.4))


def test_call_order_is_checked():
    s = D.Solver(D.F32, D.COLL_BGK, 0.1)
    with pytest.raises(D.DvmError) as e:
        s.step(1, 1e-3)
    assert e.value.code == -4
