"""GPU parity of the lattice Boltzmann step (Sec. 4: finite-volume transport
of Eq. 2 on the D2Q9 / D3Q19 / D3Q27 lattice velocities, then lattice BGK)
against the FP64 oracle, through the C ABI.

Bars: f within 1e-12 of the oracle (relative to max f) for FP64 storage and
1e-5 for FP32; the homogeneous relaxation and the conservation checks are
against closed forms."""
import numpy as np
import pytest

import oracle as O
import paper_1503_00707_gb300 as D
import workloads as W
from tests.gpu_util import rel_linf

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def gpu():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA GPU")
    from paper_1503_00707_gb300 import _build
    _build.build()


def _pair(c, precision=None):
    s = D.lbm_solver_from_config(c, precision)
    o = O.Problem(O.make_spec(c["dim"], c["base_level"], c["max_level"], c["pred"], c["c"], c["r"],
                              c["beta"], c["solid"], c["bc"]), lattice=c["lattice"])
    o.lbm_set_inflow(c["fs_rho"], c["fs_u"])
    xyz, _ = s.centres()
    xo, _ = o.centres()
    assert np.array_equal(xyz, xo)
    rho, u = W.lbm_initial_state(c, xyz)
    s.lbm_init(rho, u)
    o.lbm_init(rho, u)
    return s, o


def test_velocity_set_matches_oracle():
    for name in ("l1_2d_disk_d2q9", "l2_sphere_d3q19_small", "l2_sphere_d3q27_small"):
        c = W.CONFIGS[name]
        s, o = _pair(c)
        cv, w = s.lbm_velocities()
        assert np.array_equal(cv.astype(np.float64), o.xi)
        assert np.array_equal(w, o.w)


def test_2d_disk_d2q9_fp64():
    c = W.CONFIGS["l1_2d_disk_d2q9"]
    s, o = _pair(c)
    assert rel_linf(s.lbm_get_f(), o.get_f()) < 1e-15
    dt = o.dt_cfl(c["cfl"])
    assert s.lbm_dt_cfl(c["cfl"]) == dt
    tau = W.lbm_tau(c, dt)
    s.lbm_step(c["steps"], dt, tau)
    o.lbm_step(c["steps"], dt, tau)
    assert rel_linf(s.lbm_get_f(), o.get_f()) < 1e-12
    (r1, u1), (r2, u2) = s.lbm_moments(), o.lbm_moments()
    assert rel_linf(r1, r2) < 1e-12 and np.max(np.abs(u1 - u2)) < 1e-12


@pytest.mark.parametrize("name", ["l2_sphere_d3q19_small", "l2_sphere_d3q27_small"])
def test_sphere_fp32(name):
    """The Ma-0.5 sphere flow (solid sphere walls, inflow, outflow, hanging
    faces) in FP32 against the FP64 oracle."""
    c = W.CONFIGS[name]
    s, o = _pair(c)
    dt = o.dt_cfl(c["cfl"])
    tau = W.lbm_tau(c, dt)
    s.lbm_step(c["steps"], dt, tau)
    o.lbm_step(c["steps"], dt, tau)
    assert rel_linf(s.lbm_get_f(), o.get_f()) < 1e-5
    (r1, u1), (r2, u2) = s.lbm_moments(), o.lbm_moments()
    assert rel_linf(r1, r2) < 1e-5 and np.max(np.abs(u1 - u2)) < 1e-5


@pytest.mark.parametrize("name", ["l3_sphere_d3q19", "l3_sphere_d3q27"])
def test_sphere_full_size_fp32(name):
    """The bench's lattice Boltzmann workload at its full size (3,336,104
    cells on levels 7-10, f twice the size of L2), five steps, every element
    against the FP64 oracle."""
    c = W.CONFIGS[name]
    s, o = _pair(c)
    assert s.ncells == o.ncells == 3336104
    dt = o.dt_cfl(c["cfl"])
    tau = W.lbm_tau(c, dt)
    s.lbm_step(5, dt, tau)
    o.lbm_step(5, dt, tau)
    assert rel_linf(s.lbm_get_f(), o.get_f()) < 1e-5
    (r1, u1), (r2, u2) = s.lbm_moments(), o.lbm_moments()
    assert rel_linf(r1, r2) < 1e-5 and np.max(np.abs(u1 - u2)) < 1e-5


def test_sphere_d3q27_fp64():
    c = W.CONFIGS["l2_sphere_d3q27_small"]
    s, o = _pair(c, "f64")
    dt = o.dt_cfl(c["cfl"])
    tau = W.lbm_tau(c, dt)
    s.lbm_step(4, dt, tau)
    o.lbm_step(4, dt, tau)
    assert rel_linf(s.lbm_get_f(), o.get_f()) < 1e-12


@pytest.mark.parametrize("lattice,dim", [(D.LBM_D2Q9, 2), (D.LBM_D3Q19, 3), (D.LBM_D3Q27, 3)])
def test_homogeneous_relaxation_closed_form(lattice, dim):
    """Identical cells on a periodic tree: f - feq shrinks by 1 - dt/tau per
    step, feq fixed by the conserved rho, u."""
    c = dict(W.CONFIGS["l1_2d_disk_d2q9"])
    c.update(dim=dim, lattice=lattice, base_level=3, max_level=3, pred=W.PRED_NONE, solid=0,
             bc=(W.PERIODIC,) * 6, precision="f64")
    s = D.lbm_solver_from_config(c)
    rng = np.random.default_rng(4)
    _, w = s.lbm_velocities()
    f0 = w * rng.uniform(0.5, 1.5, s.q)
    s.lbm_set_f(np.tile(f0, (s.ncells, 1)))
    o = O.Problem(O.make_spec(dim, 1, 1), lattice=lattice)
    rho = f0.sum()
    u = o.xi.T @ f0 / rho
    feq = o.lbm_feq(rho, u)
    dt, tau, n = 0.01, 0.04, 9
    s.lbm_step(n, dt, tau)
    want = feq + (1 - dt / tau) ** n * (f0 - feq)
    assert np.max(np.abs(s.lbm_get_f() - want[None, :])) < 1e-14


def test_conservation_on_refined_periodic_tree_fp64():
    """Hanging faces on a periodic tree: total mass and momentum of the
    whole step are conserved to rounding."""
    c = dict(W.CONFIGS["l2_sphere_d3q19_small"])
    c.update(pred=W.PRED_BALL, solid=0, r=0.25, base_level=3, max_level=5, bc=(W.PERIODIC,) * 6,
             precision="f64")
    s, o = _pair(c)
    _, h = s.centres()
    V = h ** 3
    cv, _ = s.lbm_velocities()

    def totals(f):
        m = V @ f
        return np.array([m.sum(), *(m @ cv)])

    t0 = totals(s.lbm_get_f())
    dt = s.lbm_dt_cfl(0.4)
    s.lbm_step(10, dt, 2 * dt)
    t1 = totals(s.lbm_get_f())
    assert np.max(np.abs(t1 - t0)) < 1e-13 * t0[0]


def test_errors_are_reported():
    c = W.CONFIGS["l2_sphere_d3q19_small"]
    s, o = _pair(c)
    dt = s.lbm_dt_cfl(c["cfl"])
    with pytest.raises(D.DvmError) as e:
        s.lbm_step(1, dt, 0.5 * dt)  # dt / tau = 2
    assert e.value.code == -5
    f = s.lbm_get_f()
    f[5] = -np.abs(f[5]) * 3
    s.lbm_set_f(f)
    with pytest.raises(D.DvmError) as e:
        s.lbm_step(1, dt, 2 * dt)
    assert e.value.code == -5
    # the context stays usable
    s.lbm_set_f(np.abs(f))
    s.lbm_step(1, dt, 2 * dt)
    # a wrong lattice for the tree's dimension
    with pytest.raises(D.DvmError) as e:
        s.lbm_set_lattice(D.LBM_D2Q9)
    assert e.value.code == -1


def test_refine_keeps_lattice_and_clears_f():
    c = W.CONFIGS["l2_sphere_d3q19_small"]
    s, o = _pair(c)
    flags = np.zeros(s.nleaves, dtype=np.uint8)
    flags[:8] = 1
    s.refine(flags)
    with pytest.raises(D.DvmError) as e:
        s.lbm_step(1, 1e-3, 1e-2)
    assert e.value.code == -4
    xyz, _ = s.centres()
    rho, u = W.lbm_initial_state(c, xyz)
    s.lbm_init(rho, u)
    s.lbm_step(1, s.lbm_dt_cfl(0.4), 1.0)
