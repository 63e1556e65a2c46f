"""The partitioned step (Morton ranges with an upwind-halo exchange before
every step, each part run by the step kernel on its own buffers, Sec. 3.3)
against the unpartitioned step on the GPU: f and the step moments must agree
bit for bit, since every cell sees the same inputs and the same arithmetic."""
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


def _solver(c, precision, coll=D.COLL_BGK):
    s = D.solver_from_config(c, precision, coll)
    xyz, _ = s.centres()
    s.init_maxwellian(*W.initial_state(c, xyz))
    return s


@pytest.mark.parametrize("name,precision,nparts,steps,coll", [
    ("c1_2d_bump", D.F64, 3, 10, D.COLL_BGK),           # periodic quadtree: halos wrap around
    ("c2_sphere_m3", D.F32, 5, 6, D.COLL_BGK),          # walls, inflow, outflow, 16^3
    ("c3_sphere_m5_small", D.F32, 4, 3, D.COLL_BGK),    # the 24^3 Mach-5 flow
    ("c3_sphere_m5_small", D.BF16, 2, 3, D.COLL_BGK),
    ("c2_sphere_m3", D.F32, 3, 4, D.COLL_BGK_ENTROPIC),
])
def test_partitioned_step_is_bit_identical(name, precision, nparts, steps, coll):
    c = W.CONFIGS[name]
    a, b = _solver(c, precision, coll), _solver(c, precision, coll)
    dt = a.dt_cfl(c["cfl"])
    a.step(steps, dt)
    b.step_partitioned(nparts, steps, dt)
    assert np.array_equal(a.get_f(), b.get_f())
    for x, y in zip(a.step_moments(), b.step_moments()):
        assert np.array_equal(x, y)
    a.close()
    b.close()


def test_partitioned_step_rejects_other_collisions():
    c = dict(W.CONFIGS["c4_hs_bimodal"])
    c.update(base_level=2, max_level=2)
    s = D.solver_from_config(c, D.F32, D.COLL_HS)
    xyz, _ = s.centres()
    s.init_maxwellian(*W.initial_state(c, xyz))
    with pytest.raises(D.DvmError) as e:
        s.step_partitioned(2, 1, 1e-4)
    assert e.value.code == -9
    s.close()
