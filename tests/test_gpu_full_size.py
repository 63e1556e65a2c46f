"""The Mach-5 sphere flow at its full size (1,014,080 cells x 13,824 velocities,
the bench's workload) against the oracle on sampled cells: the GPU steps the
whole tree; the oracle steps only the sample, from the rows its face
neighbourhood reads (tests/sampling.py).  The sample covers wall, inflow and
outflow faces and level changes, as well as seeded random cells."""
import numpy as np
import pytest

import paper_1503_00707_gb300 as D
import workloads as W
from tests.gpu_util import pair, rel_linf
from tests.sampling import cell_sample, oracle_rows_after, oracle_sparse_for

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def gpu():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA GPU")
    from paper_1503_00707_gb300 import _build
    _build.build()


@pytest.mark.parametrize("prec,tol,tol_rho", [("f32", 1e-5, 1e-5), ("bf16", 2e-2, 1e-2)])
def test_mach5_full_size_sampled_cells(prec, tol, tol_rho):
    """Two BGK steps from per-cell random two-beam states (every cell away
    from equilibrium); the per-element error on the sampled rows, relative
    to their largest value, within the storage precision's bound.  FP32:
    1e-5.  BF16 keeps 8 significant bits (unit roundoff u = 2^-8); an element
    is rounded five times on the way (the initial state, then per step f*
    parked in shared memory and the stored result), each a relative error
    below u, and transport and relaxation are convex combinations, so the
    per-element bound is 5u = 1.95e-2.  The sampled densities, sums of
    independently rounded values, stay within the 1e-2 of the other BF16
    field checks."""
    c = dict(W.CONFIGS["c3_sphere_m5"], init="bimodal")
    s = D.solver_from_config(c, {"f32": D.F32, "bf16": D.BF16}[prec], D.COLL_BGK)
    try:
        o = oracle_sparse_for(c)
        assert s.ncells == o.ncells == 1014080 and s.nv == o.nv == 13824
        xyz, _ = s.centres()
        xo, _ = o.centres()
        assert np.array_equal(xyz, xo)
        init = W.initial_state(c, xo)
        s.init_maxwellian(*init)
        dt = o.dt_cfl(c["cfl"])
        cells = cell_sample(o, 96, 24, seed=11)
        s.step(2, dt)
        got = s.get_f_rows(cells)
        want = oracle_rows_after(o, cells, init, 2, dt, c["kn"])
        assert rel_linf(got, want) < tol
        # the density of each sampled cell, from its rows
        rho_g, rho_o = got.sum(1) * o.dV, want.sum(1) * o.dV
        assert np.max(np.abs(rho_g - rho_o) / rho_o) < tol_rho
    finally:
        s.close()


def test_row_gather_equals_full_copy():
    """dvm_get_f_rows gives exactly the rows of dvm_get_f, repeats and any
    order allowed; an index out of range is refused (DVM_EINVAL)."""
    c = dict(W.CONFIGS["c3_sphere_m5_small"], init="bimodal")
    s, _ = pair(c, collision=D.COLL_BGK)
    try:
        s.step(1, s.dt_cfl(0.4))
        f = s.get_f()
        cells = np.array([s.ncells - 1, 0, 17, 17, 5000, 3], dtype=np.int64)
        assert np.array_equal(s.get_f_rows(cells), f[cells])
        assert s.get_f_rows(np.zeros(0, dtype=np.int64)).shape == (0, s.nv)
        with pytest.raises(D.DvmError) as e:
            s.get_f_rows(np.array([0, s.ncells]))
        assert e.value.code == -1
    finally:
        s.close()
