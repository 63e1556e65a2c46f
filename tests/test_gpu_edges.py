"""Edge cases of the step on the GPU against the oracle: trees with fewer cells
than the GPU has CTAs (every CTA's first slots partly or wholly empty), the
smallest trees (4 cells in 2D, 8 in 3D), velocity grids whose quads leave
part of a warp idle (a ragged last warp), and grids larger than one CTA can
hold (refused on the host)."""
import numpy as np
import pytest

import oracle as O
import paper_1503_00707_gb300 as D
import workloads as W
from tests.gpu_util import field_errors, pair, rel_linf

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def gpu():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA GPU")
    from paper_1503_00707_gb300 import _build
    _build.build()


def _box(dim, level, n, vmax, precision, init="bimodal"):
    """A uniform periodic box at one level, from per-cell random two-beam
    states, BGK Kn 0.2 (nu dt below 1 at the CFL step); n is the velocity grid
    (nx, ny, nz)."""
    c = dict(W.CONFIGS["c4_hs_bimodal"])
    c.update(dim=dim, base_level=level, max_level=level, pred=O.PRED_NONE, n=tuple(n), lo=(-vmax,) * 3,
             hi=(vmax,) * 3, coll=D.COLL_BGK, kn=0.2, precision=precision, init=init)
    return c


@pytest.mark.parametrize("dim,level,n,vmax,prec", [
    (3, 1, (16, 16, 16), 6.0, "f32"),   # 8 cells, 16^3: fewer cells than CTAs
    (3, 1, (24, 24, 24), 8.0, "f32"),   # 8 cells, 24^3 (the throughput kernel)
    (2, 1, (8, 8, 8), 4.0, "f64"),      # 4 cells, FP64
    (3, 2, (12, 12, 16), 5.0, "f32"),   # 64 cells, 72 quads per group: the last warp 3/4 idle
    (3, 2, (20, 20, 8), 7.0, "f32"),    # 64 cells, 100 quads per group
])
def test_small_trees_match_oracle(dim, level, n, vmax, prec):
    c = _box(dim, level, n, vmax, prec)
    s, o = pair(c, collision=D.COLL_BGK)
    assert s.ncells == (2 ** dim) ** level
    dt = o.dt_cfl(0.4)
    s.step(5, dt)
    o.step(5, dt, O.COLL_BGK, c["kn"])
    tol = 1e-12 if prec == "f64" else 1e-5
    assert rel_linf(s.get_f(), o.get_f()) < tol
    err = field_errors(s.moments(), o.moments())
    assert max(err.values()) < tol, err


def test_small_tree_entropic_matches_oracle():
    c = _box(3, 1, (16, 16, 16), 6.0, "f32")
    s, o = pair(c, collision=D.COLL_BGK_ENTROPIC)
    dt = o.dt_cfl(0.4)
    s.step(3, dt)
    o.step(3, dt, O.COLL_BGK_ENTROPIC, c["kn"])
    assert rel_linf(s.get_f(), o.get_f()) < 1e-5


def test_repeated_steps_on_eight_cells():
    """Many launches on the smallest 3D tree: every launch's CTAs find the
    counter nearly empty at once."""
    c = _box(3, 1, (16, 16, 16), 6.0, "f32")
    s, o = pair(c, collision=D.COLL_BGK)
    dt = o.dt_cfl(0.4)
    for _ in range(10):
        s.step(5, dt)
    o.step(50, dt, O.COLL_BGK, c["kn"])
    err = field_errors(s.moments(), o.moments())
    assert max(err.values()) < 1e-5, err


def test_grid_beyond_one_cta_is_refused():
    """32^3 velocities need more transport warps than a CTA holds: refused
    on the host before any launch (DVM_ENOTIMPL); the context stays usable."""
    c = _box(3, 1, (32, 32, 32), 8.0, "f32", init="freestream")
    s = D.solver_from_config(c, D.F32, D.COLL_BGK)
    xyz, _ = s.centres()
    s.init_maxwellian(*W.initial_state(c, xyz))
    with pytest.raises(D.DvmError) as e:
        s.step(1, s.dt_cfl(0.4))
    assert e.value.code == -9
    rho, _, _ = s.moments()
    assert np.all(np.isfinite(rho))
