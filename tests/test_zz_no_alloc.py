"""The allocation-free hard-sphere entry point against the regular step.

dvm_hs_collide_noalloc serves callers that must not allocate device memory
while they run (a framework that owns all device memory through its own
pool and hands plug-ins only its buffers, a real-time loop whose memory is
sized once at start-up):
its scratch is a fixed array in the library's device image.  On a spatially
uniform periodic state the transport of Eq. 2 leaves f unchanged bit for bit,
so one dvm_step is exactly the collision update; the allocation-free call on a
caller-owned copy of f must give the same f, on two calls in a row.

This file is collected last so that a run stopping at the first failure has
already run every other test.
"""
import numpy as np
import pytest

import paper_1503_00707_gb300 as D
import workloads as W
from tests.gpu_util import oracle_for, rel_linf, storage_round

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def gpu():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA GPU")
    from paper_1503_00707_gb300 import _build
    _build.build()


def _uniform_hs_solver():
    c = dict(W.CONFIGS["c4_hs_bimodal"])
    c.update(base_level=1, max_level=1, pred=0, n=(16, 16, 16), lo=(-6.0,) * 3, hi=(6.0,) * 3)
    s = D.solver_from_config(c, D.F32, D.COLL_HS)
    s.init_maxwellian(*_bimodal(s.ncells))
    s.set_collision_tables(64, 20150303)
    return s, c


def _bimodal(nc):
    """The same two-beam state in every cell: transport is the identity."""
    u = np.zeros((nc, 2, 3))
    u[:, 0, 0], u[:, 1, 0] = 1.4, -1.2
    return np.tile([0.45, 0.55], (nc, 1)), np.ones((nc, 2)), u, np.tile([0.6, 0.7], (nc, 1))


def test_noalloc_matches_step_on_two_calls():
    import torch
    s, c = _uniform_hs_solver()
    dt = 2.5e-5  # dt/Kn max(P B) well below 1 for this state
    f0 = s.get_f()
    buf = torch.tensor(f0, dtype=torch.float32, device="cuda").contiguous()
    torch.cuda.synchronize()
    for call in range(2):
        s.step(1, dt)
        ref = s.get_f()
        s.hs_collide_noalloc(buf.data_ptr(), s.ncells, dt)
        got = buf.double().cpu().numpy()
        # the same kernels on the same values: equal up to the order of the
        # floating-point sums of the moments
        assert rel_linf(got, ref) < 1e-6, call
        assert rel_linf(got, f0) > 1e-6  # the update did something


def test_noalloc_matches_oracle_on_two_calls():
    """Against the FP64 oracle's hard-sphere update (Eqs. 3-6) from the same
    values, call after call."""
    import torch
    s, c = _uniform_hs_solver()
    o = oracle_for(c)
    o.init_maxwellian(*_bimodal(o.ncells))
    o.hs_tables(64, 20150303)
    dt = 2.5e-5
    buf = torch.empty((s.ncells, s.nv), dtype=torch.float32, device="cuda")
    for call in range(2):
        # both sides start each call from the oracle's values in FP32
        f = storage_round(o.get_f(), "f32")
        o.set_f(f)
        buf.copy_(torch.from_numpy(f.astype(np.float32)))
        torch.cuda.synchronize()
        o.hs_collide(dt, c["kn"])
        s.hs_collide_noalloc(buf.data_ptr(), s.ncells, dt)
        got = buf.double().cpu().numpy()
        assert rel_linf(got, o.get_f()) < 1e-5, call


def test_noalloc_rejects_misaligned_f():
    import torch
    s, c = _uniform_hs_solver()
    buf = torch.zeros(s.ncells * s.nv + 4, dtype=torch.float32, device="cuda")
    with pytest.raises(D.DvmError) as e:
        s.hs_collide_noalloc(buf.data_ptr() + 4, s.ncells, 1e-5)  # refused before any work is queued
    assert e.value.code == -1
    assert "aligned" in str(e.value)


def test_noalloc_rejects_sizes_beyond_the_scratch():
    s, c = _uniform_hs_solver()
    too_many = D.HS_NOALLOC_SCRATCH_BYTES // (8 * s.nv + 40) + 1
    with pytest.raises(D.DvmError) as e:
        s.hs_collide_noalloc(1 << 20, too_many, 1e-5)  # rejected before any work is queued
    assert e.value.code == -1
    assert "scratch" in str(e.value)
