"""GPU parity of the hard-sphere collision step (Eqs. 3-6) against the FP64
oracle through the C ABI: the seeded trial tables bit for bit, the collision
integral and the corrected step element by element, conservation of the
collision update, and the periodic 16^3 workload with its bimodal start."""
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


def _homog_cfg(n=16, vmax=6.0, base=2):
    c = dict(W.CONFIGS["c4_hs_bimodal"])
    c.update(base_level=base, max_level=base, pred=O.PRED_NONE, n=(n, n, n), lo=(-vmax,) * 3, hi=(vmax,) * 3)
    return c


@pytest.mark.parametrize("lattice", [False, True])
def test_tables_match_oracle(lattice):
    c = _homog_cfg(n=16)
    s, o = pair(c, init=False)
    M, seed = 64, 20150303
    s.set_collision_tables(M, seed, lattice=lattice)
    o.hs_tables(M, seed, lattice=lattice)
    gam, l, m, b, disc = s.collision_tables(M)
    start, og, ol, om, ob, odisc = o.hs_get_tables()
    assert disc == odisc
    nv = o.nv
    # a trial with gamma = i has |g| = 0 and b = 0, like a discarded one: compare
    # the trials that carry weight, in order
    for i in range(nv):
        sl = slice(start[i], start[i + 1])
        ko = ob[sl] != 0
        row = slice(i * M, (i + 1) * M)
        ks = b[row] != 0
        assert ko.sum() == ks.sum()
        assert np.array_equal(gam[row][ks], og[sl][ko])
        assert np.array_equal(l[row][ks], ol[sl][ko])
        assert np.array_equal(m[row][ks], om[sl][ko])
        ref = ob[sl][ko].astype(np.float32)
        assert np.all(np.abs(b[row][ks] - ref) <= np.spacing(ref))


@pytest.mark.parametrize("M", [32, 128])
def test_homogeneous_bimodal_step(M):
    c = _homog_cfg(n=16)
    s, o = pair(c)
    s.set_collision_tables(M, 7)
    o.hs_tables(M, 7)
    # the seeded bimodal start has max(P B) ~ 360 at 32 trials (in the far
    # tails): dt/Kn max(P B) ~ 0.45 keeps the explicit loss term positive
    dt = 2.5e-5
    f0 = s.get_f()
    s.step(1, dt)
    o.step(1, dt, O.COLL_HS, c["kn"])
    # the collision update conserves each cell's moments: those of the stored
    # f^{n+1} against those of the step's f* (FP32 arithmetic and storage)
    rs, us, Ts = s.step_moments()
    r1, u1, T1 = s.moments()
    assert rel_linf(r1, rs) < 1e-6 and np.max(np.abs(u1 - us)) < 1e-5 and rel_linf(T1, Ts) < 1e-5
    s.step(2, dt)
    o.step(2, dt, O.COLL_HS, c["kn"])
    fs, fo = s.get_f(), o.get_f()
    assert rel_linf(fs, fo) < 2e-5
    # and it did something
    assert rel_linf(fs, f0) > 1e-5


@pytest.mark.parametrize("M", [32, 64])
def test_24_cubed_grid_few_trials(M):
    """The 24^3 grid runs the 512-thread gather CTAs; with 32 and 64 trials a
    node has one or two lanes (128 and 256 nodes per CTA).  A periodic box of
    8 cells from per-cell two-beam states, two steps against the oracle."""
    c = _homog_cfg(n=24, vmax=8.0, base=1)
    s, o = pair(c)
    s.set_collision_tables(M, 11)
    o.hs_tables(M, 11)
    # the random two-beam start reaches max(P B) of several thousand in the
    # far tails of [-8,8]^3 with few trials (1e-5 was refused at 32 trials):
    # dt/Kn = 1.25e-4
    dt = 2.5e-6
    f0 = o.get_f()
    s.step(2, dt)
    o.step(2, dt, O.COLL_HS, c["kn"])
    fo = o.get_f()
    assert rel_linf(s.get_f(), fo) < 2e-5
    assert rel_linf(fo, f0) > 1e-4  # the two steps moved f well beyond the bar
    err = field_errors(s.moments(), o.moments())
    assert max(err.values()) < 1e-5, err


def test_c4_hs_bimodal_two_steps():
    c = W.CONFIGS["c4_hs_bimodal"]
    s, o = pair(c)
    s.set_collision_tables(c["trials"], W.SEED)
    o.hs_tables(c["trials"], W.SEED)
    # at Kn = 0.02 the bimodal start has max(P B) ~ 290 (in the far tails), so
    # the CFL step would violate dt/Kn max(P B) <= 1; a sixteenth of it keeps
    # the explicit loss term positive
    dt = o.dt_cfl(c["cfl"]) / 16
    f0 = o.get_f()
    s.step(2, dt)
    o.step(2, dt, O.COLL_HS, c["kn"])
    fs, fo = s.get_f(), o.get_f()
    assert rel_linf(fs, fo) < 1e-5
    assert rel_linf(fo, f0) > 1e-3
    err = field_errors(s.moments(), o.moments())
    assert max(err.values()) < 1e-5, err


def test_hs_needs_tables_and_fp32():
    c = _homog_cfg(n=8)
    s, o = pair(c)
    with pytest.raises(D.DvmError) as e:
        s.step(1, 1e-3)
    assert e.value.code == -4
    c2 = dict(c)
    c2["precision"] = "f64"
    s2, _ = pair(c2)
    with pytest.raises(D.DvmError) as e:
        s2.set_collision_tables(64, 1)
    assert e.value.code == -9


def test_lattice_tables_hs_step_matches_oracle():
    """Hard-sphere steps with the Korobov-lattice trials: the same collision
    operator with other tables, so the same parity bar as the random ones."""
    c = _homog_cfg(n=16)
    s, o = pair(c)
    M = 64
    s.set_collision_tables(M, 11, lattice=True)
    o.hs_tables(M, 11, lattice=True)
    dt = 2.5e-5
    s.step(2, dt)
    o.step(2, dt, O.COLL_HS, c["kn"])
    assert rel_linf(s.get_f(), o.get_f()) < 2e-5
    err = field_errors(s.moments(), o.moments())
    assert max(err.values()) < 1e-5, err
