"""The per-rank step of the Morton-range partition (dvm_rank_*, Sec. 3.3) on
one GPU: two and three ranks, each holding only its cells, its halo and the
inflow ghost, exchange their halo rows through device buffers packed and
unpacked by the library (the buffers a multi-GPU run moves with NCCL), then
step; f, the step moments and the conserved totals must equal those of the
whole-tree dvm_step bit for bit (the per-cell arithmetic does not depend on
the partition).  The ranks run one after another on the one stream: no
kernel waits on another."""
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


def _exchange(ranks):
    import torch
    for p, rp in enumerate(ranks):
        for q, rq in enumerate(ranks):
            if p == q:
                continue
            send, _ = rp.plan(q)
            if len(send) == 0:
                continue
            buf = torch.empty(len(send) * rp.row_bytes, dtype=torch.uint8, device="cuda")
            rp.pack(q, buf.data_ptr())
            rq.unpack(p, buf.data_ptr())
    torch.cuda.synchronize()


@pytest.mark.parametrize("name,prec,coll", [("c2_sphere_m3", "f32", D.COLL_BGK),
                                            ("c3_sphere_m5_small", "bf16", D.COLL_BGK),
                                            ("c1_2d_bump", "f64", D.COLL_BGK_ENTROPIC)])
@pytest.mark.parametrize("world", [2, 3])
def test_ranks_equal_the_whole_step(name, prec, coll, world):
    c = W.CONFIGS[name]
    s = D.solver_from_config(c, prec, coll)
    xyz, _ = s.centres()
    init = W.initial_state(c, xyz)
    s.init_maxwellian(*init)
    ranks = [D.Rank(c, prec, coll, world, p) for p in range(world)]
    for r in ranks:
        sl = slice(r.c0, r.c1)
        rx, _ = r.centres()
        assert np.array_equal(rx, xyz[sl])
        r.init_maxwellian(*[np.asarray(a)[sl] for a in init])
    dt = s.dt_cfl(c["cfl"])
    assert min(r.dt_cfl(c["cfl"]) for r in ranks) == dt
    steps = 3
    for _ in range(steps):
        _exchange(ranks)
        for r in ranks:
            r.step(dt)
    s.step(steps, dt)
    f = s.get_f()
    rho, u, T = s.moments()
    for r in ranks:
        sl = slice(r.c0, r.c1)
        assert np.array_equal(r.get_f(), f[sl])
        rr, ur, Tr = r.moments()
        assert np.array_equal(rr, rho[sl]) and np.array_equal(ur, u[sl]) and np.array_equal(Tr, T[sl])
    tot = np.sum([r.totals() for r in ranks], axis=0)
    _, h = s.centres()
    V = h ** c["dim"]
    want = np.array([np.sum(V * rho)] + [np.sum(V * rho * u[:, d]) for d in range(3)] +
                    [np.sum(V * rho * ((u * u).sum(1) + 3 * T))])
    assert np.allclose(tot, want, rtol=1e-12, atol=1e-15 * abs(want[0]))
    for r in ranks:
        r.close()
    s.close()
