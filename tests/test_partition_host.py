"""The Morton-range partition and its upwind halo on the host (no GPU).

The multi-GPU decomposition of the step (paper Sec. 3.3) splits the
Morton-ordered cells into contiguous ranges of equal work; a range's halo is
the cells outside it that its advection stencils read.  The stencils of a
cell read its face neighbours (every face is upwind for half of the sign
groups), so the halo of a range must be exactly the set of cells outside the
range that share a face with a cell inside it.  The exchange protocol runs
on two gloo ranks: each rank asks the other for its halo cells and checks
what it receives, then makes the step's two global reductions: the CFL time
step (minimum over ranks) and the five conservation totals (sum over
ranks)."""
import os
import socket

import numpy as np
import pytest

import paper_1503_00707_gb300 as D
import workloads as W
from paper_1503_00707_gb300 import _build


@pytest.fixture(scope="module", autouse=True)
def built():
    _build.build()


def _mesh(name, **over):
    c = dict(W.CONFIGS[name])
    c.update(over)
    s = D.Solver(D.F32, D.COLL_BGK, 0.1)
    s.build_tree(D.tree_spec(c["dim"], c["base_level"], c["max_level"], c["pred"], c["c"], c["r"],
                             c["beta"], c["solid"], c["bc"]))
    return s


def _cell_faces(s):
    """Interior faces as pairs of cell indices."""
    keys, levels, solid = s.leaves()
    cell_of_leaf = np.cumsum(solid == 0) - 1
    cell_of_leaf[solid != 0] = -1
    fm, fp, _, _ = s.faces()
    return cell_of_leaf[fm], cell_of_leaf[fp]


def _expected_halo(s, c0, c1):
    a, b = _cell_faces(s)
    own_a, own_b = (a >= c0) & (a < c1), (b >= c0) & (b < c1)
    return np.unique(np.concatenate([b[own_a & ~own_b], a[own_b & ~own_a]]))


@pytest.mark.parametrize("name,over,nparts", [
    ("c1_2d_bump", {}, 3),                                   # periodic quadtree, hanging faces
    ("c2_sphere_m3", {"base_level": 3, "max_level": 5}, 5),  # walls, inflow, outflow
    ("c4_hs_bimodal", {"base_level": 3, "max_level": 4}, 4),  # periodic octree
])
def test_halo_is_the_off_range_face_neighbours(name, over, nparts):
    s = _mesh(name, **over)
    prev = 0
    sizes = []
    for p in range(nparts):
        c0, c1, g = s.partition_info(nparts, p)
        assert c0 == prev and c1 > c0
        prev = c1
        sizes.append(c1 - c0)
        assert np.all(np.diff(g) > 0)
        assert np.array_equal(g, _expected_halo(s, c0, c1))
    assert prev == s.ncells
    assert max(sizes) - min(sizes) <= 1
    s.close()


@pytest.mark.parametrize("nparts", [2, 3, 7])
def test_weighted_partition_balances_the_cost(nparts):
    """Kinetic cells (inside a ball, cost 1) far heavier than fluid ones
    (cost 0.02): the ranges tile the cells in Morton order, every cut lies
    within half the largest weight of its target, and each range's halo is
    still its off-range face neighbours."""
    s = _mesh("c2_sphere_m3", base_level=3, max_level=5)
    xyz, _ = s.centres()
    kinetic = ((xyz - np.array([0.35, 0.5, 0.5])) ** 2).sum(axis=1) < 0.2 ** 2
    w = np.where(kinetic, 1.0, 0.02)
    Wt = w.sum()
    prev = 0
    for p in range(nparts):
        c0, c1, g = s.partition_weighted(nparts, p, w)
        assert c0 == prev and c1 > c0
        prev = c1
        if p < nparts - 1:
            assert abs(w[:c1].sum() - Wt * (p + 1) / nparts) <= 0.5 * w.max() + 1e-9
        assert np.array_equal(g, _expected_halo(s, c0, c1))
    assert prev == s.ncells
    # equal weights give ranges within one cell of each other
    sizes = [np.subtract(*s.partition_weighted(nparts, p, np.ones(s.ncells))[1::-1]) for p in range(nparts)]
    assert max(sizes) - min(sizes) <= 1
    with pytest.raises(D.DvmError):
        s.partition_weighted(nparts, 0, -w)
    s.close()


def test_partition_rejects_bad_arguments():
    s = _mesh("c1_2d_bump")
    for nparts, part in ((0, 0), (2, 2), (2, -1), (s.ncells + 1, 0)):
        with pytest.raises(D.DvmError) as e:
            s.partition_info(nparts, part)
        assert e.value.code == -1
    s.close()


def _free_port():
    with socket.socket() as so:
        so.bind(("127.0.0.1", 0))
        return so.getsockname()[1]


def _rank(rank, world, port, out):
    import torch
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        s = _mesh("c2_sphere_m3", base_level=3, max_level=5)
        xyz, _ = s.centres()
        c0, c1, halo = s.partition_info(world, rank)
        peer = 1 - rank
        # 1. tell the peer how many and which halo cells this rank needs
        n = torch.tensor([halo.size], dtype=torch.int64)
        m = torch.zeros(1, dtype=torch.int64)
        reqs = [dist.isend(n, peer), dist.irecv(m, peer)]
        for r in reqs:
            r.wait()
        want = torch.from_numpy(halo.copy())
        asked = torch.zeros(int(m.item()), dtype=torch.int64)
        reqs = [dist.isend(want, peer), dist.irecv(asked, peer)]
        for r in reqs:
            r.wait()
        # 2. answer with the owned cells' data (here: their centres)
        a = asked.numpy()
        ok_owned = bool(np.all((a >= c0) & (a < c1)))
        reply = torch.from_numpy(np.ascontiguousarray(xyz[a]))
        got = torch.zeros((halo.size, 3), dtype=torch.float64)
        reqs = [dist.isend(reply, peer), dist.irecv(got, peer)]
        for r in reqs:
            r.wait()
        # 3. the step's global reductions: the CFL time step (min over ranks)
        #    and the five conservation totals (sum over ranks)
        _, h = s.centres()
        xi_max = 6.0 - 0.375                  # the 16^3 grid on [-6, 6]: largest |node|
        smax = 3 * xi_max
        dt_loc = torch.tensor([0.4 * float(h[c0:c1].min()) / smax], dtype=torch.float64)
        dist.all_reduce(dt_loc, op=dist.ReduceOp.MIN)
        ok_dt = float(dt_loc.item()) == 0.4 * float(h.min()) / smax
        V = h ** 3
        q = np.stack([1 + 0.1 * np.sin(7 * xyz[:, 0]), np.cos(3 * xyz[:, 1]), xyz[:, 2] ** 2,
                      xyz[:, 0] * xyz[:, 1], 1.5 + xyz[:, 2]], axis=1)
        tot = torch.from_numpy((V[c0:c1, None] * q[c0:c1]).sum(axis=0))
        dist.all_reduce(tot, op=dist.ReduceOp.SUM)
        want = (V[:, None] * q).sum(axis=0)
        ok_tot = bool(np.allclose(tot.numpy(), want, rtol=1e-13, atol=0))
        out[rank] = (ok_owned and ok_dt and ok_tot, bool(np.array_equal(got.numpy(), xyz[halo])), int(halo.size))
        s.close()
    finally:
        dist.destroy_process_group()


def test_halo_exchange_on_two_gloo_ranks():
    import torch.multiprocessing as mp
    world = 2
    with mp.get_context("spawn").Manager() as mgr:
        out = mgr.dict()
        mp.spawn(_rank, args=(world, _free_port(), out), nprocs=world, join=True)
        res = dict(out)
    for r in range(world):
        ok_owned, ok_data, n = res[r]
        assert ok_owned and ok_data and n > 0
