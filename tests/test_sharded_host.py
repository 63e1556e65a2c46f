"""The sharded step's exchange on two and three gloo ranks (no GPU): the
per-rank plan of the library (dvm_rank_plan, host work) and the exchange of
paper_1503_00707_gb300.sharded (the same HaloExchange that moves the packed
device rows over NCCL), run on host rows.

Each rank fills its owned rows with a code of (global cell, column) and its
halo rows with -1; after one exchange every halo row must hold the code of
the cell it stands for, and the owned rows must be untouched.  The plan is
checked against an independent statement: a rank's halo is the set of
off-range cells its upwind stencils read, the cells a rank sends to a peer
are exactly those among the peer's halo that it owns, and the plans of the
two sides of every pair agree (what one sends is what the other receives)."""
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


def _cfg(name, **over):
    c = dict(W.CONFIGS[name])
    c.update(over)
    return c


CASES = [("c2_sphere_m3", {"base_level": 3, "max_level": 5}), ("c1_2d_bump", {})]


@pytest.mark.parametrize("name,over", CASES)
@pytest.mark.parametrize("world", [2, 3])
def test_plans_of_all_ranks_agree(name, over, world):
    c = _cfg(name, **over)
    ranks = [D.Rank(c, "f32", D.COLL_BGK, world, p, device=False) for p in range(world)]
    s = D.Solver(D.F32, D.COLL_BGK, 0.1)
    s.build_tree(D.tree_spec(c["dim"], c["base_level"], c["max_level"], c["pred"], c["c"], c["r"],
                             c["beta"], c["solid"], c["bc"]))
    for p, r in enumerate(ranks):
        c0, c1, ghosts = s.partition_info(world, p)
        assert (r.c0, r.c1, r.nhalo) == (c0, c1, len(ghosts))
        got = np.sort(np.concatenate([r.plan(q)[1] for q in range(world) if q != p]))
        assert np.array_equal(got, ghosts)
        for q in range(world):
            if q == p:
                continue
            send, recv = r.plan(q)
            # what p sends to q is what q receives from p
            assert np.array_equal(send, ranks[q].plan(p)[1])
            assert np.all((send >= r.c0) & (send < r.c1))
            assert np.all((recv >= ranks[q].c0) & (recv < ranks[q].c1))


def _free_port():
    with socket.socket() as sk:
        sk.bind(("127.0.0.1", 0))
        return sk.getsockname()[1]


def _rank_main(rank, world, port, name, out):
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        from paper_1503_00707_gb300 import sharded
        c = _cfg(name, **dict(CASES)[name])
        r = D.Rank(c, "f32", D.COLL_BGK, world, rank, device=False)
        k = 6
        rows = np.full((r.ncells + r.nhalo + 1, k), -1.0)
        own = np.arange(r.c0, r.c1)
        rows[:r.ncells] = own[:, None] * 10.0 + np.arange(k)[None, :]
        sharded.host_rows_exchange(r, rows)
        halo = np.sort(np.concatenate([r.plan(q)[1] for q in range(world) if q != rank]))
        ok_halo = np.array_equal(rows[r.ncells:r.ncells + r.nhalo], halo[:, None] * 10.0 + np.arange(k)[None, :])
        ok_own = np.array_equal(rows[:r.ncells], own[:, None] * 10.0 + np.arange(k)[None, :])
        out[rank] = (bool(ok_halo), bool(ok_own), int(r.nhalo))
    finally:
        dist.destroy_process_group()


@pytest.mark.parametrize("world", [2, 3])
def test_halo_rows_arrive_on_gloo_ranks(world):
    import torch.multiprocessing as mp
    with mp.get_context("spawn").Manager() as mgr:
        out = mgr.dict()
        mp.spawn(_rank_main, args=(world, _free_port(), "c2_sphere_m3", out), nprocs=world, join=True)
        res = dict(out)
    assert sorted(res) == list(range(world))
    for rank, (ok_halo, ok_own, nh) in res.items():
        assert ok_own, rank
        assert nh > 0 and ok_halo, (rank, nh)
