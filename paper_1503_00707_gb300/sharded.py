"""The step sharded over processes, one per GPU (paper Sec. 3.3).

Each rank owns a contiguous Morton range of the cells (dvm_rank_*: its own
cells, its halo and the inflow ghost on its device).  Before every step the
ranks exchange the rows of their upwind halos: the library packs the rows a
peer needs into a flat device buffer and unpacks the rows received; this
module only moves those buffers with torch.distributed point-to-point
operations (NCCL between GPUs, gloo on the CPU) and makes the step's two
global reductions, the CFL time step (minimum over ranks) and the conserved
totals (sum over ranks).  No kernel reads another GPU's memory.
"""
import numpy as np

from . import Rank


class HaloExchange:
    """One rank's exchange pattern: per peer, a send buffer of the rows the
    peer's stencils read and a receive buffer for the halo rows the peer
    owns (row_bytes bytes per row, in the order of the library's plan, so
    that the buffer a rank sends is the one its peer unpacks).

    run(pack, unpack) fills the send buffers (pack(peer, buf)), makes one
    round of non-blocking sends and receives, and hands each received buffer
    to unpack(peer, buf)."""

    def __init__(self, counts, row_bytes, device):
        import torch
        self.send = {q: torch.empty(ns * row_bytes, dtype=torch.uint8, device=device)
                     for q, (ns, nr) in sorted(counts.items()) if ns}
        self.recv = {q: torch.empty(nr * row_bytes, dtype=torch.uint8, device=device)
                     for q, (ns, nr) in sorted(counts.items()) if nr}

    def run(self, pack, unpack, group=None):
        import torch.distributed as dist
        for q, buf in self.send.items():
            pack(q, buf)
        ops = [dist.P2POp(dist.isend, buf, q, group) for q, buf in self.send.items()]
        ops += [dist.P2POp(dist.irecv, buf, q, group) for q, buf in self.recv.items()]
        if ops:
            for req in dist.batch_isend_irecv(ops):
                req.wait()
        for q, buf in self.recv.items():
            unpack(q, buf)


class ShardedSolver:
    """The DVM step on the calling rank's Morton range of workload `cfg`, in
    the process group `group` (default: the world).  The library's stream is
    the current torch stream, so that the NCCL transfers are ordered after the
    packing kernels and before the unpacking ones."""

    def __init__(self, cfg, precision, collision, kn=None, group=None):
        import torch
        import torch.distributed as dist
        self.group = group
        self.world = dist.get_world_size(group)
        self.rank_id = dist.get_rank(group)
        self.stream = torch.cuda.current_stream()
        self.r = Rank(cfg, precision, collision, self.world, self.rank_id, kn=kn, stream=self.stream)
        counts = {}
        for q in range(self.world):
            if q != self.rank_id:
                s, r = self.r.plan(q)
                counts[q] = (len(s), len(r))
        self.ex = HaloExchange(counts, self.r.row_bytes, "cuda")
        self.ncells = self.r.ncells
        self.nv = self.r.nv

    def exchange(self):
        self.ex.run(lambda q, b: self.r.pack(q, b.data_ptr()), lambda q, b: self.r.unpack(q, b.data_ptr()),
                    self.group)

    def step(self, nsteps, dt):
        for _ in range(nsteps):
            self.exchange()
            self.r.step(dt)

    def dt_cfl(self, cfl):
        import torch
        import torch.distributed as dist
        t = torch.tensor([self.r.dt_cfl(cfl)], dtype=torch.float64, device="cuda")
        dist.all_reduce(t, op=dist.ReduceOp.MIN, group=self.group)
        return float(t.item())

    def totals(self):
        import torch
        import torch.distributed as dist
        t = torch.tensor(self.r.totals(), dtype=torch.float64, device="cuda")
        dist.all_reduce(t, op=dist.ReduceOp.SUM, group=self.group)
        return t.cpu().numpy()

    def close(self):
        self.r.close()


def host_rows_exchange(rank, rows, group=None):
    """The exchange of ShardedSolver on host rows (no device): rows is the
    rank's local array [owned + halo + 1][k] (owned cells, then the halo in
    ascending global order, then the inflow ghost).  The rows the plan sends
    are gathered from the owned block, the rows received scattered into the
    halo block, over the group's backend (gloo).  Returns rows."""
    world = rank.nparts
    c0, nown = rank.c0, rank.ncells
    halo = np.concatenate([rank.plan(q)[1] for q in range(world) if q != rank.part] + [np.zeros(0, np.int64)])
    halo.sort()
    counts, send_rows, recv_rows = {}, {}, {}
    for q in range(world):
        if q == rank.part:
            continue
        s, r = rank.plan(q)
        counts[q] = (len(s), len(r))
        send_rows[q] = s - c0
        recv_rows[q] = nown + np.searchsorted(halo, r)
    row_bytes = rows.shape[1] * rows.itemsize
    ex = HaloExchange(counts, row_bytes, "cpu")

    def pack(q, buf):
        buf.numpy()[:] = np.ascontiguousarray(rows[send_rows[q]]).view(np.uint8).ravel()

    def unpack(q, buf):
        rows[recv_rows[q]] = buf.numpy().view(rows.dtype).reshape(-1, rows.shape[1])

    ex.run(pack, unpack, group)
    return rows
