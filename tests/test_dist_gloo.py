"""Multi-rank host logic on CPU (gloo, world size 2): cells sharded across
ranks with no data exchange, per-cell results gathered, the job time taken as
the maximum over ranks.  Each rank runs its own cells through the oracle (no
GPU here); the gathered flow-curve points must equal a single-process run
bit for bit, since cells are independent."""
import os
import socket

import numpy as np
import pytest

from paper_1004_5058_gb300 import dist as D
from paper_1004_5058_gb300 import inputs as I


def cells_and_fields():
    cells = [I.make_cell("paper", nx=16, ny=12, g_ab=0.405, bc=1, u_wall=u) for u in (2e-3, 5e-3, 1e-2, 2e-2, 3e-2)]
    ra, rb = I.random_fields(16, 12, n_cells=len(cells), seed=77)
    ux, uy = I.couette_velocity(16, 12, [c.u_wall for c in cells], n_cells=len(cells))
    return cells, ra, rb, ux, uy


def run_cells(idx):
    from oracle import lb as orc
    cells, ra, rb, ux, uy = cells_and_fields()
    out = []
    for c in idx:
        r = orc.Run(cells[c], ra[c], rb[c], ux[c], uy[c], threads=1)
        r.set_sampling(10, 2)
        r.step(30)
        s, S, Sb, _ = r.shear()
        out.append([s, S, Sb])
    return np.array(out).reshape(-1, 3)


def _worker(rank, world, port, outdir):
    import torch.distributed as dist
    dist.init_process_group("gloo", init_method="tcp://127.0.0.1:%d" % port, rank=rank, world_size=world)
    n = len(cells_and_fields()[0])
    mine = D.shard(n, rank, world)
    local = run_cells(list(mine))
    allrows = D.gather_rows(local, n)
    tmax = D.max_over_ranks(1.5 + rank)
    np.save(os.path.join(outdir, "rows_%d.npy" % rank), allrows)
    np.save(os.path.join(outdir, "tmax_%d.npy" % rank), np.array([tmax, len(mine)]))
    dist.barrier()
    dist.destroy_process_group()


def free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def test_shard_covers_once():
    for n in (0, 1, 5, 8, 64, 65):
        for w in (1, 2, 3, 8):
            got = [i for r in range(w) for i in D.shard(n, r, w)]
            assert got == list(range(n))
            sizes = [len(D.shard(n, r, w)) for r in range(w)]
            assert max(sizes) - min(sizes) <= 1
    with pytest.raises(ValueError):
        D.shard(4, 2, 2)


def test_two_ranks_gloo(tmp_path):
    import torch.multiprocessing as mp
    world = 2
    mp.spawn(_worker, args=(world, free_port(), str(tmp_path)), nprocs=world, join=True)
    ref = run_cells(range(len(cells_and_fields()[0])))
    for r in range(world):
        rows = np.load(tmp_path / ("rows_%d.npy" % r))
        assert np.array_equal(rows, ref)  # independent cells: bitwise equal
        tmax, n_local = np.load(tmp_path / ("tmax_%d.npy" % r))
        assert tmax == 2.5
    assert D.job_rate([3, 2], 2.5) == 2.0


# ---- one cell split into slabs over gloo ranks ------------------------------
def _slab_worker(rank, world, port, outdir, bc):
    import torch
    import torch.distributed as dist
    from oracle import slab
    from tests.test_oracle_slab import case
    dist.init_process_group("gloo", init_method="tcp://127.0.0.1:%d" % port, rank=rank, world_size=world)
    cell, f = case(bc)
    y0, rows = slab.split_rows(cell.ny, world)[rank]
    below, above = slab.neighbours(cell, rank, world)
    mine = slab.scatter(f, y0, rows)

    def trade(to_below, to_above):
        """Send to the neighbours, receive from them; tag 1 travels down, tag 2 up."""
        reqs, got = [], [None, None]
        if below is not None:
            reqs.append(dist.isend(torch.from_numpy(to_below), below, tag=1))
            got[0] = torch.empty(to_above.shape, dtype=torch.float64)
            reqs.append(dist.irecv(got[0], below, tag=2))
        if above is not None:
            reqs.append(dist.isend(torch.from_numpy(to_above), above, tag=2))
            got[1] = torch.empty(to_below.shape, dtype=torch.float64)
            reqs.append(dist.irecv(got[1], above, tag=1))
        for q in reqs:
            q.wait()
        return [None if g is None else g.numpy() for g in got]

    for _ in range(12):
        fb, fa = trade(*slab.ghost_send(mine))
        slab.ghost_recv(mine, fb, fa)
        out, _ = slab.step_slab(cell, y0, mine)
        fb, fa = trade(*slab.outflow_send(out))
        slab.inflow_recv(out, fb, fa)
        mine = out
    np.save(os.path.join(outdir, "slab_%d.npy" % rank), mine[:, :, 2:rows + 2])
    dist.barrier()
    dist.destroy_process_group()


@pytest.mark.parametrize("bc", [0, 1], ids=["periodic", "couette"])
def test_slab_ranks_gloo(tmp_path, bc):
    """Two gloo ranks each step one slab of a cell and trade rows over
    send/recv: the joined state equals the whole-cell oracle bit for bit."""
    import torch.multiprocessing as mp
    from oracle import lb, slab
    from tests.test_oracle_slab import case
    world = 2
    mp.spawn(_slab_worker, args=(world, free_port(), str(tmp_path), bc), nprocs=world, join=True)
    cell, f = case(bc)
    for _ in range(12):
        f, _, _ = lb.step(cell, f)
    got = np.concatenate([np.load(tmp_path / ("slab_%d.npy" % r)) for r in range(world)], axis=2)
    assert np.array_equal(got, f)


# ---- the package's rank-to-rank slab exchange, driving oracle slabs ---------
class _OracleSlab:
    """An FP64 oracle slab (orc_step_slab) behind the slab interface that
    paper_1004_5058_gb300.slabs exchanges messages for (get / put / step / empty);
    messages are CPU tensors here, device buffers on GPUs."""

    def __init__(self, cell, y0, rows, f):
        from oracle import slab
        self.slab, self.cell, self.y0, self.rows = slab, cell, y0, rows
        self.f = slab.scatter(f, y0, rows)

    def _where(self, part, put):
        from paper_1004_5058_gb300.slabs import EDGE_HI, EDGE_LO, FLOW_LO
        r = self.rows
        if part in (EDGE_LO, EDGE_HI):
            lo = part == EDGE_LO
            rows = (slice(0, 2) if lo else slice(r + 2, r + 4)) if put else (slice(2, 4) if lo else slice(r, r + 2))
            return (slice(None), slice(None), rows)
        lo = part == FLOW_LO
        planes = list(self.slab.UP if lo == put else self.slab.DOWN)
        row = (2 if lo else r + 1) if put else (1 if lo else r + 2)
        return (slice(None), planes, row)

    def get(self, part):
        import torch
        return torch.from_numpy(np.ascontiguousarray(self.f[self._where(part, False)]))

    def empty(self, part):
        import torch
        return torch.empty(self.f[self._where(part, True)].shape, dtype=torch.float64)

    def put(self, part, msg):
        self.f[self._where(part, True)] = msg.numpy()

    def step(self):
        self.f, _ = self.slab.step_slab(self.cell, self.y0, self.f)


def _dist_exchange_worker(rank, world, port, outdir, bc):
    import torch.distributed as dist
    from paper_1004_5058_gb300.slabs import DistExchange, split_rows
    from tests.test_oracle_slab import case
    dist.init_process_group("gloo", init_method="tcp://127.0.0.1:%d" % port, rank=rank, world_size=world)
    cell, f = case(bc)
    y0, rows = split_rows(cell.ny, world)[rank]
    s = _OracleSlab(cell, y0, rows, f)
    DistExchange(s, rank, world, periodic=cell.bc == 0).step(12)
    np.save(os.path.join(outdir, "dx_%d.npy" % rank), s.f[:, :, 2:rows + 2])
    dist.barrier()
    dist.destroy_process_group()


@pytest.mark.parametrize("world", [2, 3])
@pytest.mark.parametrize("bc", [0, 1], ids=["periodic", "couette"])
def test_package_slab_exchange_gloo(tmp_path, bc, world):
    """paper_1004_5058_gb300.slabs.DistExchange (the host side of the GPU slab
    mode: which message goes to which rank, in which order) over gloo ranks,
    each stepping an oracle slab: the joined state equals the whole-cell oracle
    bit for bit.  With two ranks in a periodic cell each rank is the other's
    neighbour on both sides, so the order of the point-to-point messages alone
    must pair them correctly."""
    import torch.multiprocessing as mp
    from oracle import lb
    from tests.test_oracle_slab import case
    mp.spawn(_dist_exchange_worker, args=(world, free_port(), str(tmp_path), bc), nprocs=world, join=True)
    cell, f = case(bc)
    for _ in range(12):
        f, _, _ = lb.step(cell, f)
    got = np.concatenate([np.load(tmp_path / ("dx_%d.npy" % r)) for r in range(world)], axis=2)
    assert np.array_equal(got, f)


def test_package_slab_exchange_in_process():
    """The same exchange with every slab in one process (LocalExchange), 2 to 4
    slabs (and one slab between the walls of a Couette cell), periodic and
    Couette: equal to the whole-cell oracle bit for bit."""
    from oracle import lb
    from paper_1004_5058_gb300.slabs import LocalExchange, split_rows
    from tests.test_oracle_slab import case
    for bc in (0, 1):
        cell, f0 = case(bc)
        ref = f0
        for _ in range(8):
            ref, _, _ = lb.step(cell, ref)
        for world in ((1, 2, 3, 4) if bc == 1 else (2, 3, 4)):
            parts = split_rows(cell.ny, world)
            slabs = [_OracleSlab(cell, y0, rows, f0) for y0, rows in parts]
            LocalExchange(slabs, periodic=cell.bc == 0).step(8)
            got = np.concatenate([s.f[:, :, 2:rows + 2] for s, (_, rows) in zip(slabs, parts)], axis=2)
            assert np.array_equal(got, ref), (bc, world)


class _PointerLattice:
    """The pointer-level face of a slab handle (lb_slab_get / lb_slab_put into
    buffers given by address, one step per call) over an oracle slab, for the
    stream-ordered exchange, which moves messages between preallocated buffers."""

    stream_ptr = 1  # every slab "on one stream"

    def __init__(self, oslab):
        self.o = oslab

    def slab_get(self, part, ptr):
        import ctypes
        src = np.ascontiguousarray(self.o.f[self.o._where(part, False)])
        ctypes.memmove(ptr, src.ctypes.data, src.nbytes)

    def slab_put(self, part, ptr):
        import ctypes
        shape = self.o.f[self.o._where(part, True)].shape
        n = int(np.prod(shape))
        self.o.f[self.o._where(part, True)] = np.ctypeslib.as_array(
            (ctypes.c_double * n).from_address(ptr)).reshape(shape)

    def step(self, n):
        assert n == 1
        self.o.step()


class _PointerSlab:
    def __init__(self, oslab):
        self.o, self.lat = oslab, _PointerLattice(oslab)

    def empty(self, part):
        return self.o.empty(part)


def test_stream_exchange_pairs_messages_in_process():
    """The one-device exchange without host waits (StreamExchange: one buffer per
    slab and message part, gets of every slab first, then the puts from the
    neighbours' buffers) over oracle slabs: equal to the whole-cell oracle bit for
    bit, 2 to 4 slabs, periodic and Couette."""
    from oracle import lb
    from paper_1004_5058_gb300.slabs import StreamExchange, split_rows
    from tests.test_oracle_slab import case
    for bc in (0, 1):
        cell, f0 = case(bc)
        ref = f0
        for _ in range(8):
            ref, _, _ = lb.step(cell, ref)
        for world in (2, 3, 4):
            parts = split_rows(cell.ny, world)
            oslabs = [_OracleSlab(cell, y0, rows, f0) for y0, rows in parts]
            StreamExchange([_PointerSlab(o) for o in oslabs], periodic=cell.bc == 0).step(8)
            got = np.concatenate([o.f[:, :, 2:rows + 2] for o, (_, rows) in zip(oslabs, parts)], axis=2)
            assert np.array_equal(got, ref), (bc, world)
