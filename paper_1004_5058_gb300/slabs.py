"""One cell split into horizontal slabs: the exchange between slabs around each
time step, on one device or one slab per rank.

A slab holds rows [y0, y0 + rows) of the cell and two ghost rows on each side.
Per time step (the trade the C ABI's lb_slab_get / lb_slab_put perform; see
include/lbhb.h):
  1. edges:  each slab's first two and last two rows (all 18 populations) go
             into the neighbours' ghost rows, because the interaction stencil of
             Eq. (FFF) reaches two rows out;
  2. step:   every slab takes one time step of its own rows;
  3. flows:  the populations that streamed out of a slab (c_y = -1 through its
             lower edge, c_y = +1 through its upper edge) go into the
             neighbours' first or last rows.
The slab below a slab holds the rows just below it; in a periodic cell the
first and last slabs are neighbours, across a Couette wall there is none.

Message naming (both sides use the part of their own edge): what a slab sends
through its lower edge is its *_LO message, and the slab below receives it as
its *_HI part; upwards the other way round.

The exchange only moves opaque messages.  A slab object provides
  get(part) -> message        put(part, message)        step()
  empty(part) -> a receive buffer of the message's size
(SlabLattice below over the CUDA library; the tests also drive an FP64 oracle
slab through the same exchange).  StreamExchange is the one-device form without
host waits: all slabs on one stream, preallocated message buffers.
"""
from __future__ import annotations

from typing import List, Optional, Sequence, Tuple

from . import _lib as L

EDGE_LO, EDGE_HI = L.LB_SLAB_EDGE_LO, L.LB_SLAB_EDGE_HI
FLOW_LO, FLOW_HI = L.LB_SLAB_FLOW_LO, L.LB_SLAB_FLOW_HI


def split_rows(ny: int, world: int) -> List[Tuple[int, int]]:
    """(y0, rows) of each slab, as even as possible (the first ny % world slabs
    one row more)."""
    if world < 1 or ny < 2 * world:
        raise ValueError("cannot split %d rows into %d slabs of at least 2 rows" % (ny, world))
    base, extra = divmod(ny, world)
    out, y0 = [], 0
    for r in range(world):
        rows = base + (1 if r < extra else 0)
        out.append((y0, rows))
        y0 += rows
    return out


def neighbours(periodic: bool, rank: int, world: int) -> Tuple[Optional[int], Optional[int]]:
    """(below, above): the slabs holding the rows below and above slab `rank`
    (slab 0 at the bottom), or None across a Couette wall."""
    below = rank - 1 if rank > 0 else (world - 1 if periodic else None)
    above = rank + 1 if rank < world - 1 else (0 if periodic else None)
    return below, above


class LocalExchange:
    """All slabs of a cell in this process (for instance on one GPU): messages
    move between the slabs' own buffers."""

    def __init__(self, slabs: Sequence, periodic: bool):
        self.slabs = list(slabs)
        self.periodic = periodic

    def _trade(self, lo: int, hi: int):
        world = len(self.slabs)
        links = [neighbours(self.periodic, r, world) for r in range(world)]
        msgs = [(s.get(lo) if b is not None else None, s.get(hi) if a is not None else None)
                for s, (b, a) in zip(self.slabs, links)]
        for s, (below, above) in zip(self.slabs, links):
            if below is not None:
                s.put(lo, msgs[below][1])  # what the slab below sent upwards
            if above is not None:
                s.put(hi, msgs[above][0])  # what the slab above sent downwards

    def step(self, n: int = 1):
        for _ in range(n):
            self._trade(EDGE_LO, EDGE_HI)
            for s in self.slabs:
                s.step()
            self._trade(FLOW_LO, FLOW_HI)
        return self


class DistExchange:
    """One slab per rank, messages over torch.distributed point-to-point (NCCL
    between GPUs with device buffers, gloo with CPU tensors).  Each trade runs
    in two phases, downwards then upwards, so that with two ranks in a periodic
    cell (each the other's neighbour on both sides) the messages between the
    same pair of ranks are matched in posting order without tags."""

    def __init__(self, slab, rank: int, world: int, periodic: bool, group=None):
        self.slab, self.rank, self.world, self.periodic, self.group = slab, rank, world, periodic, group

    def _trade(self, lo: int, hi: int):
        import torch.distributed as dist
        below, above = neighbours(self.periodic, self.rank, self.world)
        if self.world == 1:  # a periodic cell in one slab trades with itself
            if below is not None:
                m_lo, m_hi = self.slab.get(lo), self.slab.get(hi)
                self.slab.put(lo, m_hi)
                self.slab.put(hi, m_lo)
            return
        ops, recv = [], {}
        # downwards: my lower-edge message to the slab below, the slab above's into my upper part
        if below is not None:
            ops.append(dist.P2POp(dist.isend, self.slab.get(lo), below, self.group))
        if above is not None:
            recv[hi] = self.slab.empty(hi)
            ops.append(dist.P2POp(dist.irecv, recv[hi], above, self.group))
        # upwards: my upper-edge message to the slab above, the slab below's into my lower part
        if above is not None:
            ops.append(dist.P2POp(dist.isend, self.slab.get(hi), above, self.group))
        if below is not None:
            recv[lo] = self.slab.empty(lo)
            ops.append(dist.P2POp(dist.irecv, recv[lo], below, self.group))
        if ops:
            for req in dist.batch_isend_irecv(ops):
                req.wait()
        for part, buf in recv.items():
            self.slab.put(part, buf)

    def step(self, n: int = 1):
        for _ in range(n):
            self._trade(EDGE_LO, EDGE_HI)
            self.slab.step()
            self._trade(FLOW_LO, FLOW_HI)
        return self


class StreamExchange:
    """All slabs of a cell on one device and one CUDA stream: every message
    packing, unpacking and time step is stream-ordered, so a step enqueues its
    whole exchange without waiting on the host (the slabs must share the
    stream: SlabLattice(..., stream=s) with one s).  Each slab keeps one
    preallocated device buffer per message part."""

    def __init__(self, slabs: Sequence, periodic: bool):
        self.slabs = list(slabs)
        self.periodic = periodic
        streams = {s.lat.stream_ptr for s in self.slabs}
        if len(streams) != 1:
            raise ValueError("StreamExchange needs every slab on the same stream")
        self.bufs = [{p: s.empty(p) for p in (EDGE_LO, EDGE_HI, FLOW_LO, FLOW_HI)} for s in self.slabs]

    def _trade(self, lo: int, hi: int):
        world = len(self.slabs)
        links = [neighbours(self.periodic, r, world) for r in range(world)]
        for s, b, (below, above) in zip(self.slabs, self.bufs, links):
            if below is not None:
                s.lat.slab_get(lo, b[lo].data_ptr())
            if above is not None:
                s.lat.slab_get(hi, b[hi].data_ptr())
        for s, (below, above) in zip(self.slabs, links):
            if below is not None:
                s.lat.slab_put(lo, self.bufs[below][hi].data_ptr())  # what the slab below sent upwards
            if above is not None:
                s.lat.slab_put(hi, self.bufs[above][lo].data_ptr())  # what the slab above sent downwards

    def step(self, n: int = 1):
        for _ in range(n):
            self._trade(EDGE_LO, EDGE_HI)
            for s in self.slabs:
                s.lat.step(1)
            self._trade(FLOW_LO, FLOW_HI)
        return self


class SlabLattice:
    """A slab of the CUDA library (lb_create_slab) with its messages in torch
    device buffers, for LocalExchange / DistExchange / StreamExchange.  The
    library's copies run on the handle's stream (`stream`: a torch stream or a
    cudaStream_t address; default the library's own); get() waits for them and
    put() waits for the current torch stream first, so messages may be handed
    to other streams, handles or NCCL."""

    def __init__(self, cells, y0: int, rows: int, precision: str = "fp32", device=None, stream=None):
        import torch
        from .lattice import Lattice
        self.torch = torch
        self.device = torch.device("cuda", torch.cuda.current_device()) if device is None else torch.device(device)
        self.lat = Lattice(cells, precision, slab=(y0, rows), stream=stream)
        self.y0, self.rows = y0, rows

    def empty(self, part: int):
        return self.torch.empty(self.lat.message_bytes(part), dtype=self.torch.uint8, device=self.device)

    def get(self, part: int):
        buf = self.empty(part)
        self.torch.cuda.current_stream(self.device).synchronize()  # the buffer's allocation is complete
        self.lat.slab_get(part, buf.data_ptr())
        self.lat.sync()
        return buf

    def put(self, part: int, buf):
        self.torch.cuda.current_stream(self.device).synchronize()  # a received message has landed
        self.lat.slab_put(part, buf.data_ptr())

    def step(self):
        self.lat.step(1)

    def close(self):
        self.lat.close()
