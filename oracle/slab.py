"""Decomposition of one cell into horizontal slabs over host ranks, each rank
stepping its slab with the oracle (orc_step_slab) and trading two kinds of
rows with its neighbours every step.

TEST INFRASTRUCTURE ONLY: this is the plain statement of the exchange a split
of one large cell over several devices needs (the paper runs a single lattice;
the split is ours), pinned by being equal bit for bit to the whole-cell oracle.

Per step, rank r owning rows [y0, y0 + rows):
  1. ghost rows: rows y0-2, y0-1 come from the rank below, rows y0+rows,
     y0+rows+1 from the rank above (all 18 populations), because the interaction
     stencil of Eq. (FFF) reaches two rows out; a Couette wall has no rank
     beyond it (the stencil mirrors into the cell there);
  2. the slab step (moments, forces, collision, streaming);
  3. inflow: the populations with c_y = +1 that the rank below streamed out of
     its top row land in this slab's first row, those with c_y = -1 from the rank
     above in its last row.

A slab array has shape [2, 9, rows + 4, nx]: slab row e is global row y0-2+e.
Every rank needs rows >= 2 so that its ghost rows come from one neighbour.
"""
from __future__ import annotations

import ctypes as C

import numpy as np

from . import lb

UP = (2, 5, 6)    # D2Q9 directions with c_y = +1
DOWN = (4, 7, 8)  # c_y = -1


def split_rows(ny: int, world: int):
    """(y0, rows) per rank, as even as possible, the first ny % world ranks one row more."""
    base, extra = divmod(ny, world)
    out, y0 = [], 0
    for r in range(world):
        rows = base + (1 if r < extra else 0)
        out.append((y0, rows))
        y0 += rows
    return out


def neighbours(cell, rank: int, world: int):
    """(below, above): the ranks owning the rows below and above the slab, or
    None across a Couette wall."""
    periodic = cell.bc == 0
    below = rank - 1 if rank > 0 else (world - 1 if periodic else None)
    above = rank + 1 if rank < world - 1 else (0 if periodic else None)
    return below, above


def _lib():
    L = lb.lib()
    if not getattr(L, "_slab_ready", False):
        P = C.POINTER(lb.Params)
        L.orc_step_slab.argtypes = [P, C.c_int, C.c_int, lb._DP, lb._DP, C.POINTER(lb.Obs), C.c_void_p]
        L.orc_step_slab.restype = C.c_int
        L._slab_ready = True
    return L


def scatter(f: np.ndarray, y0: int, rows: int):
    """Slab array of rows [y0, y0+rows) of a whole-cell population array (ghost rows zero)."""
    nx = f.shape[-1]
    s = np.zeros((2, 9, rows + 4, nx))
    s[:, :, 2:rows + 2] = f[:, :, y0:y0 + rows]
    return s


def gather(slabs, ny: int):
    nx = slabs[0].shape[-1]
    f = np.empty((2, 9, ny, nx))
    y = 0
    for s in slabs:
        rows = s.shape[2] - 4
        f[:, :, y:y + rows] = s[:, :, 2:rows + 2]
        y += rows
    return f


# ---- what a rank sends and how it places what it receives ------------------
def ghost_send(f_slab):
    """(to_below, to_above): the slab's first two and last two rows."""
    rows = f_slab.shape[2] - 4
    return f_slab[:, :, 2:4].copy(), f_slab[:, :, rows:rows + 2].copy()


def ghost_recv(f_slab, from_below, from_above):
    rows = f_slab.shape[2] - 4
    if from_below is not None:
        f_slab[:, :, 0:2] = from_below
    if from_above is not None:
        f_slab[:, :, rows + 2:rows + 4] = from_above


def outflow_send(out_slab):
    """(to_below, to_above): the c_y = -1 populations streamed into slab row 1
    and the c_y = +1 ones streamed into slab row rows+2."""
    rows = out_slab.shape[2] - 4
    return out_slab[:, list(DOWN), 1].copy(), out_slab[:, list(UP), rows + 2].copy()


def inflow_recv(out_slab, from_below, from_above):
    rows = out_slab.shape[2] - 4
    if from_below is not None:
        out_slab[:, list(UP), 2] = from_below
    if from_above is not None:
        out_slab[:, list(DOWN), rows + 1] = from_above


def step_slab(cell, y0: int, f_slab: np.ndarray, want_obs: bool = False):
    """orc_step_slab on one slab (ghost rows already filled).  Returns
    (out slab, obs dict or None)."""
    rows = f_slab.shape[2] - 4
    f_slab = np.ascontiguousarray(f_slab, dtype=np.float64)
    out = np.zeros_like(f_slab)
    o = lb.Obs()
    rc = _lib().orc_step_slab(C.byref(lb.params(cell)), int(y0), int(rows), f_slab, out,
                              C.byref(o) if want_obs else None, None)
    if rc != 0:
        raise ValueError("slab [%d, %d) does not fit the cell" % (y0, y0 + rows))
    return out, (lb.obs_dict(o) if want_obs else None)


def run_in_process(cell, f: np.ndarray, n_steps: int, world: int):
    """n_steps of the whole cell as `world` slab ranks stepped one after the
    other in this process, exchanging through plain copies.  Returns the
    whole-cell population array and the last step's observables summed over
    ranks."""
    parts = split_rows(cell.ny, world)
    if min(r for _, r in parts) < 2:
        raise ValueError("every rank needs at least two rows")
    slabs = [scatter(f, y0, rows) for y0, rows in parts]
    obs = None
    for t in range(n_steps):
        sends = [ghost_send(s) for s in slabs]
        for r in range(world):
            below, above = neighbours(cell, r, world)
            ghost_recv(slabs[r], None if below is None else sends[below][1],
                       None if above is None else sends[above][0])
        results = [step_slab(cell, parts[r][0], slabs[r], want_obs=(t == n_steps - 1)) for r in range(world)]
        outs = [o for o, _ in results]
        flows = [outflow_send(o) for o in outs]
        for r in range(world):
            below, above = neighbours(cell, r, world)
            inflow_recv(outs[r], None if below is None else flows[below][1],
                        None if above is None else flows[above][0])
        slabs = outs
        if t == n_steps - 1:
            obs = {k: tuple(np.sum([res[1][k] for res in results], axis=0).tolist())
                   if isinstance(results[0][1][k], tuple) else float(sum(res[1][k] for res in results))
                   for k in results[0][1]}
    return gather(slabs, cell.ny), obs
