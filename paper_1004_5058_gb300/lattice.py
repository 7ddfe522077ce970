"""Python front end of the C ABI: a handle of one or more lattice cells.

Thin marshalling over liblbhb.so (see include/lbhb.h for the meaning of every
call); numpy arrays in and out, float64 host fields laid out [cell][y][x].
"""
from __future__ import annotations

import ctypes as C
from typing import Iterable, Optional

import numpy as np

from . import _lib as L
from .inputs import CellParams

PRECISIONS = {"fp32": L.LB_FP32, "fp16": L.LB_FP16_SHIFTED, "fp16_shifted": L.LB_FP16_SHIFTED, "fp64": L.LB_FP64,
              "fp16sr": L.LB_FP16_SHIFTED_SR}
KERNELS = {"auto": L.LB_KERNEL_AUTO, "generic": L.LB_KERNEL_GENERIC, "tiled": L.LB_KERNEL_TILED}
KERNEL_NAMES = {v: k for k, v in KERNELS.items()}


def _dp(a):
    return None if a is None else a.ctypes.data_as(L._D)


def _stream_ptr(stream) -> Optional[int]:
    if stream is None:
        return None
    if isinstance(stream, int):
        return stream or None
    return int(stream.cuda_stream) or None  # torch.cuda.Stream / ExternalStream


def cell_struct(c: CellParams) -> L.lb_cell_params:
    return L.lb_cell_params(c.nx, c.ny, c.tau, c.rho0, c.g_aa1, c.g_aa2, c.g_bb1, c.g_bb2, c.g_ab,
                            c.u_wall, getattr(c, "f0", 0.0), c.rho_bar_a, c.rho_bar_b, c.bc,
                            getattr(c, "tau_b", 0.0), getattr(c, "s_e", 0.0), getattr(c, "s_eps", 0.0),
                            getattr(c, "s_q", 0.0), getattr(c, "s_nu", 0.0))


class Lattice:
    """n_cells independent cells advanced together (lb_create .. lb_destroy).

    slab=(y0, rows): a handle over rows [y0, y0 + rows) of each cell only, one
    slab of a cell split along y (lb_create_slab); host arrays then cover the own
    rows ([n_cells][rows][nx]), and the slab trades rows with its neighbours
    between steps (paper_1004_5058_gb300.slabs)."""

    def __init__(self, cells: Iterable[CellParams], precision: str = "fp32", stream=None, slab=None):
        self.lib = L.load()
        self.cells = list(cells)
        self.n_cells = len(self.cells)
        self.nx, self.ny = self.cells[0].nx, self.cells[0].ny
        self.ny_global = self.ny
        self.slab = None if slab is None else (int(slab[0]), int(slab[1]))
        self.precision = precision
        arr = (L.lb_cell_params * self.n_cells)(*[cell_struct(c) for c in self.cells])
        h = L._H()
        if self.slab is None:
            st = self.lib.lb_create(arr, self.n_cells, PRECISIONS[precision], _stream_ptr(stream), C.byref(h))
        else:
            st = self.lib.lb_create_slab(arr, self.n_cells, PRECISIONS[precision], self.slab[0], self.slab[1],
                                         _stream_ptr(stream), C.byref(h))
            self.ny = self.slab[1]
        L.check(st, None)
        self.h = h

    # ---- slab exchange (lb_slab_*): messages in the caller's device buffers
    def message_bytes(self, part: int) -> int:
        n = C.c_size_t()
        self._chk(self.lib.lb_slab_message_bytes(self.h, int(part), C.byref(n)))
        return int(n.value)

    def slab_get(self, part: int, dst_ptr: int):
        """Packs the message `part` into device memory at dst_ptr (stream-ordered)."""
        self._chk(self.lib.lb_slab_get(self.h, int(part), C.c_void_p(int(dst_ptr))))
        return self

    def slab_put(self, part: int, src_ptr: int):
        """Unpacks the message `part` from device memory at src_ptr (stream-ordered)."""
        self._chk(self.lib.lb_slab_put(self.h, int(part), C.c_void_p(int(src_ptr))))
        return self

    def wall_momentum(self):
        """Time sums [n_cells][2] of the x-momentum delivered by the top and
        bottom walls over the sampled steps, and the number of sampled steps."""
        s = np.empty((self.n_cells, 2))
        n = C.c_longlong()
        self._chk(self.lib.lb_wall_momentum(self.h, _dp(s), C.byref(n)))
        return s, n.value

    # ---- life cycle
    def close(self):
        if getattr(self, "h", None):
            self.lib.lb_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    def _chk(self, st):
        return L.check(st, self.h)

    def _field(self, a):
        if a is None:
            return None
        a = np.ascontiguousarray(a, dtype=np.float64)
        a = a.reshape(self.n_cells, self.ny, self.nx)
        return a

    # ---- state
    def init_fields(self, rho_a, rho_b, ux=None, uy=None):
        ra, rb, u, v = (self._field(a) for a in (rho_a, rho_b, ux, uy))
        self._chk(self.lib.lb_init_fields(self.h, _dp(ra), _dp(rb), _dp(u), _dp(v)))
        return self

    def stage_fields(self, rho_a, rho_b, ux=None, uy=None):
        """Start the host-to-device copy of the next run's fields on the handle's
        copy stream (lb_stage_fields) and return; init_fields_staged() then
        sets f = f^eq from them.  The arrays are held here until then; pass
        page-locked arrays for an asynchronous copy."""
        arrs = tuple(self._field(a) for a in (rho_a, rho_b, ux, uy))
        self._chk(self.lib.lb_stage_fields(self.h, *(_dp(a) for a in arrs)))
        self._staged_refs = arrs
        return self

    def init_fields_staged(self):
        """f = f^eq of the staged fields, enqueued without synchronising
        (lb_init_fields_staged); counters reset as in init_fields."""
        self._chk(self.lib.lb_init_fields_staged(self.h))
        self._staged_refs = None
        return self

    def set_populations(self, f):
        f = np.ascontiguousarray(f, dtype=np.float64).reshape(self.n_cells, 2, 9, self.ny, self.nx)
        self._chk(self.lib.lb_set_populations(self.h, _dp(f)))
        return self

    def save(self, path: str):
        """Checkpoint of the whole state (lb_save): populations bit for bit, time
        step, sampling window and time sums, cell parameters."""
        self._chk(self.lib.lb_save(self.h, str(path).encode()))
        return self

    def load(self, path: str):
        """Resume from a checkpoint written by save() on a handle of the same
        shape and precision (lb_load)."""
        self._chk(self.lib.lb_load(self.h, str(path).encode()))
        return self

    def get_populations(self):
        f = np.empty((self.n_cells, 2, 9, self.ny, self.nx))
        self._chk(self.lib.lb_get_populations(self.h, _dp(f)))
        return f

    def step(self, n: int):
        self._chk(self.lib.lb_step(self.h, int(n)))
        return self

    def sync(self):
        self._chk(self.lib.lb_sync(self.h))
        return self

    # ---- observables
    def set_sampling(self, start: int, every: int):
        self._chk(self.lib.lb_set_sampling(self.h, int(start), int(every)))
        return self

    def shear_stress(self):
        s = np.empty(self.n_cells)
        r = np.empty(self.n_cells)
        b = np.empty(self.n_cells)
        self._chk(self.lib.lb_shear_stress(self.h, _dp(s), _dp(r), _dp(b)))
        return s, r, b

    def profile(self):
        u = np.empty((self.n_cells, self.ny))
        n = C.c_longlong()
        self._chk(self.lib.lb_get_profile(self.h, _dp(u), C.byref(n)))
        return u, n.value

    def fields(self):
        out = [np.empty((self.n_cells, self.ny, self.nx)) for _ in range(4)]
        self._chk(self.lib.lb_get_fields(self.h, *[_dp(o) for o in out]))
        return tuple(out)

    def reductions(self):
        m = np.empty((self.n_cells, 2))
        p = np.empty((self.n_cells, 2))
        self._chk(self.lib.lb_reductions(self.h, _dp(m), _dp(p)))
        return m, p

    # ---- kernels
    def set_kernel(self, kind: str = "auto", tile_x: int = 0, tile_y: int = 0):
        self._chk(self.lib.lb_set_kernel(self.h, KERNELS[kind], int(tile_x), int(tile_y)))
        return self

    def kernel(self):
        k, tx, ty = C.c_int(), C.c_int(), C.c_int()
        self._chk(self.lib.lb_get_kernel(self.h, C.byref(k), C.byref(tx), C.byref(ty)))
        return KERNEL_NAMES[k.value], tx.value, ty.value

    def launch_shape(self):
        """(CTAs of plain steps, CTAs of sampled steps, threads, shared memory
        bytes) of the tiled kernel in use, or None for the generic kernel."""
        v = [C.c_int() for _ in range(4)]
        st = self.lib.lb_launch_shape(self.h, *[C.byref(x) for x in v])
        if st == L.LB_ERR_UNSUPPORTED:
            return None
        self._chk(st)
        return tuple(x.value for x in v)

    def autotune(self, cache_path: Optional[str] = None):
        self._chk(self.lib.lb_autotune(self.h, cache_path.encode() if cache_path else None))
        return self.kernel()

    @property
    def steps_done(self) -> int:
        return int(self.lib.lb_steps_done(self.h))

    @property
    def kernel_launches(self) -> int:
        return int(self.lib.lb_kernel_launches(self.h))

    @property
    def stream_ptr(self) -> int:
        return int(self.lib.lb_stream(self.h) or 0)


def hb_fit(shear_rate, sigma, beta_lo: float = 0.02, beta_hi: float = 3.0):
    """Herschel-Bulkley fit sigma = sigma_Y + A S^beta (lb_hb_fit)."""
    S = np.ascontiguousarray(shear_rate, dtype=np.float64)
    sg = np.ascontiguousarray(sigma, dtype=np.float64)
    out = np.empty(4)
    L.check(L.load().lb_hb_fit(_dp(S), _dp(sg), int(S.size), float(beta_lo), float(beta_hi), _dp(out)))
    return dict(sigma_y=float(out[0]), A=float(out[1]), beta=float(out[2]), rss=float(out[3]))
