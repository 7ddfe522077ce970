"""ctypes front end of the FP64 C oracle (oracle/lb_oracle.c).

TEST INFRASTRUCTURE ONLY: used by tests, the smoke check and the CPU-baseline
leg of the benchmark.  Arrays are float64 numpy arrays; a population array has
shape [2, 9, ny, nx] (species, D2Q9 direction, y, x).  See lb_oracle.c for the
equations each function follows.
"""
from __future__ import annotations

import ctypes as C

import numpy as np

from .build import build_oracle

_lib = None


class Params(C.Structure):
    _fields_ = [("nx", C.c_int), ("ny", C.c_int), ("tau", C.c_double), ("rho0", C.c_double),
                ("g_aa1", C.c_double), ("g_aa2", C.c_double), ("g_bb1", C.c_double),
                ("g_bb2", C.c_double), ("g_ab", C.c_double), ("u_wall", C.c_double),
                ("f0", C.c_double), ("bc", C.c_int), ("tau_b", C.c_double),
                ("s_e", C.c_double), ("s_eps", C.c_double), ("s_q", C.c_double), ("s_nu", C.c_double)]


class Obs(C.Structure):
    _fields_ = [("mass", C.c_double * 2), ("mom", C.c_double * 2),
                ("pi_top", C.c_double), ("pi_bot", C.c_double)]


class Acc(C.Structure):
    _fields_ = [("sum_pi_top", C.c_double), ("sum_pi_bot", C.c_double),
                ("n_samples", C.c_longlong)]


_DP = np.ctypeslib.ndpointer(dtype=np.float64, flags="C_CONTIGUOUS")


def lib():
    global _lib
    if _lib is None:
        L = C.CDLL(build_oracle())
        P = C.POINTER(Params)
        L.orc_equilibrium.argtypes = [P, _DP, _DP, C.c_void_p, C.c_void_p, _DP]
        L.orc_moments.argtypes = [P, _DP, C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p]
        L.orc_forces.argtypes = [P, _DP, _DP, C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p]
        L.orc_step.argtypes = [P, _DP, _DP, C.POINTER(Obs), C.c_void_p]
        L.orc_run.argtypes = [P, _DP, C.c_longlong, C.c_longlong, C.c_longlong, C.c_longlong,
                              C.POINTER(Acc), C.c_void_p, C.POINTER(Obs), C.c_int]
        L.orc_belt_weight.argtypes = [C.c_int, C.c_int, C.c_int]
        L.orc_belt_weight.restype = C.c_double
        L.orc_max_threads.restype = C.c_int
        _lib = L
    return _lib


def _ptr(a):
    return None if a is None else a.ctypes.data_as(C.c_void_p)


def params(cell) -> Params:
    """Params from an inputs.CellParams (or any object with the same fields)."""
    return Params(cell.nx, cell.ny, cell.tau, cell.rho0, cell.g_aa1, cell.g_aa2, cell.g_bb1,
                  cell.g_bb2, cell.g_ab, cell.u_wall, getattr(cell, "f0", 0.0), cell.bc,
                  getattr(cell, "tau_b", 0.0), getattr(cell, "s_e", 0.0), getattr(cell, "s_eps", 0.0),
                  getattr(cell, "s_q", 0.0), getattr(cell, "s_nu", 0.0))


def _f64(a, shape):
    a = np.ascontiguousarray(a, dtype=np.float64)
    assert a.shape == shape, (a.shape, shape)
    return a


def equilibrium(cell, rho_a, rho_b, ux=None, uy=None):
    """f_is = f^eq_is(rho_s, u) (D2Q9, cs^2 = 1/3)."""
    sh = (cell.ny, cell.nx)
    ra, rb = _f64(rho_a, sh), _f64(rho_b, sh)
    ux = None if ux is None else _f64(ux, sh)
    uy = None if uy is None else _f64(uy, sh)
    f = np.empty((2, 9, cell.ny, cell.nx))
    lib().orc_equilibrium(C.byref(params(cell)), ra, rb, _ptr(ux), _ptr(uy), f)
    return f


def moments(cell, f):
    """(rho_a, rho_b, jx, jy), each [ny, nx]."""
    f = _f64(f, (2, 9, cell.ny, cell.nx))
    out = [np.empty((cell.ny, cell.nx)) for _ in range(4)]
    lib().orc_moments(C.byref(params(cell)), f, *[_ptr(o) for o in out])
    return tuple(out)


def forces(cell, rho_a, rho_b):
    """Eq. (FFF) forces (fax, fay, fbx, fby) from given density fields."""
    sh = (cell.ny, cell.nx)
    ra, rb = _f64(rho_a, sh), _f64(rho_b, sh)
    out = [np.empty(sh) for _ in range(4)]
    lib().orc_forces(C.byref(params(cell)), ra, rb, *[_ptr(o) for o in out])
    return tuple(out)


def step(cell, f, want_profile=False):
    """One step of Eq. (be).  Returns (f_next, obs dict, profile or None)."""
    f = _f64(f, (2, 9, cell.ny, cell.nx))
    g = np.empty_like(f)
    o = Obs()
    prof = np.empty(cell.ny) if want_profile else None
    lib().orc_step(C.byref(params(cell)), f, g, C.byref(o), _ptr(prof))
    return g, obs_dict(o), prof


def obs_dict(o: Obs):
    return dict(mass=(o.mass[0], o.mass[1]), mom=(o.mom[0], o.mom[1]),
                pi_top=o.pi_top, pi_bot=o.pi_bot)


class Run:
    """A running oracle lattice: f plus the time averages of sampled steps."""

    def __init__(self, cell, rho_a, rho_b, ux=None, uy=None, threads=0):
        self.cell = cell
        self.f = equilibrium(cell, rho_a, rho_b, ux, uy)
        self.t = 0
        self.start, self.every = 0, 0
        self.acc = Acc(0.0, 0.0, 0)
        self.prof = np.zeros(cell.ny)
        self.threads = threads
        self.last = None

    def set_sampling(self, start, every):
        self.start, self.every = int(start), int(every)

    def step(self, n):
        o = Obs()
        lib().orc_run(C.byref(params(self.cell)), self.f, self.t, int(n), self.start, self.every,
                      C.byref(self.acc), _ptr(self.prof), C.byref(o), int(self.threads))
        self.t += int(n)
        self.last = obs_dict(o)
        return self

    def fields(self):
        """(rho_a, rho_b, ux, uy) with u = j / (rho_a + rho_b) (the paper's u)."""
        ra, rb, jx, jy = moments(self.cell, self.f)
        r = ra + rb
        return ra, rb, jx / r, jy / r

    def shear(self):
        """(sigma_xy, S, S_bulk, Ubar profile).  sigma = (Pi_top - Pi_bot)/(2 nx n_samples);
        Ubar(y) = time average of sum_x u_phys_x / nx; S = (Ubar(ny-1) - Ubar(0))/(ny-1);
        S_bulk = least-squares slope of Ubar over the central half of the rows."""
        n = self.acc.n_samples
        nx, ny = self.cell.nx, self.cell.ny
        if n == 0:
            return float("nan"), float("nan"), float("nan"), None
        sigma = 0.5 * (self.acc.sum_pi_top - self.acc.sum_pi_bot) / (nx * n)
        ub = self.prof / (nx * n)
        S = (ub[ny - 1] - ub[0]) / (ny - 1)
        lo, hi = ny // 4, ny - ny // 4
        y = np.arange(lo, hi, dtype=np.float64)
        yc = y - y.mean()
        S_bulk = float(np.sum(yc * ub[lo:hi]) / np.sum(yc * yc))
        return float(sigma), float(S), S_bulk, ub


def belt_weight(belt, cx, cy):
    return lib().orc_belt_weight(belt, cx, cy)


def max_threads():
    return lib().orc_max_threads()
