"""Seeded synthetic inputs shared by the CUDA path's tests/bench and by the oracle.

This module holds no arithmetic of the lattice Boltzmann method itself: it only
draws the initial density/velocity fields and the coupling presets that both
sides receive as plain arrays.

Random numbers: SplitMix64 (Steele, Lea and Flood, "Fast splittable pseudorandom
number generators", OOPSLA 2014), used in counter form: output k of a stream with
seed s is mix(s + (k+1)*0x9E3779B97F4A7C15), mix being the SplitMix64 finaliser.
A uniform double in [0,1) is the top 53 bits times 2**-53.  Site order inside a
field is y-major ([cell][y][x], x fastest).
"""
from __future__ import annotations

import math
from dataclasses import dataclass, asdict

import numpy as np

_GAMMA = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)


def splitmix64(seed: int, n: int, offset: int = 0) -> np.ndarray:
    """Outputs offset..offset+n-1 of the SplitMix64 stream with the given seed."""
    k = np.arange(offset + 1, offset + n + 1, dtype=np.uint64)
    with np.errstate(over="ignore"):
        z = np.uint64(seed & 0xFFFFFFFFFFFFFFFF) + k * _GAMMA
        z = (z ^ (z >> np.uint64(30))) * _M1
        z = (z ^ (z >> np.uint64(27))) * _M2
        z = z ^ (z >> np.uint64(31))
    return z


def uniform01(seed: int, n: int, offset: int = 0) -> np.ndarray:
    """Uniform doubles in [0, 1) from the top 53 bits of SplitMix64."""
    return (splitmix64(seed, n, offset) >> np.uint64(11)).astype(np.float64) * (2.0 ** -53)


@dataclass
class CellParams:
    """One lattice cell, in the paper's symbols (Eq. (be), Eq. (FFF), footnote of
    the Numerical Results section).

    g_aa1/g_bb1: G^a_ss (belt 1, attractive when negative); g_aa2/g_bb2: G^r_ss
    (belts 1+2, repulsive when positive); g_ab: G_AB (belt 1, cross species).
    bc: 0 = fully periodic, 1 = Couette (periodic x, moving walls at y=-1/2 and
    y=ny-1/2 with x-velocities -u_wall and +u_wall).
    f0: Kolmogorov body force F_x(y) = f0 sin(2 pi y / ny) (section "Numerical
    Results"), shared by the species in proportion to their density.
    rho_bar_a/b: reference densities of the FP16 shifted storage f_i - w_i*rho_bar.
    tau_b: relaxation time of species B, 0 for tau (the paper uses one time,
    tau = 1, and leaves a coupling-dependent one unexplored); tau is species A's.
    s_e, s_eps, s_q, s_nu: rates of a multiple-relaxation-time collision
    (Lallemand and Luo's orthogonal D2Q9 moments e, eps, q_x/q_y, p_xx/p_xy; not
    in the paper), each 0 for 1/tau_s; all 0 is the paper's BGK collision.  The
    density and momentum moments always relax with 1/tau_s, so tau_s still sets
    the force shift, and s_nu sets the shear viscosity (1/s_nu - 1/2)/3.
    """
    nx: int = 64
    ny: int = 64
    tau: float = 1.0
    rho0: float = 0.83
    g_aa1: float = -9.0
    g_aa2: float = 8.1
    g_bb1: float = -8.0
    g_bb2: float = 7.1
    g_ab: float = 0.045
    u_wall: float = 0.0
    f0: float = 0.0
    rho_bar_a: float = 0.6
    rho_bar_b: float = 0.6
    bc: int = 0
    tau_b: float = 0.0
    s_e: float = 0.0
    s_eps: float = 0.0
    s_q: float = 0.0
    s_nu: float = 0.0

    def as_dict(self):
        return asdict(self)


# Coupling presets.  "paper": the footnote of the Numerical Results section
# (G^a_AA=-9, G^r_AA=8.1, G^a_BB=-8, G^r_BB=7.1, G_AB=0.045, tau=1).
# "symmetric": equal A/B couplings -9/8.1 and G_AB=0.405 (the value a dropped
# digit in the footnote would give); used where a symmetric pair of species is wanted.
PRESETS = {
    "paper": dict(g_aa1=-9.0, g_aa2=8.1, g_bb1=-8.0, g_bb2=7.1, g_ab=0.045, tau=1.0, rho0=0.83),
    "symmetric": dict(g_aa1=-9.0, g_aa2=8.1, g_bb1=-9.0, g_bb2=8.1, g_ab=0.405, tau=1.0, rho0=0.83),
    "ideal": dict(g_aa1=0.0, g_aa2=0.0, g_bb1=0.0, g_bb2=0.0, g_ab=0.0, tau=1.0, rho0=0.83),
}


def make_cell(preset: str = "paper", **over) -> CellParams:
    kw = dict(PRESETS[preset])
    kw.update(over)
    return CellParams(**kw)


def random_fields(nx: int, ny: int, n_cells: int = 1, rho_bar: float = 0.6,
                  amp: float = 0.1, seed: int = 1004):
    """rho_A = rho_bar(1 + amp*xi), rho_B = rho_bar(1 - amp*xi), xi ~ U[-1,1] per
    site, drawn once from one SplitMix64 stream over [cell][y][x].
    Returns (rho_a, rho_b) as float64 arrays of shape [n_cells, ny, nx]."""
    n = n_cells * ny * nx
    xi = 2.0 * uniform01(seed, n) - 1.0
    xi = xi.reshape(n_cells, ny, nx)
    return rho_bar * (1.0 + amp * xi), rho_bar * (1.0 - amp * xi)


def couette_velocity(nx: int, ny: int, u_wall, n_cells: int = 1):
    """Linear Couette start u_x(y) = U (2 (y + 1/2)/ny - 1), u_y = 0, for walls at
    y=-1/2 (velocity -U) and y=ny-1/2 (velocity +U).  u_wall: scalar or one per cell."""
    u = np.broadcast_to(np.asarray(u_wall, dtype=np.float64), (n_cells,)).copy()
    y = np.arange(ny, dtype=np.float64)
    prof = 2.0 * (y + 0.5) / ny - 1.0
    ux = u[:, None, None] * prof[None, :, None] * np.ones((1, 1, nx))
    return ux, np.zeros_like(ux)


def sine_fields(nx: int, ny: int, n_cells: int = 1, noise: float = 0.0, seed: int = 1004):
    """The paper's initial state (Numerical Results): rho_A = 0.61(1+0.1 sin(k y)),
    rho_B = 0.61(1+0.01 sin(k y)), k = 64*pi/L with L = ny.

    That state is invariant under translations in x, and so is every later state
    of an update that treats all columns with the same arithmetic: the lamellae
    never break up into the droplets the paper shows.  noise > 0 multiplies each
    density by (1 + noise xi), xi uniform in [-1, 1) from the SplitMix64 stream
    (species A then B, cell-major, y-major), to break that symmetry."""
    k = 64.0 * math.pi / ny
    y = np.arange(ny, dtype=np.float64)
    ra = 0.61 * (1.0 + 0.1 * np.sin(k * y))
    rb = 0.61 * (1.0 + 0.01 * np.sin(k * y))
    shape = (n_cells, ny, nx)
    ra = np.broadcast_to(ra[None, :, None], shape).copy()
    rb = np.broadcast_to(rb[None, :, None], shape).copy()
    if noise > 0.0:
        n = n_cells * nx * ny
        xi = 2.0 * uniform01(seed, 2 * n) - 1.0
        ra *= 1.0 + noise * xi[:n].reshape(shape)
        rb *= 1.0 + noise * xi[n:].reshape(shape)
    return ra, rb


def kolmogorov_f0(u0: float, ny: int, rho: float = 1.22, tau: float = 1.0) -> float:
    """Forcing amplitude of a laminar Kolmogorov flow of peak speed u0:
    F0 = rho nu k^2 u0, nu = (tau - 1/2)/3, k = 2 pi / ny (the paper tunes F0 to
    produce u0 = 0.1 in standard stationary conditions)."""
    k = 2.0 * math.pi / ny
    return rho * (tau - 0.5) / 3.0 * k * k * u0


def log_spaced(lo: float, hi: float, n: int):
    """n values log-spaced from lo to hi inclusive (10**(a + (b-a) k/(n-1)))."""
    a, b = math.log10(lo), math.log10(hi)
    return [10.0 ** (a + (b - a) * k / (n - 1)) for k in range(n)]
